// Backward pass of the object-aware rasterizer (Eqs. 1-2) for the map
// refinement of the NBV loop: given the gradient of a loss with respect to
// every pixel's colour C, depth D, opacity A and object channels O, the
// gradient with respect to each Gaussian's projected quantities
//   u = (mean2D, conic A B C, sigma), colour, camera depth z, probabilities p.
//
// One thread block per tile, one thread per pixel (8 x 4 pixels per warp).
// The forward pass is recomputed per tile with the same decisions (no
// per-pixel lists are stored): it gives each pixel's final transmittance
// T_f and the end of its blended list. The backward pass then walks the
// list back to front. With T_i the transmittance before splat i,
// w_i = alpha_i T_i, and the pixel's loss-weighted value of a splat
//   s_i = g_C . c_i + g_D z_i + sum_{k >= 1} (g_O_k - g_O_0) p_ik
// (O_0 = 1 - sum_{k >= 1} O'_k, so channel 0 passes its gradient to the
// others with a minus sign and none to p_i0), the suffix
// S_i = sum_{j > i} w_j s_j gives
//   dL / d alpha_i = T_i s_i - S_i / (1 - alpha_i) + g_A T_f / (1 - alpha_i)
// and, unless alpha_i was clamped, with alpha = sigma exp(p),
//   dL/dmean2D = dL/dalpha alpha (-(A dx + B dy), -(B dx + C dy)),
//   dL/d(A, B, C) = dL/dalpha alpha (-dx^2/2, -dx dy, -dy^2/2),
//   dL/dsigma = dL/dalpha alpha / sigma;
// dL/dc_i = w_i g_C, dL/dz_i = w_i g_D, dL/dp_ik = w_i (g_O_k - g_O_0).
// Contributions are summed over the warp by shuffles, over the tile in
// shared memory and added to the Gaussian's accumulator once per
// (tile, Gaussian).
#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kBB = 32;   // Gaussians staged per round

template <int KCM>
__global__ void __launch_bounds__(kTilePix) k_render_backward(BackwardArgs a, Consts c) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int KC = c.KC, GW = a.gw;
  float4* s0 = reinterpret_cast<float4*>(smem);
  float4* s1 = s0 + kBB;
  float4* s2 = s1 + kBB;
  int* sid = reinterpret_cast<int*>(s2 + kBB);
  float* sp = reinterpret_cast<float*>(sid + kBB);       // [kBB][KC]
  float* gacc = sp + kBB * KC;                           // [kBB][GW]
  __shared__ int s_last_max;
  const DevCam& cam = a.cam;
  const int tile = blockIdx.x;
  const int tx = tile % cam.GX, ty = tile / cam.GX;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  const int wx = cam.TW >> 3;
  const int px = tx * cam.TW + 8 * (wq % wx) + (lane & 7), py = ty * cam.TH + 4 * (wq / wx) + (lane >> 3);
  const bool inside = px < cam.W && py < cam.H;
  const float pxc = __fadd_rn((float)px, 0.5f), pyc = __fadd_rn((float)py, 0.5f);
  const uint2 rg = a.ranges[tile];

  // forward recomputation: final transmittance and the end of the blended list
  float T = 1.0f;
  uint32_t last = rg.x;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += kBB) {
    if (__syncthreads_count(done) == kTilePix) break;
    const uint32_t nj = min((uint32_t)kBB, rg.y - start);
    if (tid < (int)nj) {
      const uint32_t g = a.vals[start + tid];
      s0[tid] = a.r0[g];
      s1[tid] = a.r1[g];
    }
    __syncthreads();
    if (!done) {
      for (uint32_t j = 0; j < nj; ++j) {
        const float4 a0 = s0[j], a1 = s1[j];
        const float pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
        if (pw > 0.0f || pw < a0.z) continue;
        const float alpha = (pw >= a0.w) ? c.alpha_max : a1.w * expf(pw);
        const float tt = T * (1.0f - alpha);
        if (tt < c.t_min) { done = true; break; }
        T = tt;
        last = start + j + 1;
      }
    }
  }
  if (tid == 0) s_last_max = (int)rg.x;
  __syncthreads();
  if (inside) atomicMax(&s_last_max, (int)last);
  __syncthreads();
  const uint32_t last_max = (uint32_t)s_last_max;

  // this pixel's output gradients
  float gc0 = 0.0f, gc1 = 0.0f, gc2 = 0.0f, gd = 0.0f, ga = 0.0f;
  float go[KCM];
#pragma unroll
  for (int k = 0; k < KCM; ++k) go[k] = 0.0f;
  if (inside) {
    const size_t pix = (size_t)py * cam.W + px;
    if (a.g_rgb) { gc0 = a.g_rgb[3 * pix]; gc1 = a.g_rgb[3 * pix + 1]; gc2 = a.g_rgb[3 * pix + 2]; }
    if (a.g_depth) gd = a.g_depth[pix];
    if (a.g_alpha) ga = a.g_alpha[pix];
    if (a.g_obj) {
      const float g0 = a.g_obj[pix * KC];
#pragma unroll
      for (int k = 1; k < KCM; ++k)
        if (k < KC) go[k] = a.g_obj[pix * KC + k] - g0;
    }
  }
  const float Tf = T;
  float Tb = T, S = 0.0f;
  for (uint32_t end = last_max; end > rg.x;) {
    const uint32_t start = (end - rg.x > (uint32_t)kBB) ? end - kBB : rg.x;
    const int nj = (int)(end - start);
    __syncthreads();
    if (tid < nj) {
      const uint32_t g = a.vals[start + tid];
      s0[tid] = a.r0[g];
      s1[tid] = a.r1[g];
      s2[tid] = a.r2[g];
      sid[tid] = (int)g;
    }
    for (int i = tid; i < nj * KC; i += kTilePix) {
      const int j = i / KC, k = i - j * KC;
      sp[i] = a.p[(size_t)a.vals[start + j] * KC + k];
    }
    for (int i = tid; i < nj * GW; i += kTilePix) gacc[i] = 0.0f;
    __syncthreads();
    for (int j = nj - 1; j >= 0; --j) {
      const uint32_t idx = start + j;
      const float4 a0 = s0[j], a1 = s1[j], a2 = s2[j];
      bool act = false;
      float pw = 0.0f;
      if (inside && idx < last) {
        pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
        act = !(pw > 0.0f || pw < a0.z);
      }
      if (__ballot_sync(0xffffffffu, act) == 0u) continue;
      float gu[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      float w = 0.0f;
      if (act) {
        const bool clamped = pw >= a0.w;
        const float alpha = clamped ? c.alpha_max : a1.w * expf(pw);
        const float inv_om = 1.0f / (1.0f - alpha);
        const float Ti = Tb * inv_om;
        w = alpha * Ti;
        const float* pj = sp + j * KC;
        float si = gc0 * a2.x + gc1 * a2.y + gc2 * a2.z + gd * a2.w;
#pragma unroll
        for (int k = 1; k < KCM; ++k)
          if (k < KC) si += go[k] * pj[k];
        const float dla = Ti * si - (S - ga * Tf) * inv_om;
        if (!clamped) {
          const float dx = a0.x - pxc, dy = a0.y - pyc;
          const float gp = dla * alpha;
          gu[0] = -gp * (a1.x * dx + a1.y * dy);
          gu[1] = -gp * (a1.y * dx + a1.z * dy);
          gu[2] = -0.5f * gp * dx * dx;
          gu[3] = -gp * dx * dy;
          gu[4] = -0.5f * gp * dy * dy;
          gu[5] = gp / a1.w;
        }
        S += w * si;
        Tb = Ti;
      }
      // warp sums of u, colour, depth and probability gradients, lane 0 to the tile
      float* gj = gacc + j * GW;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        float v = gu[q];
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0f) atomicAdd(&gj[q], v);
      }
      const float wv[4] = {w * gc0, w * gc1, w * gc2, w * gd};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float v = wv[q];
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0f) atomicAdd(&gj[6 + q], v);
      }
#pragma unroll
      for (int k = 1; k < KCM; ++k) {
        if (k < KC) {
          float v = w * go[k];
          for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0 && v != 0.0f) atomicAdd(&gj[10 + k], v);
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < nj * GW; i += kTilePix) {
      const int j = i / GW, q = i - j * GW;
      const float v = gacc[i];
      if (v != 0.0f) atomicAdd(&a.gacc[(size_t)sid[j] * GW + q], v);
    }
    end = start;
  }
}

template <int KCM>
int launch_bk(const BackwardArgs& a, const Consts& c, cudaStream_t st) {
  const int ntiles = a.cam.GX * a.cam.GY;
  if (ntiles <= 0) return 0;
  const size_t sm = sizeof(float4) * 3 * kBB + sizeof(int) * kBB + sizeof(float) * (size_t)kBB * c.KC +
                    sizeof(float) * (size_t)kBB * a.gw;
  cudaFuncSetAttribute(k_render_backward<KCM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_render_backward<KCM><<<ntiles, kTilePix, sm, st>>>(a, c);
  return 1;
}

}  // namespace

int backward_width(const Consts& c) { return 10 + c.KC; }

int launch_render_backward(const BackwardArgs& a, const Consts& c, cudaStream_t st) {
  if (c.KC <= 8) return launch_bk<8>(a, c, st);
  if (c.KC <= 24) return launch_bk<24>(a, c, st);
  if (c.KC <= 40) return launch_bk<40>(a, c, st);
  if (c.KC <= 72) return launch_bk<72>(a, c, st);
  return launch_bk<128>(a, c, st);
}

}  // namespace nbv
