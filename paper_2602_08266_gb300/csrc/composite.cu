// Front-to-back compositing (Eqs. 1-2) fused with the per-pixel
// information-gain reduction (Eqs. 6-9): one thread block per 16x16 tile,
// one thread per pixel.
//
// Pass 1 (forward): each pixel walks its tile's depth-sorted list,
//   alpha = min(alpha_max, sigma exp(p)),  p = -(A dx^2 + C dy^2)/2 - B dx dy,
// skipping a splat when p > 0 or alpha < alpha_min and stopping before a
// splat that would take the transmittance below t_min; it accumulates
// colour, depth D = sum w z, opacity and the K+1 object channels
// O' = sum w softmax(o), w = alpha T, and writes O = O' + e0 (1 - 1^T O').
// Both alpha decisions are comparisons of p against per-Gaussian exponent
// thresholds, with p computed by correctly rounded operations in a fixed
// order.
//
// Pass 2 (information): the same list is walked back to front over the
// splats each pixel blended, recovering T_i = T_{i+1} / (1 - alpha_i) and
// the suffix sums R_i = sum_{j>i} w_j x_j, which give
//   d X / d alpha_i = T_i x_i - R_i / (1 - alpha_i)
// for every output X (and d O_0 / d alpha_i gets the residual term
// -T_final / (1 - alpha_i)). Each pixel forms its share of the structured
// 2D Gauss-Newton block of every splat (layout in nbv_internal.cuh); the
// block is reduced over the warp with a shuffle transpose-reduce, over the
// tile in shared memory, and added to the per-Gaussian block in global
// memory with one vector atomic per 4 floats per (tile, Gaussian).
#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kBatch = 32;   // Gaussians staged in shared memory per round

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

// Splat exponent at a pixel centre: the decision quantity, fixed order.
__device__ __forceinline__ float splat_power(float mx, float my, float A, float B, float C, float pxc,
                                             float pyc) {
  const float dx = fs(mx, pxc), dy = fs(my, pyc);
  const float dxx = fm(dx, dx), dyy = fm(dy, dy), dxy = fm(dx, dy);
  const float q = fa(fm(A, dxx), fm(C, dyy));
  return fs(fm(-0.5f, q), fm(B, dxy));
}

// Lane L returns sum over the warp of v[L] (recursive halving).
__device__ __forceinline__ float transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

struct TriIdx {
  int m[21], n[21];
  __host__ __device__ constexpr TriIdx() : m(), n() {
    int e = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j <= i; ++j) { m[e] = i; n[e] = j; ++e; }
  }
};

template <int KCM>
struct PairTerms {
  float a[6];
  float w, qr, qd, qo, sr[3], sd;
  float ds[KCM];       // s_j - s_0, j >= 1
};

template <int KCM>
__device__ __forceinline__ float block_value(int e, const PairTerms<KCM>& t) {
  constexpr TriIdx T{};
  if (e < 21) return t.qr * t.a[T.m[e]] * t.a[T.n[e]];
  if (e < 42) return t.qd * t.a[T.m[e - 21]] * t.a[T.n[e - 21]];
  if (e < 63) return t.qo * t.a[T.m[e - 42]] * t.a[T.n[e - 42]];
  if (e < 81) return t.w * t.sr[(e - 63) / 6] * t.a[(e - 63) % 6];
  if (e < 87) return t.w * t.sd * t.a[e - 81];
  if (e == 87) return t.w * t.w;
  const int j = (e - 88) / 6 + 1;
  if (j < KCM) return t.w * t.ds[j] * t.a[(e - 88) % 6];
  return 0.0f;
}

template <int KCM>
__global__ void __launch_bounds__(kTilePix, 1)
    k_composite(CompositeArgs args, Consts c) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int KC = c.KC;
  const int nBp = (args.nB + 3) & ~3;
  float4* s0 = reinterpret_cast<float4*>(smem);
  float4* s1 = s0 + kBatch;
  float4* s2 = s1 + kBatch;
  int* sid = reinterpret_cast<int*>(s2 + kBatch);
  float* sp = reinterpret_cast<float*>(sid + kBatch);            // [kBatch][KC]
  float* acc = sp + kBatch * KC;                                  // [kBatch][nBp]
  int* touched = reinterpret_cast<int*>(acc + kBatch * nBp);      // [kBatch]
  __shared__ int s_last_max;

  const DevCam& cam = args.cam;
  const int tile = blockIdx.x;
  const int tx = tile % cam.GX, ty = tile / cam.GX;
  const int tid = threadIdx.x, lane = tid & 31;
  const int px = tx * kTile + (tid % kTile), py = ty * kTile + (tid / kTile);
  const bool inside = px < cam.W && py < cam.H;
  const float pxc = fa((float)px, 0.5f), pyc = fa((float)py, 0.5f);
  const uint2 rg = args.ranges[tile];

  // ------------------------------------------------------------- pass 1
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, D = 0.0f;
  float O[KCM];
#pragma unroll
  for (int k = 0; k < KCM; ++k) O[k] = 0.0f;
  uint32_t last = rg.x;     // one past the list index of the last blended splat
  bool done = !inside;
  uint32_t n_eval = 0, n_blend = 0;
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(done) == kTilePix) break;
    const uint32_t nj = min((uint32_t)kBatch, rg.y - start);
    if (tid < (int)nj) {
      const uint32_t g = args.vals[start + tid];
      s0[tid] = args.r0[g];
      s1[tid] = args.r1[g];
      s2[tid] = args.r2[g];
      sid[tid] = (int)g;
    }
    for (int i = tid; i < (int)nj * KC; i += kTilePix) {
      const int j = i / KC, k = i - j * KC;
      sp[i] = args.p[(size_t)args.vals[start + j] * KC + k];
    }
    __syncthreads();
    if (!done) {
      for (uint32_t j = 0; j < nj; ++j) {
        const float4 a0 = s0[j], a1 = s1[j];
        const float pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
        ++n_eval;
        if (pw > 0.0f || pw < a0.z) continue;
        const float alpha = (pw >= a0.w) ? c.alpha_max : a1.w * expf(pw);
        const float tt = T * (1.0f - alpha);
        if (tt < c.t_min) { done = true; break; }
        const float w = alpha * T;
        const float4 a2 = s2[j];
        C0 += w * a2.x; C1 += w * a2.y; C2 += w * a2.z; D += w * a2.w;
#pragma unroll
        for (int k = 0; k < KCM; ++k)
          if (k < KC) O[k] += w * sp[j * KC + k];
        T = tt;
        last = start + j + 1;
        ++n_blend;
      }
    }
  }
  if (args.stats) {
    __shared__ unsigned long long s_cnt[2];
    if (tid == 0) { s_cnt[0] = 0; s_cnt[1] = 0; }
    __syncthreads();
    atomicAdd(&s_cnt[0], (unsigned long long)n_eval);
    atomicAdd(&s_cnt[1], (unsigned long long)n_blend);
    __syncthreads();
    if (tid == 0) { atomicAdd(&args.stats[0], s_cnt[0]); atomicAdd(&args.stats[1], s_cnt[1]); }
  }
  if (inside) {
    const size_t pix = (size_t)py * cam.W + px;
    if (args.rgb) {
      args.rgb[3 * pix] = C0; args.rgb[3 * pix + 1] = C1; args.rgb[3 * pix + 2] = C2;
    }
    if (args.depth) args.depth[pix] = D;
    if (args.alpha) args.alpha[pix] = 1.0f - T;
    if (args.obj) {
      float sum = 0.0f;
#pragma unroll
      for (int k = 0; k < KCM; ++k)
        if (k < KC) sum += O[k];
#pragma unroll
      for (int k = 0; k < KCM; ++k)
        if (k < KC) args.obj[pix * KC + k] = O[k] + (k == 0 ? 1.0f - sum : 0.0f);
    }
  }
  if (args.blocks == nullptr) return;

  // ------------------------------------------------------------- pass 2
  if (tid == 0) s_last_max = (int)rg.x;
  __syncthreads();
  if (inside) atomicMax(&s_last_max, (int)last);
  __syncthreads();
  const uint32_t last_max = (uint32_t)s_last_max;
  const float Tf = T;
  float Rr0 = 0.0f, Rr1 = 0.0f, Rr2 = 0.0f, Rd = 0.0f;
  float Ro[KCM];
#pragma unroll
  for (int k = 0; k < KCM; ++k) Ro[k] = 0.0f;
  float Tb = T;   // transmittance after the splat being visited
  const int nchunk = (nBp + 31) / 32;
  for (uint32_t end = last_max; end > rg.x;) {
    const uint32_t start = (end - rg.x > (uint32_t)kBatch) ? end - kBatch : rg.x;
    const int nj = (int)(end - start);
    __syncthreads();
    if (tid < nj) {
      const uint32_t g = args.vals[start + tid];
      s0[tid] = args.r0[g];
      s1[tid] = args.r1[g];
      s2[tid] = args.r2[g];
      sid[tid] = (int)g;
      touched[tid] = 0;
    }
    for (int i = tid; i < nj * KC; i += kTilePix) {
      const int j = i / KC, k = i - j * KC;
      sp[i] = args.p[(size_t)args.vals[start + j] * KC + k];
    }
    for (int i = tid; i < nj * nBp; i += kTilePix) acc[i] = 0.0f;
    __syncthreads();
    for (int j = nj - 1; j >= 0; --j) {
      const uint32_t idx = start + j;
      bool act = false;
      PairTerms<KCM> t;
      float4 a0 = s0[j], a1 = s1[j], a2 = s2[j];
      if (inside && idx < last) {
        const float pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
        if (!(pw > 0.0f || pw < a0.z)) {
          act = true;
          const bool clamped = pw >= a0.w;
          const float alpha = clamped ? c.alpha_max : a1.w * expf(pw);
          const float om = 1.0f - alpha;
          const float inv_om = 1.0f / om;
          const float Ti = Tb * inv_om;
          const float w = alpha * Ti;
          t.w = w;
          t.sr[0] = Ti * a2.x - Rr0 * inv_om;
          t.sr[1] = Ti * a2.y - Rr1 * inv_om;
          t.sr[2] = Ti * a2.z - Rr2 * inv_om;
          t.sd = Ti * a2.w - Rd * inv_om;
          t.qr = t.sr[0] * t.sr[0] + t.sr[1] * t.sr[1] + t.sr[2] * t.sr[2];
          t.qd = t.sd * t.sd;
          const float* pj = sp + j * KC;
          const float s0v = Ti * pj[0] - Ro[0] * inv_om - Tf * inv_om;
          float qo = s0v * s0v;
          t.ds[0] = 0.0f;
#pragma unroll
          for (int k = 1; k < KCM; ++k) {
            if (k < KC) {
              const float sk = Ti * pj[k] - Ro[k] * inv_om;
              qo += sk * sk;
              t.ds[k] = sk - s0v;
            } else {
              t.ds[k] = 0.0f;
            }
          }
          t.qo = qo;
          if (clamped) {
#pragma unroll
            for (int m = 0; m < 6; ++m) t.a[m] = 0.0f;
          } else {
            const float dx = a0.x - pxc, dy = a0.y - pyc;
            t.a[0] = alpha * (-(a1.x * dx + a1.y * dy));
            t.a[1] = alpha * (-(a1.y * dx + a1.z * dy));
            t.a[2] = alpha * (-0.5f * dx * dx);
            t.a[3] = alpha * (-dx * dy);
            t.a[4] = alpha * (-0.5f * dy * dy);
            t.a[5] = alpha / a1.w;
          }
          // extend the suffix sums with this splat and step T back
          Rr0 += w * a2.x; Rr1 += w * a2.y; Rr2 += w * a2.z; Rd += w * a2.w;
#pragma unroll
          for (int k = 0; k < KCM; ++k)
            if (k < KC) Ro[k] += w * pj[k];
          Tb = Ti;
        }
      }
      const unsigned any = __ballot_sync(0xffffffffu, act);
      if (any == 0u) continue;
      if (!act) {
#pragma unroll
        for (int m = 0; m < 6; ++m) t.a[m] = 0.0f;
        t.w = 0.0f; t.qr = t.qd = t.qo = 0.0f; t.sr[0] = t.sr[1] = t.sr[2] = 0.0f; t.sd = 0.0f;
#pragma unroll
        for (int k = 0; k < KCM; ++k) t.ds[k] = 0.0f;
      }
      if (lane == 0) touched[j] = 1;
      float* accj = acc + j * nBp;
#pragma unroll
      for (int ch = 0; ch < (kOffXo + 6 * KCM + 31) / 32; ++ch) {
        if (ch < nchunk) {
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = block_value<KCM>(ch * 32 + i, t);
          const float r = transpose_reduce(v, lane);
          const int e = ch * 32 + lane;
          if (e < args.nB) atomicAdd(&accj[e], r);
        }
      }
    }
    __syncthreads();
    // flush the tile's share of each touched Gaussian's block
    const int n4 = nBp / 4;
    if (args.stats && tid < nj && touched[tid]) atomicAdd(&args.stats[2], 1ull);
    for (int i = tid; i < nj * n4; i += kTilePix) {
      const int j = i / n4, q = i - j * n4;
      if (!touched[j]) continue;
      const float4 v = reinterpret_cast<const float4*>(acc + j * nBp)[q];
      float4* dst = reinterpret_cast<float4*>(args.blocks + (size_t)sid[j] * nBp) + q;
      atomicAdd(dst, v);
    }
    end = start;
  }
}

template <int KCM>
int launch_k(const CompositeArgs& a, const Consts& c, cudaStream_t st) {
  const int nBp = (a.nB + 3) & ~3;
  const size_t sm = sizeof(float4) * 3 * kBatch + sizeof(int) * kBatch +
                    sizeof(float) * (size_t)kBatch * c.KC + sizeof(float) * (size_t)kBatch * nBp +
                    sizeof(int) * kBatch;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_composite<KCM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const int ntiles = a.cam.GX * a.cam.GY;
  if (ntiles <= 0) return 0;
  k_composite<KCM><<<ntiles, kTilePix, sm, st>>>(a, c);
  return 1;
}

}  // namespace

int launch_composite(const CompositeArgs& a, const Consts& c, cudaStream_t st) {
  if (c.KC <= 8) return launch_k<8>(a, c, st);
  if (c.KC <= 24) return launch_k<24>(a, c, st);
  if (c.KC <= 40) return launch_k<40>(a, c, st);
  if (c.KC <= 72) return launch_k<72>(a, c, st);
  return launch_k<128>(a, c, st);
}

}  // namespace nbv
