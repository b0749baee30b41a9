// Front-to-back compositing (Eqs. 1-2) fused with the per-pixel
// information-gain reduction (Eqs. 6-9): one thread block per 16x16 tile,
// one thread per pixel.
//
// Pass 1 (forward): each pixel walks its tile's depth-sorted list,
//   alpha = min(alpha_max, sigma exp(p)),  p = -(A dx^2 + C dy^2)/2 - B dx dy,
// skipping a splat when p > 0 or alpha < alpha_min and stopping before a
// splat that would take the transmittance below t_min; when an image is
// asked for it accumulates colour, depth D = sum w z, opacity and the K+1
// object channels O' = sum w softmax(o), w = alpha T, and writes
// O = O' + e0 (1 - 1^T O'). Both alpha decisions are comparisons of p
// against per-Gaussian exponent thresholds, with p computed by correctly
// rounded operations in a fixed order.
//
// Pass 2 (information): the same list is walked back to front over the
// splats each pixel blended, recovering T_i = T_{i+1} / (1 - alpha_i) and
// the suffix sums R_i = sum_{j>i} w_j x_j, which give
//   d X / d alpha_i = T_i x_i - R_i / (1 - alpha_i)
// for every output X (and d O_0 / d alpha_i gets the residual term
// -T_final / (1 - alpha_i)). Each pixel forms its share of the structured
// 2D Gauss-Newton block of every splat (layout in nbv_internal.cuh); the
// shares are summed over the warp's pixels by TF32 tensor-core products
// (error-compensated by default: three products of high and low parts per
// term), over the tile's warps in shared memory, and added to the
// per-Gaussian block in global memory with one vector atomic per 4 floats
// per (tile, Gaussian).
//
// A scoring launch (blocks, no images) runs the two passes as two kernels:
// k_forward (pass 1 only: transmittance, list ends and the first splat with
// an information block per pixel; records staged by bulk copies into a
// double-buffered mbarrier ring) and k_composite reading those results
// (pass 2 only, each warp walking back to front down to its pixels' first
// information splat, the next round's records gathered by cp.async while
// the current one runs). Images (and the rare launch that wants both) run
// both passes in k_composite.
#include <type_traits>

#include "nbv_internal.cuh"

namespace nbv {
namespace {


__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }

// TF32 tensor-core helper (warp-level mma.sync, FP32 accumulation).
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Four 8 x 8 tiles of 16-bit pairs from shared memory (one row address per lane).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const float* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a)
               : "memory");
}

// An FP32 value as a TF32 operand of the contraction. The tensor core reads
// only the upper 19 bits of a TF32 operand word (sign, exponent, 10 mantissa
// bits), so adding half a TF32 unit in the last place (bit 12) to the bit
// pattern makes it read the value rounded to nearest, ties away from zero,
// which is what cvt.rna.tf32.f32 produces, for a single integer add. Finite
// x only (all U and V entries are).
__device__ __forceinline__ float tf32f(float x) { return __uint_as_float(__float_as_uint(x) + 0x1000u); }

// A U or V entry as stored for the contraction: the TF32 operand (single
// products, 10 mantissa bits) or the FP32 value itself, split into two TF32
// terms when the fragments are loaded (kSplit).
template <bool kSplit>
__device__ __forceinline__ float uvst(float x) { return kSplit ? x : tf32f(x); }

// x = hi + lo with hi the TF32 value nearest x (ties away from zero) and lo
// the exact remainder, itself given to the tensor core rounded to nearest:
// the error-compensated product a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (three TF32 products, FP32 accumulation) keeps about 21 bits of each
// product instead of 10 (Markidis et al., 2018; Ootomo and Yokota, 2022).
__device__ __forceinline__ void split_tf32(uint32_t x, uint32_t& hi, uint32_t& lo) {
  hi = (x + 0x1000u) & 0xFFFFE000u;
  lo = __float_as_uint(__uint_as_float(x) - __uint_as_float(hi)) + 0x1000u;
}

// d += A B over one k-step, single TF32 products or error-compensated.
template <bool kSplit>
__device__ __forceinline__ void mma_k(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if (!kSplit) {
    mma_tf32(d, a[0], a[1], a[2], a[3], b0, b1);
  } else {
    uint32_t ah[4], al[4], bh0, bl0, bh1, bl1;
#pragma unroll
    for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], al[i]);
    split_tf32(b0, bh0, bl0);
    split_tf32(b1, bh1, bl1);
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
  }
}

// Per-warp contraction buffers are value-major: element (value s, pixel
// slot) at s * kCS + slot. With kCS = 36 (= 4 mod 32) the per-pixel stores
// (one value, 32 slots) and the mma fragment loads (value 4 g + slot t) both
// hit 32 distinct banks. U needs 3 + 16 * ceil((K + 5) / 16) value rows, V 32.
__host__ __device__ __forceinline__ int u_tiles(int K) { return (K + 5 + 15) / 16; }
__host__ __device__ __forceinline__ int u_rows(int K) { return 3 + 16 * u_tiles(K); }
constexpr int kCS = 36;
constexpr int kVRows = 32;

// Asynchronous staging of the forward pass's records (scoring launches):
// every round's {r0, r1} pairs (2 x 16 bytes per splat, gathered by
// Gaussian index) are fetched by bulk copies of the tensor memory accelerator
// (cp.async.bulk, global -> shared) into one of two buffers, each completed
// by its own mbarrier (expected bytes set by one arrival), while the block
// composites the other buffer. Waits are bounded: on a time-out the kernel
// sets *err, marks its pixels done and drains (again bounded) before leaving.
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Per-thread asynchronous gathers (cp.async) into shared memory: 16-byte
// records and 4-byte words; each thread waits for its own copies, and a
// barrier afterwards publishes them to the block.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct StageRing {
  float4* buf;           // [2][2][kBatch]: buffer b, record r0 / r1, splat
  uint32_t bar;          // shared address of two consecutive mbarriers
  uint32_t use0, use1;   // phases waited for per buffer (the parity of the next wait)
  int* err;

  __device__ float4* rec(int b, int r, int kBatch) { return buf + (2 * b + r) * kBatch; }
  // warp 0: round k of the list [lo, hi) into buffer k & 1
  __device__ void issue(const CompositeArgs& a, uint32_t lo, uint32_t hi, uint32_t k, size_t rec_off, int lane,
                        int kBatch) {
    const uint32_t start = lo + k * (uint32_t)kBatch;
    const int nj = (int)min((uint32_t)kBatch, hi - start);
    const int b = (int)(k & 1u);
    const uint32_t bb = bar + 8u * (uint32_t)b;
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"((uint32_t)(32 * nj))
                   : "memory");
    __syncwarp();
    if (lane < nj) {
      const uint32_t g = a.vals[start + lane];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_g2s(rec(b, 0, kBatch) + lane, a.r0 + rec_off + g, 16u, bb);
      bulk_g2s(rec(b, 1, kBatch) + lane, a.r1 + rec_off + g, 16u, bb);
    }
  }
  // every thread: wait for buffer b's current phase (bounded)
  __device__ bool wait(int b) {
    const uint32_t bb = bar + 8u * (uint32_t)b, parity = (b ? use1 : use0) & 1u;
    if (b) ++use1; else ++use0;
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
      uint32_t ok;
      asm volatile(
          "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
          : "=r"(ok)
          : "r"(bb), "r"(parity)
          : "memory");
      if (ok) return true;
    }
    if (err) atomicExch(err, 1);
    return false;
  }
};

// Byte offset of the staging ring in the dynamic shared memory: after the
// round's records, ids, probabilities, block accumulators, flags and the
// per-warp contraction buffers, rounded up to 16 bytes.
__host__ __device__ inline size_t ring_offset(int K, int KC, int nB, int kBatch) {
  const int nBp = (nB + 3) & ~3;
  const size_t end = sizeof(float4) * 3 * kBatch + sizeof(int) * kBatch + sizeof(float) * (size_t)kBatch * ((KC + 1) & ~1) +
                     sizeof(float) * (size_t)kBatch * nBp + sizeof(int) * kBatch +
                     sizeof(float) * (kTilePix / 32) * kCS * (size_t)(u_rows(K) + kVRows);
  return (end + 15) & ~(size_t)15;
}

// Byte offset of the information pass's second staging set (the records,
// block slots, flags and probabilities of the round after the current one),
// past the staging ring and its barriers; and its size.
__host__ __device__ inline size_t stage2_offset(int K, int KC, int nB, int kBatch) {
  return (ring_offset(K, KC, nB, kBatch) + sizeof(float4) * 4 * kBatch + 16 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t stage2_bytes(int KC, int kBatch) {
  return sizeof(float4) * 3 * kBatch + sizeof(int) * 2 * kBatch + sizeof(float) * (size_t)kBatch * ((KC + 1) & ~1);
}

// One 16x16 tile of one view: both passes. blocks_v is the view's block
// array (NULL: render only).
template <int KCM, int kBatch, bool kSplit>
__device__ __forceinline__ void composite_tile(const CompositeArgs& args, const Consts& c, const DevCam& cam,
                                               int tile, uint32_t gt, uint2 rg, float* blocks_v, size_t rec_off,
                                               unsigned char* smem, StageRing& ring) {
  const int KC = c.KC;
  const int nB = args.nB, nBp = (nB + 3) & ~3;
  float4* s0 = reinterpret_cast<float4*>(smem);
  float4* s1 = s0 + kBatch;
  float4* s2 = s1 + kBatch;
  int* sid = reinterpret_cast<int*>(s2 + kBatch);
  const int KCP = (KC + 1) & ~1;                                  // even row stride: float2 loads
  float* sp = reinterpret_cast<float*>(sid + kBatch);            // [kBatch][KCP]
  float* acc = sp + kBatch * KCP;                                 // [kBatch][nBp]
  int* touched = reinterpret_cast<int*>(acc + kBatch * nBp);      // [kBatch]
  __shared__ int s_last_max;

  const int tx = tile % cam.GX, ty = tile / cam.GX;
  const int tid = threadIdx.x, lane = tid & 31;
  // each warp covers an 8 x 4 pixel block (compact footprints keep more of a
  // warp's lanes inside a splat); 8 warps tile a 16 x 16 or a 32 x 8 tile
  const int wq = tid >> 5;
  const int wx = cam.TW >> 3;                 // 8-wide warp blocks per tile row (2 or 4)
  const int px = tx * cam.TW + 8 * (wq % wx) + (lane & 7), py = ty * cam.TH + 4 * (wq / wx) + (lane >> 3);
  const bool inside = px < cam.W && py < cam.H;
  const float pxc = fa((float)px, 0.5f), pyc = fa((float)py, 0.5f);

  // An information launch over an active subset (a target object, Eq. 12):
  // the list entries before the first active splat need no information
  // pass, and a tile without one needs neither pass (a scoring launch
  // writes no image).
  __shared__ int s_first;
  uint32_t first_info = rg.x;
  const bool info_only = args.fwd != nullptr;        // the forward pass ran in launch_forward
  if (info_only) {
    first_info = args.tile_first[gt];
    if (first_info >= rg.y) return;
  } else if (blocks_v != nullptr && args.n_act < args.n) {
    if (tid == 0) s_first = (int)rg.y;
    __syncthreads();
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kTilePix) {
      const uint32_t i = b0 + tid;
      if (i < rg.y && args.slot[args.vals[i]] >= 0) atomicMin(&s_first, (int)i);
      if (__syncthreads_or(s_first < (int)rg.y)) break;
    }
    first_info = (uint32_t)s_first;
    if (first_info >= rg.y && args.rgb == nullptr && args.depth == nullptr && args.alpha == nullptr &&
        args.obj == nullptr)
      return;
  }

  // ------------------------------------------------------------- pass 1
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, D = 0.0f;
  float2 O2[KCM / 2];                       // object channels in pairs (packed f32x2 FMA)
#pragma unroll
  for (int q = 0; q < KCM / 2; ++q) O2[q] = make_float2(0.0f, 0.0f);
  uint32_t last = rg.x;     // one past the list index of the last blended splat
  uint32_t first_pix = kNoEntry;   // the first blended splat with an information block
  bool done = !inside;
  uint32_t n_eval = 0, n_blend = 0;
  // colour, depth and object sums only when an image is asked for (the
  // information pass needs only the final transmittance and list ends)
  const bool want_cd = args.rgb != nullptr || args.depth != nullptr;
  const bool want_o = args.obj != nullptr;
  if (info_only) {
    const uint4 f = args.fwd[(size_t)gt * kTilePix + tid];
    T = __uint_as_float(f.x);
    last = f.y;
    first_pix = f.z;
  } else if (!want_cd && !want_o) {
    // records staged by bulk copies, the next round in flight meanwhile
    const uint32_t nst = (rg.y - rg.x + kBatch - 1) / kBatch;
    if (nst > 0 && wq == 0) ring.issue(args, rg.x, rg.y, 0, rec_off, lane, kBatch);
    uint32_t k = 0;
    for (; k < nst; ++k) {
      if (__syncthreads_count(done) == kTilePix) break;
      if (k + 1 < nst && wq == 0) ring.issue(args, rg.x, rg.y, k + 1, rec_off, lane, kBatch);
      const int b = (int)(k & 1u);
      if (!ring.wait(b)) done = true;
      const float4* q0 = ring.rec(b, 0, kBatch);
      const float4* q1 = ring.rec(b, 1, kBatch);
      const uint32_t start = rg.x + k * kBatch;
      const uint32_t nj = min((uint32_t)kBatch, rg.y - start);
      if (!done) {
        for (uint32_t j = 0; j < nj; ++j) {
          const float4 a0 = q0[j], a1 = q1[j];
          const float pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
          ++n_eval;
          if (pw > 0.0f || pw < a0.z) continue;
          const float alpha = (pw >= a0.w) ? c.alpha_max : a1.w * __expf(pw);
          const float tt = T * (1.0f - alpha);
          if (tt < c.t_min) { done = true; break; }
          T = tt;
          last = start + j + 1;
          ++n_blend;
        }
      }
    }
    // a round fetched ahead but not composited (every pixel had stopped)
    if (k < nst) ring.wait((int)(k & 1u));
  } else {
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(done) == kTilePix) break;
    const uint32_t nj = min((uint32_t)kBatch, rg.y - start);
    if (tid < (int)nj) {
      const uint32_t g = args.vals[start + tid];
      s0[tid] = args.r0[rec_off + g];
      s1[tid] = args.r1[rec_off + g];
      if (want_cd) s2[tid] = args.r2[rec_off + g];
      sid[tid] = (int)g;
    }
    if (want_o) {
      for (int i = tid; i < (int)nj * KCP; i += kTilePix) {
        const int j = i / KCP, k = i - j * KCP;
        sp[i] = k < KC ? args.p[(size_t)args.vals[start + j] * KC + k] : 0.0f;
      }
    }
    __syncthreads();
    if (!done) {
      for (uint32_t j = 0; j < nj; ++j) {
        const float4 a0 = s0[j], a1 = s1[j];
        const float pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
        ++n_eval;
        if (pw > 0.0f || pw < a0.z) continue;
        const float alpha = (pw >= a0.w) ? c.alpha_max : a1.w * __expf(pw);
        const float tt = T * (1.0f - alpha);
        if (tt < c.t_min) { done = true; break; }
        const float w = alpha * T;
        if (want_cd) {
          const float4 a2 = s2[j];
          C0 += w * a2.x; C1 += w * a2.y; C2 += w * a2.z; D += w * a2.w;
        }
        if (want_o) {
          const float2 w2 = make_float2(w, w);
          const float2* pj2 = reinterpret_cast<const float2*>(sp + j * KCP);
#pragma unroll
          for (int q = 0; q < KCM / 2; ++q)
            if (2 * q < KC) O2[q] = __ffma2_rn(w2, pj2[q], O2[q]);
        }
        T = tt;
        last = start + j + 1;
        ++n_blend;
      }
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
        if (k < KC) sum += (k & 1) ? O2[k >> 1].y : O2[k >> 1].x;
#pragma unroll
      for (int k = 0; k < KCM; ++k)
        if (k < KC) args.obj[pix * KC + k] = ((k & 1) ? O2[k >> 1].y : O2[k >> 1].x) + (k == 0 ? 1.0f - sum : 0.0f);
    }
  }
  if (blocks_v == nullptr) return;

  // ------------------------------------------------------------- pass 2
  // The walk runs back to front from the tile's last blended splat. With the
  // forward pass's per-pixel first information splat it ends, per warp, at
  // the earliest one among the warp's pixels (nothing in front of it reaches
  // a block: it would only extend suffix sums that are no longer read), and
  // per tile at the earliest among all pixels.
  __shared__ uint32_t s_first_min;
  if (tid == 0) { s_last_max = (int)rg.x; s_first_min = kNoEntry; }
  __syncthreads();
  if (inside) {
    atomicMax(&s_last_max, (int)last);
    if (info_only) atomicMin(&s_first_min, first_pix);
  }
  __syncthreads();
  const uint32_t last_max = (uint32_t)s_last_max;
  if (info_only) first_info = max(first_info, s_first_min);
  // splats at or past every pixel of this warp's last blended one are skipped warp-wide
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, inside ? last : rg.x);
  const uint32_t wfirst = info_only ? __reduce_min_sync(0xffffffffu, inside ? first_pix : kNoEntry) : 0u;
  const float Tf = T;
  float Rr0 = 0.0f, Rr1 = 0.0f, Rr2 = 0.0f, Rd = 0.0f;
  float2 Ro2[KCM / 2];                      // object suffix sums in pairs
#pragma unroll
  for (int q = 0; q < KCM / 2; ++q) Ro2[q] = make_float2(0.0f, 0.0f);
  float Tb = T;   // transmittance after the splat being visited
  uint32_t n_ig = 0;  // (pixel, active splat) pairs of the information pass
  // Per-warp contraction buffers: row = pixel (lane). U holds the pixel's
  // scalars [q_rgb a^2, q_d a^2, q_o a^2 | w s_c a (3), w s_D a, w (s_j - s_0) a
  // (K) | w^2] (a = alpha, or 0 when clamped); V holds the splat geometry
  // v = d alpha / d(mx, my, A, B, C, sigma) / alpha at the pixel as
  // [v_m v_n (21, packed lower) 0 0 0 | v_m (6) 1 0]. The sums over the warp's
  // pixels of U_s V_c are the structured block entries: two TF32 tensor-core
  // contractions, D_Q = U[0..16)^T V[0..24) and D_X = U[3..)^T V[24..32).
  const int K = c.K;
  const int NU = u_rows(K), MTB = u_tiles(K);
  float* Uw = reinterpret_cast<float*>(touched + kBatch) + (size_t)(tid >> 5) * kCS * (NU + kVRows);
  float* Vw = Uw + kCS * NU;
  for (int i = lane; i < kCS * (NU + kVRows); i += 32) Uw[i] = 0.0f;
  __syncwarp();
  constexpr int MTBM = (KCM + 4 + 15) / 16;
  const int gq = lane >> 2, t4 = lane & 3;
  // where each D fragment element of this lane goes in the structured block
  int eq[6];                                  // Q rows (U row gq < 3), V columns < 21
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int cc = 8 * (q >> 1) + 2 * t4 + (q & 1);
    eq[q] = (gq < 3 && cc < 21) ? 21 * gq + cc : -1;
  }
  int ex[MTBM][4];                            // X / W2 rows (U[3..]), V columns 24..31
#pragma unroll
  for (int mt = 0; mt < MTBM; ++mt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = 16 * mt + gq + (i >= 2 ? 8 : 0);
      const int cc = 2 * t4 + (i & 1);
      int e = -1;
      if (mt < MTB) {
        if (cc < 6) {
          if (r < 4) e = kOffXrgb + 6 * r + cc;          // X_rgb (3 rows) then X_d
          else if (r < 4 + K) e = kOffXo + 6 * (r - 4) + cc;
        } else if (cc == 6 && r == 4 + K) {
          e = kOffW2;
        }
      }
      ex[mt][i] = e;
    }
  // The records of this pass are staged one round ahead: while the block
  // works on round r from one set of buffers, every warp gathers its share
  // of round r + 1 (the 16-byte records, the block slot and the K + 1
  // probabilities of kSPW splats) into the other set with cp.async, using
  // Gaussian ids it loaded during round r - 1; each thread waits for its own
  // copies after the round's flush, and the next round's opening barrier
  // publishes them.
  constexpr int kSPW = kBatch / (kTilePix / 32);          // splats a warp stages per round
  unsigned char* st2 = smem + stage2_offset(K, KC, nB, kBatch);
  float4* x0 = reinterpret_cast<float4*>(st2);
  float4* x1 = x0 + kBatch;
  float4* x2 = x1 + kBatch;
  int* xid = reinterpret_cast<int*>(x2 + kBatch);
  int* xtouched = xid + kBatch;
  float* xsp = reinterpret_cast<float*>(xtouched + kBatch);
  auto rstart = [&](uint32_t e) -> uint32_t {
    return (e - first_info > (uint32_t)kBatch) ? e - kBatch : first_info;
  };
  // lanes < kSPW: the Gaussian ids of this warp's splats of round [st_, en_)
  auto load_ids = [&](uint32_t st_, uint32_t en_) -> uint32_t {
    const int j = wq * kSPW + lane;
    return (lane < kSPW && j < (int)(en_ - st_)) ? args.vals[st_ + j] : 0u;
  };
  auto issue = [&](uint32_t st_, uint32_t en_, int set, uint32_t gq) {
    float4* d0 = set ? x0 : s0;
    float4* d1 = set ? x1 : s1;
    float4* d2 = set ? x2 : s2;
    int* did = set ? xid : sid;
    float* dp = set ? xsp : sp;
    const int njr = (int)(en_ - st_);
#pragma unroll
    for (int q = 0; q < kSPW; ++q) {
      const int j = wq * kSPW + q;
      const uint32_t g = __shfl_sync(0xffffffffu, gq, q);
      if (j < njr) {                                        // warp-uniform
        if (lane == 0) cp_async16(d0 + j, args.r0 + rec_off + g);
        else if (lane == 1) cp_async16(d1 + j, args.r1 + rec_off + g);
        else if (lane == 2) cp_async16(d2 + j, args.r2 + rec_off + g);
        else if (lane == 3) cp_async4(did + j, args.slot + g);   // block slot, or -1: only extends the suffix sums
        for (int k = lane; k < KCP; k += 32) {
          float* d = dp + j * KCP + k;
          if (k < KC) cp_async4(d, args.p + (size_t)g * KC + k);
          else *d = 0.0f;
        }
      }
    }
    cp_async_commit();
  };
  uint32_t gnext = 0u;
  if (tid < kBatch) touched[tid] = 0;
  if (last_max > first_info) {
    const uint32_t st0 = rstart(last_max);
    issue(st0, last_max, 0, load_ids(st0, last_max));
    if (st0 > first_info) gnext = load_ids(rstart(st0), st0);
    cp_async_wait_all();
  }
  int set = 0;
  for (uint32_t end = last_max; end > first_info; set ^= 1) {
    const uint32_t start = rstart(end);
    const int nj = (int)(end - start);
    __syncthreads();     // this round's set is complete and published; the last round's flush is done
    const float4* c0 = set ? x0 : s0;
    const float4* c1 = set ? x1 : s1;
    const float4* c2 = set ? x2 : s2;
    const int* cid = set ? xid : sid;
    const float* csp = set ? xsp : sp;
    int* ctouched = set ? xtouched : touched;
    // the other set's flags were last read by the flush before this barrier
    // and are next written in the following round
    if (tid < kBatch) (set ? touched : xtouched)[tid] = 0;
    if (start > first_info) {
      const uint32_t s1n = rstart(start);
      issue(s1n, start, set ^ 1, gnext);
      gnext = (s1n > first_info) ? load_ids(rstart(s1n), s1n) : 0u;
    }
    for (int j = nj - 1; j >= 0; --j) {
      const uint32_t idx = start + j;
      if (idx >= wlast) continue;
      if (idx < wfirst) break;            // warp-uniform: nothing of this warp's is left in front
      bool act = false;
      const float4 a0 = c0[j], a1 = c1[j], a2 = c2[j];
      float pw = 0.0f;
      if (inside && idx < last) {
        pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
        act = !(pw > 0.0f || pw < a0.z);
      }
      const unsigned any = __ballot_sync(0xffffffffu, act);
      if (any == 0u) continue;
      const bool info = cid[j] >= 0;     // the same for the whole tile
      // active pixels are compacted into the first rows of the warp's buffers
      const int nact = __popc(any);
      const int nks = (nact + 7) >> 3;
      const int slot = __popc(any & ((1u << lane) - 1u));
      if (act) {
        float* Ur = Uw + slot;           // value s at Ur[s * kCS]
        float* Vr = Vw + slot;
        const bool clamped = pw >= a0.w;
        const float alpha = clamped ? c.alpha_max : a1.w * __expf(pw);
        const float inv_om = __fdividef(1.0f, 1.0f - alpha);
        const float Ti = Tb * inv_om;
        const float w = alpha * Ti;
        const float2* pj2 = reinterpret_cast<const float2*>(csp + j * KCP);
        if (info) {
        const float ae = clamped ? 0.0f : alpha;
        const float wa = w * ae;
        // d out / d alpha_i = T_i x_i - R_i / (1 - alpha_i)
        const float sr0 = Ti * a2.x - Rr0 * inv_om;
        const float sr1 = Ti * a2.y - Rr1 * inv_om;
        const float sr2 = Ti * a2.z - Rr2 * inv_om;
        const float sd = Ti * a2.w - Rd * inv_om;
        // s_k = T_i p_k - R_k / (1 - alpha), two channels per packed FMA; the
        // residual channel 0 also carries -T_final / (1 - alpha)
        const float2 Ti2 = make_float2(Ti, Ti), ni2 = make_float2(-inv_om, -inv_om);
        float2 s01 = __ffma2_rn(Ti2, pj2[0], __fmul2_rn(Ro2[0], ni2));
        s01.x -= Tf * inv_om;
        const float s0v = s01.x;
        const float2 wa2 = make_float2(wa, wa), off2 = make_float2(-wa * s0v, -wa * s0v);
        float2 qo2 = make_float2(s0v * s0v, s01.y * s01.y);
        if (KC > 1) Ur[7 * kCS] = uvst<kSplit>(fmaf(wa, s01.y, -wa * s0v));
#pragma unroll
        for (int q = 1; q < KCM / 2; ++q) {
          if (2 * q < KC) {
            const float2 sk2 = __ffma2_rn(Ti2, pj2[q], __fmul2_rn(Ro2[q], ni2));
            qo2 = __ffma2_rn(sk2, sk2, qo2);
            const float2 u2 = __ffma2_rn(wa2, sk2, off2);
            Ur[(6 + 2 * q) * kCS] = uvst<kSplit>(u2.x);
            if (2 * q + 1 < KC) Ur[(7 + 2 * q) * kCS] = uvst<kSplit>(u2.y);
          }
        }
        const float qo = qo2.x + qo2.y;
        const float ae2 = ae * ae;
        Ur[0] = uvst<kSplit>((sr0 * sr0 + sr1 * sr1 + sr2 * sr2) * ae2);
        Ur[kCS] = uvst<kSplit>(sd * sd * ae2);
        Ur[2 * kCS] = uvst<kSplit>(qo * ae2);
        Ur[3 * kCS] = uvst<kSplit>(wa * sr0);
        Ur[4 * kCS] = uvst<kSplit>(wa * sr1);
        Ur[5 * kCS] = uvst<kSplit>(wa * sr2);
        Ur[6 * kCS] = uvst<kSplit>(wa * sd);
        Ur[(7 + K) * kCS] = uvst<kSplit>(w * w);
        // splat geometry at this pixel
        const float dx = a0.x - pxc, dy = a0.y - pyc;
        const float v[6] = {-(a1.x * dx + a1.y * dy), -(a1.y * dx + a1.z * dy), -0.5f * dx * dx,
                            -dx * dy, -0.5f * dy * dy, __fdividef(1.0f, a1.w)};
#pragma unroll
        for (int m = 0; m < 6; ++m) {
#pragma unroll
          for (int n = 0; n <= m; ++n) Vr[(m * (m + 1) / 2 + n) * kCS] = uvst<kSplit>(v[m] * v[n]);
          Vr[(24 + m) * kCS] = uvst<kSplit>(v[m]);
        }
        Vr[30 * kCS] = 1.0f;
        }
        // extend the suffix sums with this splat and step T back
        Rr0 += w * a2.x; Rr1 += w * a2.y; Rr2 += w * a2.z; Rd += w * a2.w;
        const float2 w2 = make_float2(w, w);
#pragma unroll
        for (int q = 0; q < KCM / 2; ++q)
          if (2 * q < KC) Ro2[q] = __ffma2_rn(w2, pj2[q], Ro2[q]);
        Tb = Ti;
      }
      if (!info) continue;
      n_ig += act ? 1u : 0u;
      if (lane == 0) ctouched[j] = 1;
      __syncwarp();
      float dq[3][4], dxo[MTBM][4];
#pragma unroll
      for (int q = 0; q < 3; ++q) dq[q][0] = dq[q][1] = dq[q][2] = dq[q][3] = 0.0f;
#pragma unroll
      for (int q = 0; q < MTBM; ++q) dxo[q][0] = dxo[q][1] = dxo[q][2] = dxo[q][3] = 0.0f;
      // fragments by ldmatrix (8 x 8 tiles of 16-bit pairs = 8 rows x 4 TF32
      // words): lane l addresses row l % 8 of tile l / 8. A: tiles (rows
      // 0-7 | 8-15) x (slots 0-3 | 4-7); V (B, one row per output column):
      // (rows 0-7 | 8-15, then 16-23 | 24-31) x (slots 0-3 | 4-7)
      const int i8 = lane & 7, m4 = lane >> 3;
      const float* aq = Uw + (8 * (m4 & 1) + i8) * kCS + 4 * (m4 >> 1);
      const float* ax = aq + 3 * kCS;
      const float* vq = Vw + (8 * (m4 >> 1) + i8) * kCS + 4 * (m4 & 1);
      for (int ks = 0; ks < nks; ++ks) {
        const int c0 = 8 * ks + t4, c1 = c0 + 4;          // pixel slots of this lane's fragments
        // slots at or past nact hold an earlier splat's values: their V (the B
        // operand of both contractions) enters as zero
        const bool ok0 = c0 < nact, ok1 = c1 < nact;
        uint32_t qa[4], vb[4], vc[4];
        ldsm_x4(qa, aq + 8 * ks);
        ldsm_x4(vb, vq + 8 * ks);
        ldsm_x4(vc, vq + 16 * kCS + 8 * ks);
        const uint32_t b00 = ok0 ? vb[0] : 0u, b01 = ok1 ? vb[1] : 0u;   // columns 0-7
        const uint32_t b10 = ok0 ? vb[2] : 0u, b11 = ok1 ? vb[3] : 0u;   // 8-15
        const uint32_t b20 = ok0 ? vc[0] : 0u, b21 = ok1 ? vc[1] : 0u;   // 16-23
        const uint32_t xb0 = ok0 ? vc[2] : 0u, xb1 = ok1 ? vc[3] : 0u;   // 24-31
        mma_k<kSplit>(dq[0], qa, b00, b01);
        mma_k<kSplit>(dq[1], qa, b10, b11);
        mma_k<kSplit>(dq[2], qa, b20, b21);
#pragma unroll
        for (int mt = 0; mt < MTBM; ++mt)
          if (mt < MTB) {
            uint32_t xa[4];
            ldsm_x4(xa, ax + 16 * mt * kCS + 8 * ks);
            mma_k<kSplit>(dxo[mt], xa, xb0, xb1);
          }
      }
      __syncwarp();
      // scatter D into the tile's block of splat j: the needed fragment
      // entries are staged at their block offsets in the (now free) V buffer,
      // then added with one atomic per block entry, 32 consecutive entries
      // per warp instruction (half the atomics of adding from the fragments)
      float* stage = Vw;
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (eq[q] >= 0) stage[eq[q]] = dq[q >> 1][q & 1];
#pragma unroll
      for (int mt = 0; mt < MTBM; ++mt)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (ex[mt][i] >= 0) stage[ex[mt][i]] = dxo[mt][i];
      __syncwarp();
      float* accj = acc + j * nBp;
      for (int e = lane; e < nB; e += 32) atomicAdd(&accj[e], stage[e]);
      __syncwarp();
    }
    __syncthreads();
    // flush the tile's share of each touched Gaussian's block
    const int n4 = nBp / 4;
    if (args.stats && tid < nj && ctouched[tid]) atomicAdd(&args.stats[2], 1ull);
    for (int i = tid; i < nj * n4; i += kTilePix) {
      const int j = i / n4, q = i - j * n4;
      if (!ctouched[j]) continue;
      float4* src = reinterpret_cast<float4*>(acc + j * nBp) + q;
      const float4 v = *src;
      *src = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // the accumulators stay zero between rounds
      float4* dst = reinterpret_cast<float4*>(blocks_v + (size_t)cid[j] * nBp) + q;
      atomicAdd(dst, v);
    }
    cp_async_wait_all();   // this thread's copies of the next round have landed
    end = start;
  }
  if (args.stats) {
    __shared__ unsigned long long s_ig;
    if (tid == 0) s_ig = 0;
    __syncthreads();
    const unsigned wsum = __reduce_add_sync(0xffffffffu, n_ig);
    if (lane == 0 && wsum) atomicAdd(&s_ig, (unsigned long long)wsum);
    __syncthreads();
    if (tid == 0 && s_ig) atomicAdd(&args.stats[3], s_ig);
  }
}

template <int KCM, int kBatch, bool kSplit>
__global__ void __launch_bounds__(kTilePix, (KCM <= 24 ? 2 : 1))
    k_composite(CompositeArgs args, Consts c) {
  extern __shared__ __align__(16) unsigned char smem[];
  // per-splat block accumulators start at zero and are zeroed as they are
  // flushed; the staging ring and its two mbarriers live past the per-warp
  // buffers (offsets as launch_k sizes them)
  const int KCP = (c.KC + 1) & ~1;
  const int nBp = (args.nB + 3) & ~3;
  float* acc = reinterpret_cast<float*>(smem + sizeof(float4) * 3 * kBatch + sizeof(int) * kBatch) + kBatch * KCP;
  for (int i = threadIdx.x; i < kBatch * nBp; i += kTilePix) acc[i] = 0.0f;
  const size_t ring_off = ring_offset(c.K, c.KC, args.nB, kBatch);
  StageRing ring;
  ring.buf = reinterpret_cast<float4*>(smem + ring_off);
  ring.bar = smem_u32(smem + ring_off + sizeof(float4) * 4 * kBatch);
  ring.use0 = ring.use1 = 0u;
  ring.err = args.err;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ring.bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ring.bar + 8u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (args.queue == nullptr) {                 // one tile of one view per block
    composite_tile<KCM, kBatch, kSplit>(args, c, args.cam, blockIdx.x, blockIdx.x, args.ranges[blockIdx.x],
                                        args.blocks, 0, smem, ring);
    return;
  }
  // persistent: (view, tile) items in queue order (longest lists first)
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(args.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= args.n_items) break;
    const uint32_t gt = args.queue[it];
    const int v = args.tile_view[gt];
    const DevCam cam = args.cams[v];
    composite_tile<KCM, kBatch, kSplit>(args, c, cam, (int)(gt - args.tile_base[v]), gt, args.ranges[gt],
                                        args.blocks + (size_t)v * args.n_act * ((args.nB + 3) & ~3),
                                        (size_t)v * args.n, smem, ring);
  }
}

// The forward pass of a scoring launch, on its own: a tile's list walked
// front to back in rounds of kFwd splats staged by bulk copies (the next
// round in flight meanwhile), per pixel only what the information pass needs
// (transmittance, list ends, the first blended splat with an information
// block). With an active subset, a tile without an active splat is skipped
// (its first active entry recorded as its list end).
constexpr int kFwd = 32;   // one bit per staged splat in a 32-bit mask

// Two pixels per thread: thread t takes the information pass's pixels t and
// t + kFwdThreads (the same column, 8 rows apart in a 16x16 tile, 4 in a
// 32x8 one), so every staged record is read once for both and each thread
// has two independent blend chains.
constexpr int kFwdThreads = kTilePix / 2;

__device__ __forceinline__ void forward_tile(const CompositeArgs& args, const Consts& c, const DevCam& cam, int tile,
                                             uint32_t gt, uint2 rg, size_t rec_off, StageRing& ring) {
  const int tx = tile % cam.GX, ty = tile / cam.GX;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  const int wx = cam.TW >> 3;
  // pixel of the information pass's thread t (its 8 x 4 warp blocks)
  auto pixel = [&](int t, int& px, int& py) {
    const int q = t >> 5, l = t & 31;
    px = tx * cam.TW + 8 * (q % wx) + (l & 7);
    py = ty * cam.TH + 4 * (q / wx) + (l >> 3);
  };
  int px0, py0, px1, py1;
  pixel(tid, px0, py0);
  pixel(tid + kFwdThreads, px1, py1);
  const bool in0 = px0 < cam.W && py0 < cam.H, in1 = px1 < cam.W && py1 < cam.H;
  const float pxc0 = fa((float)px0, 0.5f), pyc0 = fa((float)py0, 0.5f);
  const float pxc1 = fa((float)px1, 0.5f), pyc1 = fa((float)py1, 0.5f);
  __shared__ int s_first;
  uint32_t first_info = rg.x;
  if (args.n_act < args.n) {
    if (tid == 0) s_first = (int)rg.y;
    __syncthreads();
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kFwdThreads) {
      const uint32_t i = b0 + tid;
      if (i < rg.y && args.slot[args.vals[i]] >= 0) atomicMin(&s_first, (int)i);
      if (__syncthreads_or(s_first < (int)rg.y)) break;
    }
    first_info = (uint32_t)s_first;
  }
  if (tid == 0) args.tile_first[gt] = first_info;
  float T0 = 1.0f, T1 = 1.0f;
  uint32_t last0 = rg.x, last1 = rg.x, first0 = kNoEntry, first1 = kNoEntry;
  uint32_t n_eval = 0, n_blend = 0;
  // Per round, a mask of the staged splats that have an information block:
  // warp 0 loads it with the round's copies and stores it before the
  // barrier that opens the round (the slot loads' latency hides behind the
  // round before).
  __shared__ uint32_t s_info[2];
  const bool subset = args.n_act < args.n;
  auto info_mask = [&](uint32_t kk) -> uint32_t {      // warp 0, all lanes
    const uint32_t s = rg.x + kk * kFwd;
    const uint32_t m = min((uint32_t)kFwd, rg.y - s);
    const bool on = (uint32_t)lane < m && (!subset || args.slot[args.vals[s + lane]] >= 0);
    return __ballot_sync(0xffffffffu, on);
  };
  if (first_info < rg.y) {
    bool done0 = !in0, done1 = !in1;
    const uint32_t nst = (rg.y - rg.x + kFwd - 1) / kFwd;
    if (nst > 0 && wq == 0) {
      ring.issue(args, rg.x, rg.y, 0, rec_off, lane, kFwd);
      const uint32_t m0 = info_mask(0);
      if (lane == 0) s_info[0] = m0;
    }
    uint32_t k = 0;
    for (; k < nst; ++k) {
      if (__syncthreads_count(done0 && done1) == kFwdThreads) break;
      uint32_t pend = 0;
      if (k + 1 < nst && wq == 0) {
        ring.issue(args, rg.x, rg.y, k + 1, rec_off, lane, kFwd);
        pend = info_mask(k + 1);
      }
      const int b = (int)(k & 1u);
      if (!ring.wait(b)) done0 = done1 = true;
      const float4* q0 = ring.rec(b, 0, kFwd);
      const float4* q1 = ring.rec(b, 1, kFwd);
      const uint32_t start = rg.x + k * kFwd;
      const uint32_t nj = min((uint32_t)kFwd, rg.y - start);
      const uint32_t imask = s_info[b];
      // the first-splat check only in rounds with an information splat that
      // a pixel of the warp may still need (warp-uniform, so the common
      // rounds run the plain loop)
      const bool watch =
          __any_sync(0xffffffffu, (first0 == kNoEntry && !done0) || (first1 == kNoEntry && !done1)) && imask != 0u;
      auto walk = [&](auto kWatch) {
        // one pixel's blend step with splat j (the decisions as in pass 1)
        auto step = [&](float pxc, float pyc, const float4& a0, const float4& a1, uint32_t j, float& T,
                        uint32_t& last, uint32_t& first, bool& done) {
          const float pw = splat_power(a0.x, a0.y, a1.x, a1.y, a1.z, pxc, pyc);
          ++n_eval;
          if (pw > 0.0f || pw < a0.z) return;
          const float alpha = (pw >= a0.w) ? c.alpha_max : a1.w * __expf(pw);
          const float tt = T * (1.0f - alpha);
          if (tt < c.t_min) { done = true; return; }
          T = tt;
          last = start + j + 1;
          if constexpr (decltype(kWatch)::value) {
            if (first == kNoEntry && ((imask >> j) & 1u)) first = start + j;
          }
          ++n_blend;
        };
        for (uint32_t j = 0; j < nj; ++j) {
          const float4 a0 = q0[j], a1 = q1[j];
          if (!done0) step(pxc0, pyc0, a0, a1, j, T0, last0, first0, done0);
          if (!done1) step(pxc1, pyc1, a0, a1, j, T1, last1, first1, done1);
          if (done0 && done1) break;
        }
      };
      if (!(done0 && done1)) {
        if (watch) walk(std::true_type{});
        else walk(std::false_type{});
      }
      // every warp has read s_info[(k + 1) & 1] of round k - 1 (it passed this
      // round's opening barrier); the next round's barrier publishes the store
      if (k + 1 < nst && wq == 0 && lane == 0) s_info[(k + 1) & 1u] = pend;
    }
    if (k < nst) ring.wait((int)(k & 1u));   // a round fetched ahead but not composited
  }
  uint4* f = args.fwd + (size_t)gt * kTilePix;
  f[tid] = make_uint4(__float_as_uint(T0), in0 ? last0 : rg.x, in0 ? first0 : kNoEntry, 0u);
  f[tid + kFwdThreads] = make_uint4(__float_as_uint(T1), in1 ? last1 : rg.x, in1 ? first1 : kNoEntry, 0u);
  if (args.stats) {
    const unsigned e = __reduce_add_sync(0xffffffffu, n_eval), bl = __reduce_add_sync(0xffffffffu, n_blend);
    if (lane == 0 && e) {
      atomicAdd(&args.stats[0], (unsigned long long)e);
      atomicAdd(&args.stats[1], (unsigned long long)bl);
    }
  }
}

__global__ void __launch_bounds__(kFwdThreads, 8) k_forward(CompositeArgs args, Consts c) {
  __shared__ __align__(16) float4 ring_buf[4 * kFwd];
  __shared__ __align__(8) uint64_t ring_bar[2];
  StageRing ring;
  ring.buf = ring_buf;
  ring.bar = smem_u32(ring_bar);
  ring.use0 = ring.use1 = 0u;
  ring.err = args.err;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ring.bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ring.bar + 8u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (args.queue == nullptr) {
    forward_tile(args, c, args.cam, blockIdx.x, blockIdx.x, args.ranges[blockIdx.x], 0, ring);
    return;
  }
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(args.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= args.n_items) break;
    const uint32_t gt = args.queue[it];
    const int v = args.tile_view[gt];
    const DevCam cam = args.cams[v];
    forward_tile(args, c, cam, (int)(gt - args.tile_base[v]), gt, args.ranges[gt], (size_t)v * args.n, ring);
  }
}

// Dynamic shared memory of k_composite for K objects and rounds of kBatch splats.
inline size_t composite_smem(const Consts& c, int nB, int kBatch) {
  return stage2_offset(c.K, c.KC, nB, kBatch) + stage2_bytes(c.KC, kBatch);
}

// The largest dynamic shared memory a block of this device may opt into.
inline size_t smem_optin() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 48 * 1024;
    }
  }
  return (size_t)v;
}

template <int KCM, int kBatch, bool kSplit>
int launch_k(const CompositeArgs& a, const Consts& c, cudaStream_t st) {
  const size_t sm = composite_smem(c, a.nB, kBatch);
  static size_t attr_set = 0;
  if (attr_set < sm) {
    cudaFuncSetAttribute(k_composite<KCM, kBatch, kSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr_set = sm;
  }
  if (a.queue) {
    int per_sm = 1;
    const int nsm = device_sm_count();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite<KCM, kBatch, kSplit>, kTilePix, sm);
    if (per_sm < 1) per_sm = 1;
    int grid = nsm * per_sm;
    if (grid > a.n_items) grid = a.n_items;
    if (grid <= 0) return 0;
    k_composite<KCM, kBatch, kSplit><<<grid, kTilePix, sm, st>>>(a, c);
    return 1;
  }
  const int ntiles = a.cam.GX * a.cam.GY;
  if (ntiles <= 0) return 0;
  k_composite<KCM, kBatch, kSplit><<<ntiles, kTilePix, sm, st>>>(a, c);
  return 1;
}

template <bool kSplit>
int launch_stage(const CompositeArgs& a, const Consts& c, cudaStream_t st, int stage) {
  // rounds of 32 splats need the most shared memory (many object channels):
  // 16 where 32 does not fit (the stage depth changes only speed)
  if (stage != 16 && composite_smem(c, a.nB, 32) > smem_optin()) stage = 16;
  if (stage == 16) {
    if (c.KC <= 8) return launch_k<8, 16, kSplit>(a, c, st);
    if (c.KC <= 24) return launch_k<24, 16, kSplit>(a, c, st);
    if (c.KC <= 40) return launch_k<40, 16, kSplit>(a, c, st);
    if (c.KC <= 72) return launch_k<72, 16, kSplit>(a, c, st);
    return launch_k<128, 16, kSplit>(a, c, st);
  }
  if (c.KC <= 8) return launch_k<8, 32, kSplit>(a, c, st);
  if (c.KC <= 24) return launch_k<24, 32, kSplit>(a, c, st);
  if (c.KC <= 40) return launch_k<40, 32, kSplit>(a, c, st);
  if (c.KC <= 72) return launch_k<72, 32, kSplit>(a, c, st);
  return launch_k<128, 32, kSplit>(a, c, st);
}

}  // namespace

int launch_composite(const CompositeArgs& a, const Consts& c, cudaStream_t st, int stage) {
  return c.tf32 ? launch_stage<false>(a, c, st, stage) : launch_stage<true>(a, c, st, stage);
}

int launch_forward(const CompositeArgs& a, const Consts& c, cudaStream_t st) {
  if (a.queue) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward, kFwdThreads, 0);
    if (per_sm < 1) per_sm = 1;
    int grid = device_sm_count() * per_sm;
    if (grid > a.n_items) grid = a.n_items;
    if (grid <= 0) return 0;
    k_forward<<<grid, kFwdThreads, 0, st>>>(a, c);
    return 1;
  }
  const int ntiles = a.cam.GX * a.cam.GY;
  if (ntiles <= 0) return 0;
  k_forward<<<ntiles, kFwdThreads, 0, st>>>(a, c);
  return 1;
}

}  // namespace nbv
