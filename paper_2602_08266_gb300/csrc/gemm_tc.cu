// BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores (tcgen05):
//   D[m][n] = sum_k A(m, k) B(n, k),  A(m, k) = A[m a_sm + k a_sk],  B(n, k) = B[n b_sn + k b_sk]
// the contraction of the learned surrogate's layers (forward, input gradient
// and weight gradient: the strides express every transpose, so one kernel
// serves all five products).
//
// One CTA of 4 warps computes a 128 x NT tile of D with NT <= 256. For every
// block of 64 k, A (128 x 64) and B (NT x 64) are staged into shared memory
// in the canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices of 128 contiguous bytes, core matrices adjacent in k 128 bytes
// apart (leading byte offset), 8-row groups 1024 bytes apart (stride byte
// offset). Every 16-byte row segment (8 consecutive k of one row) that is
// contiguous and aligned in global memory and lies inside the matrix is
// fetched by a bulk copy of the tensor memory accelerator (cp.async.bulk,
// completed on a staging mbarrier on which every thread arrives with its
// byte count); the other segments (matrix edges, strided operands) are
// loaded by the threads. One elected thread then issues four tcgen05.mma
// (K = 16 each, M = 128, N = NT, FP32 accumulators in tensor memory) and
// commits them to an mbarrier that every thread waits on. Waits are
// bounded: on a time-out the kernel records an error, waits once more with
// a bound for what it has in flight, frees its tensor memory and returns.
// After the last block each warp reads its 32 accumulator lanes (rows) with
// tcgen05.ld and writes D.
#include <cuda_bf16.h>
#include <stdint.h>

#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kTM = 128;        // rows of D per CTA (one tensor-memory lane each)
constexpr int kKB = 64;         // k per staged block
constexpr int kGemmThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row r, k) inside a staged R x 64 block.
__device__ __forceinline__ uint32_t canon_off(int r, int k) {
  return (uint32_t)((((r >> 3) * (kKB / 8)) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version 1
// (46-47), no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((128u >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((1024u >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulate (bits 4-5 = 1), BF16
// A and B (7-9 = 1, 10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22),
// M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Stages row r of one operand's k-block [k0, k0 + 64) (global row gr of a
// rows-x-K matrix with element (row, k) at X[row sx_r + k sx_k]) into the
// canonical layout at dst: 16-byte segments by bulk copy where possible.
// Returns the bytes the bulk copies will deliver to the staging barrier.
__device__ __forceinline__ uint32_t stage_row(const __nv_bfloat16* __restrict__ X, int64_t sx_r, int64_t sx_k,
                                              int rows, int K, int gr, int k0, int r, unsigned char* dst,
                                              uint32_t tbar) {
  uint32_t bytes = 0;
#pragma unroll
  for (int ch = 0; ch < kKB / 8; ++ch) {
    const int gk = k0 + 8 * ch;
    unsigned char* d = dst + canon_off(r, 8 * ch);
    const __nv_bfloat16* src = X + (int64_t)gr * sx_r + (int64_t)gk * sx_k;
    const bool bulk = gr < rows && gk + 8 <= K && sx_k == 1 && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0);
    if (bulk) {
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];"
                   ::"r"(smem_u32(d)), "l"(src), "r"(tbar)
                   : "memory");
      bytes += 16;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (gr < rows && gk + q < K) v = X[(int64_t)gr * sx_r + (int64_t)(gk + q) * sx_k];
        reinterpret_cast<__nv_bfloat16*>(d)[q] = v;
      }
    }
  }
  return bytes;
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16(const __nv_bfloat16* __restrict__ A, int64_t a_sm,
                                                            int64_t a_sk, const __nv_bfloat16* __restrict__ B,
                                                            int64_t b_sn, int64_t b_sk, float* __restrict__ D,
                                                            int64_t ldd, int M, int N, int K, int NT,
                                                            int* __restrict__ err, uint32_t first_polls) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sa = smem;                             // 128 x 64 bf16 = 16 KB
  unsigned char* sb = smem + kTM * kKB * 2;             // NT x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb + 256 * kKB * 2);
  uint64_t* tbar = bar + 1;                             // staging barrier: kGemmThreads arrivals
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * NT;
  const uint32_t ncols = NT <= 32 ? 32u : (NT <= 64 ? 64u : (NT <= 128 ? 128u : 256u));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tbar)), "r"(kGemmThreads) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_bf16(kTM, NT);
  const int nkb = (K + kKB - 1) / kKB;
  bool ok = true;
  for (int kb = 0; kb < nkb && ok; ++kb) {
    const int k0 = kb * kKB;
    // stage the A and B blocks (zero outside the matrices): one row of A and
    // up to two rows of B per thread, then one arrival per thread with the
    // bytes its bulk copies will deliver
    uint32_t bytes = stage_row(A, a_sm, a_sk, M, K, m0 + tid, k0, tid, sa, smem_u32(tbar));
    for (int r = tid; r < NT; r += kGemmThreads) bytes += stage_row(B, b_sn, b_sk, N, K, n0 + r, k0, r, sb, smem_u32(tbar));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(tbar)), "r"(bytes)
                 : "memory");
    bool staged = mbar_wait(smem_u32(tbar), (uint32_t)(kb & 1));
    if (!staged) {
      if (err && lane == 0) atomicExch(err, 1);
      mbar_wait(smem_u32(tbar), (uint32_t)(kb & 1));   // the copies in flight land before the kernel leaves
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(staged ? 1 : 0)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kKB / 16; ++kk) {
        const uint64_t ad = smem_desc(smem_u32(sa) + kk * 256);
        const uint64_t bd = smem_desc(smem_u32(sb) + kk * 256);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(bar))
                   : "memory");
    }
    ok = mbar_wait(smem_u32(bar), (uint32_t)(kb & 1), kb == 0 ? first_polls : kWaitLimit);
    if (!ok && err && lane == 0) atomicExch(err, 1);
    if (!ok) {
      // the commit did not arrive in time: one more bounded wait before the
      // tensor memory is released
      mbar_wait(smem_u32(bar), (uint32_t)(kb & 1));
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
  }
  if (!ok) {
    // nothing more in flight (every wait above was followed by a bounded drain)
  } else if (nkb > 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < NT; c0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                     "=r"(v[7])
                   : "r"(taddr)
                   : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = n0 + c0 + q;
          if (c0 + q < NT && col < N) D[(int64_t)row * ldd + col] = __uint_as_float(v[q]);
        }
      }
    }
  } else {
    // K = 0: D = 0
    const int row = m0 + warp * 32 + lane;
    if (row < M)
      for (int q = 0; q < NT; ++q)
        if (n0 + q < N) D[(int64_t)row * ldd + n0 + q] = 0.0f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace

size_t gemm_bf16_smem() { return (size_t)kTM * kKB * 2 + (size_t)256 * kKB * 2 + 32; }

namespace {
// Polls of the first wait for the tensor cores' commit in a GEMM launch
// (tests of the time-out path set 0: that wait gives up at once; the drain
// wait after it keeps the full bound, so nothing is in flight when the
// tensor memory is released).
uint32_t g_first_polls = kWaitLimit;
}  // namespace

int launch_gemm_bf16(const void* A, int64_t a_sm, int64_t a_sk, const void* B, int64_t b_sn, int64_t b_sk,
                     float* D, int64_t ldd, int M, int N, int K, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return 0;
  // N tile: the largest multiple of 16 <= 256 that splits N evenly enough
  const int ntiles = (N + 255) / 256;
  int NT = (N + ntiles - 1) / ntiles;
  NT = (NT + 15) / 16 * 16;
  const size_t sm = gemm_bf16_smem();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 grid((unsigned)((M + kTM - 1) / kTM), (unsigned)((N + NT - 1) / NT));
  k_gemm_bf16<<<grid, kGemmThreads, sm, st>>>(static_cast<const __nv_bfloat16*>(A), a_sm, a_sk,
                                               static_cast<const __nv_bfloat16*>(B), b_sn, b_sk, D, ldd, M, N,
                                               K, NT, err, g_first_polls);
  return 1;
}

}  // namespace nbv

extern "C" int nbv_set_gemm_wait_polls(int64_t polls) {
  if (polls > (int64_t)0xFFFFFFFF) return NBV_ERR_ARG;
  nbv::g_first_polls = polls < 0 ? nbv::kWaitLimit : (uint32_t)polls;
  return NBV_OK;
}
