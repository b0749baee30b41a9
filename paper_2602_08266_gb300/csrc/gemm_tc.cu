// BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores (tcgen05):
//   D[m][n] = sum_k A(m, k) B(n, k),  A(m, k) = A[m a_sm + k a_sk],  B(n, k) = B[n b_sn + k b_sk]
// the contraction of the learned surrogate's layers (forward, input gradient
// and weight gradient: the strides express every transpose, so one kernel
// serves all five products).
//
// One CTA of 4 warps computes a 128 x NT tile of D with NT <= 256. For every
// block of 64 k the threads stage A (128 x 64) and B (NT x 64) into shared
// memory in the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices of 128 contiguous bytes, core matrices adjacent in k 128
// bytes apart (leading byte offset), 8-row groups 1024 bytes apart (stride
// byte offset). One elected thread then issues four tcgen05.mma (K = 16
// each, M = 128, N = NT, FP32 accumulators in tensor memory) and commits
// them to an mbarrier that every thread waits on (a bounded wait: on a
// time-out the kernel records an error, waits once more with a bound, frees
// its tensor memory and returns). After the last block each warp reads its
// 32 accumulator lanes (rows) with tcgen05.ld and writes D.
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
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

__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16(const __nv_bfloat16* __restrict__ A, int64_t a_sm,
                                                            int64_t a_sk, const __nv_bfloat16* __restrict__ B,
                                                            int64_t b_sn, int64_t b_sk, float* __restrict__ D,
                                                            int64_t ldd, int M, int N, int K, int NT,
                                                            int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sa = smem;                             // 128 x 64 bf16 = 16 KB
  unsigned char* sb = smem + kTM * kKB * 2;             // NT x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb + 256 * kKB * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
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
    // stage the A and B blocks (zero outside the matrices)
    for (int e = tid; e < kTM * kKB; e += kGemmThreads) {
      const int r = e / kKB, k = e - r * kKB;
      const int gm = m0 + r, gk = k0 + k;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (gm < M && gk < K) v = A[(int64_t)gm * a_sm + (int64_t)gk * a_sk];
      *reinterpret_cast<__nv_bfloat16*>(sa + canon_off(r, k)) = v;
    }
    for (int e = tid; e < NT * kKB; e += kGemmThreads) {
      const int r = e / kKB, k = e - r * kKB;
      const int gn = n0 + r, gk = k0 + k;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (gn < N && gk < K) v = B[(int64_t)gn * b_sn + (int64_t)gk * b_sk];
      *reinterpret_cast<__nv_bfloat16*>(sb + canon_off(r, k)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
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
    ok = mbar_wait(smem_u32(bar), (uint32_t)(kb & 1));
    if (!ok && err && lane == 0) atomicExch(err, 1);
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
  }
  if (!ok) {
    // the last commit did not arrive in time: give it one more bounded wait
    // before the tensor memory is released
    mbar_wait(smem_u32(bar), (uint32_t)((nkb - 1) & 1));
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

size_t gemm_bf16_smem() { return (size_t)kTM * kKB * 2 + (size_t)256 * kKB * 2 + 16; }

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
                                               K, NT, err);
  return 1;
}

}  // namespace nbv
