// Throughput of fused multiply-adds on the FP32 pipes: the denominator of
// the compositing kernel's roofline. Every thread runs 8 independent FMA
// chains in registers (enough to cover the pipe latency at 8 warps per
// scheduler), scalar fma.rn.f32 or packed fma.rn.f32x2; nothing is read from
// memory inside the loop, and the chains' sums are stored only when a
// runtime flag that is never set asks for it, so the compiler keeps them.
#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 16384;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_scalar(float a, float b, int store, float* out) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
  }
  float sum = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) sum += x[k];
  if (store) out[blockIdx.x * kThreads + threadIdx.x] = sum;
}

__global__ void __launch_bounds__(kThreads) k_fma_packed(float a, float b, int store, float* out) {
  float2 x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float sum = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) sum += x[k].x + x[k].y;
  if (store) out[blockIdx.x * kThreads + threadIdx.x] = sum;
}

}  // namespace
}  // namespace nbv

extern "C" int nbv_measure_fp32_fma(int packed, void* cuda_stream, double* tflops) {
  if (!tflops) return NBV_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int grid = nbv::device_sm_count() * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return NBV_ERR_CUDA;
  }
  // a <= 1 keeps the chains bounded (no overflow to inf and its slower paths)
  const float a = 0.999999f, b = 1e-6f;
  float ms = 0.0f;
  for (int rep = 0; rep < 2; ++rep) {               // untimed, then timed
    cudaEventRecord(e0, st);
    if (packed)
      nbv::k_fma_packed<<<grid, nbv::kThreads, 0, st>>>(a, b, 0, nullptr);
    else
      nbv::k_fma_scalar<<<grid, nbv::kThreads, 0, st>>>(a, b, 0, nullptr);
    cudaEventRecord(e1, st);
  }
  const cudaError_t err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess || ms <= 0.0f) return NBV_ERR_CUDA;
  const double lane_fmas = (double)grid * nbv::kThreads * nbv::kIters * nbv::kChains * (packed ? 2.0 : 1.0);
  *tflops = 2.0 * lane_fmas / (ms * 1e-3) / 1e12;
  return NBV_OK;
}
