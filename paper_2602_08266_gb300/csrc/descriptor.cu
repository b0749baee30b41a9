// Per-view descriptors for the learned candidate pre-scoring: histograms of
// the projected Gaussian centres over an 8 x 8 image grid (opacity,
// confidence, confidence over depth, confidence discounted by how strongly
// the training views already observe the Gaussian) and of the confidence
// per most probable object id, log-compressed. One pass over the scene per chunk of
// 8 views; the histograms live in shared memory and are added to global
// memory once per block.
#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kDescDim = 384;
constexpr int kViewChunk = 8;

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }

__global__ void k_descriptor_hist(DevScene s, float near_z, const DevCam* __restrict__ cams, int nv,
                                  const float* __restrict__ tblocks, int n_train, int nBp,
                                  float* __restrict__ raw) {
  __shared__ float h[kViewChunk][kDescDim];
  const int v0 = blockIdx.y * kViewChunk;
  const int nvc = min(kViewChunk, nv - v0);
  for (int i = threadIdx.x; i < kViewChunk * kDescDim; i += blockDim.x) (&h[0][0])[i] = 0.0f;
  __syncthreads();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < s.n; g += (int64_t)gridDim.x * blockDim.x) {
    const float4 ms = s.mu_sig[g], ax = s.aux[g];
    const float sig = ms.w, cs = fm(ax.y, ms.w);
    int id = __float_as_int(ax.w);          // the most probable object id, stored as int bits
    id = id < 0 ? 0 : (id > 127 ? 127 : id);
    float obs = 0.0f;                       // sum over training views of sum_pixels w^2
    for (int t = 0; t < n_train; ++t) obs += tblocks[((size_t)t * s.n + g) * nBp + kOffW2];
    const float nov = __fdiv_rn(cs, fa(1.0f, obs));
    for (int q = 0; q < nvc; ++q) {
      const DevCam& c = cams[v0 + q];
      const float tx = fa(fa(fa(fm(c.R[0], ms.x), fm(c.R[1], ms.y)), fm(c.R[2], ms.z)), c.t[0]);
      const float ty = fa(fa(fa(fm(c.R[3], ms.x), fm(c.R[4], ms.y)), fm(c.R[5], ms.z)), c.t[1]);
      const float tz = fa(fa(fa(fm(c.R[6], ms.x), fm(c.R[7], ms.y)), fm(c.R[8], ms.z)), c.t[2]);
      if (!(tz > near_z)) continue;
      const float mx = fa(fm(c.fx, __fdiv_rn(tx, tz)), c.cx);
      const float my = fa(fm(c.fy, __fdiv_rn(ty, tz)), c.cy);
      const float W = (float)c.W, H = (float)c.H;
      if (!(mx >= 0.0f && mx < W && my >= 0.0f && my < H)) continue;
      const int ix = min(7, (int)floorf(__fdiv_rn(fm(8.0f, mx), W)));
      const int iy = min(7, (int)floorf(__fdiv_rn(fm(8.0f, my), H)));
      const int cell = iy * 8 + ix;
      atomicAdd(&h[q][cell], sig);
      atomicAdd(&h[q][64 + cell], cs);
      atomicAdd(&h[q][128 + cell], __fdiv_rn(cs, tz));
      atomicAdd(&h[q][192 + cell], nov);
      atomicAdd(&h[q][256 + id], cs);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvc * kDescDim; i += blockDim.x) {
    const int q = i / kDescDim, f = i - q * kDescDim;
    const float x = h[q][f];
    if (x != 0.0f) atomicAdd(&raw[(size_t)(v0 + q) * kDescDim + f], x);
  }
}

__global__ void k_descriptor_finish(const float* __restrict__ raw, int nv, float cell_scale, float obj_scale,
                                    float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nv * kDescDim) return;
  const int f = (int)(i % kDescDim);
  out[i] = log1pf(raw[i] * (f < 256 ? cell_scale : obj_scale));
}

}  // namespace

int launch_descriptors(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const float* tblocks,
                       int n_train, int nBp, float* raw, float* out, cudaStream_t st) {
  if (nv <= 0) return 0;
  cudaMemsetAsync(raw, 0, sizeof(float) * (size_t)nv * kDescDim, st);
  const int nchunk = (nv + kViewChunk - 1) / kViewChunk;
  int gx = (int)((s.n + 255) / 256);
  const int want = (152 * 8 + nchunk - 1) / nchunk;
  if (gx > want) gx = want;
  if (gx < 1) gx = 1;
  k_descriptor_hist<<<dim3(gx, nchunk), 256, 0, st>>>(s, c.near_z, cams, nv, tblocks, n_train, nBp, raw);
  const int64_t tot = (int64_t)nv * kDescDim;
  k_descriptor_finish<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      raw, nv, (float)(64.0 / (double)s.n), (float)((double)c.KC / (double)s.n), out);
  return 2;
}

}  // namespace nbv
