// Per-view descriptors for the learned candidate pre-scoring: histograms of
// the projected Gaussian centres over an 8 x 8 image grid (opacity,
// confidence, confidence over depth, confidence discounted by how strongly
// the training views already observe the Gaussian, confidence weighted by
// the angular novelty of the viewing direction against the training
// cameras), of the confidence per most probable object id, and view totals,
// log-compressed. One pass over the scene per chunk of
// 8 views; the histograms live in shared memory and are added to global
// memory once per block.
#include "nbv_internal.cuh"

namespace nbv {
namespace {

constexpr int kDescDim = 448;
constexpr int kViewChunk = 8;
constexpr int kMaxTrainDirs = 64;   // training cameras the angular novelty looks at
constexpr int kObjBins = 56;

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }

// Feature layout (per view): 8 x 8 image cells c of the projected centre,
//   [0, 64)    sigma
//   [64, 128)  c_g sigma
//   [128, 192) c_g sigma / z
//   [192, 256) c_g sigma / (1 + o_g)          o_g: training observation
//   [256, 320) c_g sigma nu                   nu: angular novelty
//   [320, 384) c_g sigma nu^2
//   [384, 440) c_g sigma per most probable object id (ids >= 55 share the last bin)
//   [440, 448) view totals: c_g sigma nu, c_g sigma [nu > 0.1], c_g sigma [nu > 0.3],
//              c_g sigma sqrt(nu), sigma, c_g sigma, c_g sigma / (1 + o_g), c_g sigma / z
// with nu = 1 - max over training cameras of the cosine between the
// directions from the camera centres to the Gaussian (candidate vs training).
__global__ void k_descriptor_hist(DevScene s, float near_z, const DevCam* __restrict__ cams, int nv,
                                  const DevCam* __restrict__ tcams, int n_train, const float* __restrict__ tblocks,
                                  int nBp, float* __restrict__ raw) {
  __shared__ float h[kViewChunk][kDescDim];
  __shared__ float tc[kMaxTrainDirs][3];
  const int v0 = blockIdx.y * kViewChunk;
  const int nvc = min(kViewChunk, nv - v0);
  const int ntd = min(n_train, kMaxTrainDirs);
  for (int i = threadIdx.x; i < kViewChunk * kDescDim; i += blockDim.x) (&h[0][0])[i] = 0.0f;
  for (int i = threadIdx.x; i < ntd * 3; i += blockDim.x) tc[i / 3][i % 3] = tcams[i / 3].campos[i % 3];
  __syncthreads();
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < s.n; g += (int64_t)gridDim.x * blockDim.x) {
    const float4 ms = s.mu_sig[g], ax = s.aux[g];
    const float sig = ms.w, cs = fm(ax.y, ms.w);
    int id = __float_as_int(ax.w);          // the most probable object id, stored as int bits
    id = id < 0 ? 0 : (id >= kObjBins ? kObjBins - 1 : id);
    float obs = 0.0f;                       // sum over training views of sum_pixels w^2
    const int sl = s.slot[g];            // training blocks exist for active Gaussians only
    if (sl >= 0)
      for (int t = 0; t < n_train; ++t) obs += tblocks[((size_t)t * s.n_act + sl) * nBp + kOffW2];
    const float cov = __fdiv_rn(cs, fa(1.0f, obs));
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
      // angular novelty against the training cameras
      const float dx = ms.x - c.campos[0], dy = ms.y - c.campos[1], dz = ms.z - c.campos[2];
      const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
      float best = -1.0f;
      for (int t = 0; t < ntd; ++t) {
        const float ex = ms.x - tc[t][0], ey = ms.y - tc[t][1], ez = ms.z - tc[t][2];
        const float jl = rsqrtf(ex * ex + ey * ey + ez * ez);
        best = fmaxf(best, (dx * ex + dy * ey + dz * ez) * il * jl);
      }
      const float nu = ntd > 0 ? fmaxf(0.0f, 1.0f - best) : 1.0f;
      const float csz = __fdiv_rn(cs, tz);
      float* hq = h[q];
      atomicAdd(&hq[cell], sig);
      atomicAdd(&hq[64 + cell], cs);
      atomicAdd(&hq[128 + cell], csz);
      atomicAdd(&hq[192 + cell], cov);
      atomicAdd(&hq[256 + cell], cs * nu);
      atomicAdd(&hq[320 + cell], cs * nu * nu);
      atomicAdd(&hq[384 + id], cs);
      atomicAdd(&hq[440], cs * nu);
      if (nu > 0.1f) atomicAdd(&hq[441], cs);
      if (nu > 0.3f) atomicAdd(&hq[442], cs);
      atomicAdd(&hq[443], cs * sqrtf(nu));
      atomicAdd(&hq[444], sig);
      atomicAdd(&hq[445], cs);
      atomicAdd(&hq[446], cov);
      atomicAdd(&hq[447], csz);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvc * kDescDim; i += blockDim.x) {
    const int q = i / kDescDim, f = i - q * kDescDim;
    const float x = h[q][f];
    if (x != 0.0f) atomicAdd(&raw[(size_t)(v0 + q) * kDescDim + f], x);
  }
}

// log(1 + s x): s = 64 / n for the cell features and 1 / n for the totals,
// (K + 1) / n for the object bins
__global__ void k_descriptor_finish(const float* __restrict__ raw, int nv, float cell_scale, float obj_scale,
                                    float tot_scale, float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nv * kDescDim) return;
  const int f = (int)(i % kDescDim);
  out[i] = log1pf(raw[i] * (f < 384 ? cell_scale : (f < 440 ? obj_scale : tot_scale)));
}

}  // namespace

int launch_descriptors(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const DevCam* tcams,
                       int n_train, const float* tblocks, int nBp, float* raw, float* out, cudaStream_t st) {
  if (nv <= 0) return 0;
  cudaMemsetAsync(raw, 0, sizeof(float) * (size_t)nv * kDescDim, st);
  const int nchunk = (nv + kViewChunk - 1) / kViewChunk;
  int gx = (int)((s.n + 255) / 256);
  const int want = (device_sm_count() * 8 + nchunk - 1) / nchunk;
  if (gx > want) gx = want;
  if (gx < 1) gx = 1;
  k_descriptor_hist<<<dim3(gx, nchunk), 256, 0, st>>>(s, c.near_z, cams, nv, tcams, n_train, tblocks, nBp, raw);
  const int64_t tot = (int64_t)nv * kDescDim;
  k_descriptor_finish<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      raw, nv, (float)(64.0 / (double)s.n), (float)((double)c.KC / (double)s.n), (float)(1.0 / (double)s.n), out);
  return 2;
}

}  // namespace nbv
