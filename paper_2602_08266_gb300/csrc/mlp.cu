// The learned candidate scorer: a 3-layer MLP over per-view descriptors,
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3,
// BF16 weights and activations with FP32 accumulation on the tcgen05 tensor
// cores (gemm_tc.cu), its hand-written backward for the mean squared error
// against exact normalised scores, and Adam on FP32 master weights.
// The exact renderer labels its training data and judges its pruning.
#include <cuda_bf16.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "nbv_internal.cuh"

namespace nbv {
size_t gemm_bf16_smem();
int launch_gemm_bf16(const void* A, int64_t a_sm, int64_t a_sk, const void* B, int64_t b_sn, int64_t b_sk,
                     float* D, int64_t ldd, int M, int N, int K, int* err, cudaStream_t st);

namespace {

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

// out[m][n] = bf16(relu(Z[m][n] + b[n]))
__global__ void k_bias_relu(const float* __restrict__ Z, const float* __restrict__ b, int rows, int w,
                            __nv_bfloat16* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * w) return;
  const float v = Z[i] + b[i % w];
  out[i] = __float2bfloat16(v > 0.0f ? v : 0.0f);
}

// y[m] = w3 . h2[m] + b3, one warp per row
__global__ void k_head(const __nv_bfloat16* __restrict__ H2, const float* __restrict__ w3, const float* b3,
                       int rows, int w, float* __restrict__ y) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= rows) return;
  float a = 0.0f;
  for (int n = lane; n < w; n += 32) a += __bfloat162float(H2[(int64_t)row * w + n]) * w3[n];
  for (int o = 16; o >= 1; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) y[row] = a + b3[0];
}

// dy = 2 (y - t) / B; dZ2 = dy w3 [h2 > 0] (FP32 and BF16 copies)
__global__ void k_head_grad(const float* __restrict__ y, const float* __restrict__ t, int rows, int w,
                            const float* __restrict__ w3, const __nv_bfloat16* __restrict__ H2,
                            float* __restrict__ dy, float* __restrict__ dZf, __nv_bfloat16* __restrict__ dZb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * w) return;
  const int m = (int)(i / w), n = (int)(i - (int64_t)m * w);
  const float g = 2.0f * (y[m] - t[m]) / (float)rows;
  if (n == 0) dy[m] = g;
  const float d = __bfloat162float(H2[i]) > 0.0f ? g * w3[n] : 0.0f;
  dZf[i] = d;
  dZb[i] = __float2bfloat16(d);
}

// dZ1 = dH1 [h1 > 0]
__global__ void k_relu_grad(const float* __restrict__ dH, const __nv_bfloat16* __restrict__ H, int64_t n,
                            float* __restrict__ dZf, __nv_bfloat16* __restrict__ dZb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float d = __bfloat162float(H[i]) > 0.0f ? dH[i] : 0.0f;
  dZf[i] = d;
  dZb[i] = __float2bfloat16(d);
}

// out[n] = sum_m X[m][n] * (s ? s[m] : 1), one thread per column (double sum)
__global__ void k_colsum(const float* __restrict__ X, const __nv_bfloat16* __restrict__ Xb,
                         const float* __restrict__ s, int rows, int w, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= w) return;
  double a = 0.0;
  for (int m = 0; m < rows; ++m) {
    const float x = X ? X[(int64_t)m * w + n] : __bfloat162float(Xb[(int64_t)m * w + n]);
    a += (double)x * (s ? (double)s[m] : 1.0);
  }
  out[n] = (float)a;
}

// mean squared error (double)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, int rows, double* out) {
  __shared__ double sm[256];
  double a = 0.0;
  for (int m = threadIdx.x; m < rows; m += 256) {
    const double d = (double)y[m] - (double)t[m];
    a += d * d;
  }
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int h = 128; h >= 1; h >>= 1) {
    if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0] / (double)(rows > 0 ? rows : 1);
}

// Adam (Kingma & Ba) on FP32 master weights: m <- b1 m + (1 - b1) g,
// v <- b2 v + (1 - b2) g^2, p <- p - lr mhat / (sqrt(vhat) + eps)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace nbv

struct nbv_mlp {
  int d_in = 0, width = 0;
  int64_t P = 0;                 // parameters: W1 [w][d_in], b1 [w], W2 [w][w], b2 [w], w3 [w], b3 [1]
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, ow3 = 0, ob3 = 0;
  cudaStream_t st = nullptr;
  float* params = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int64_t step = 0;
  __nv_bfloat16* W1b = nullptr;
  __nv_bfloat16* W2b = nullptr;
  int cap = 0;                   // rows the activation buffers hold
  __nv_bfloat16 *Xb = nullptr, *H1b = nullptr, *H2b = nullptr, *dZ1b = nullptr, *dZ2b = nullptr;
  float *Z = nullptr, *dZ1f = nullptr, *dZ2f = nullptr, *y = nullptr, *dy = nullptr;
  int* d_err = nullptr;
  double* d_loss = nullptr;
};

namespace {

using nbv::blocks;

template <class T>
bool dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n > 0 ? n : 1)) == cudaSuccess;
}

void free_acts(nbv_mlp* q) {
  void* ps[] = {q->Xb, q->H1b, q->H2b, q->dZ1b, q->dZ2b, q->Z, q->dZ1f, q->dZ2f, q->y, q->dy};
  for (void* p : ps)
    if (p) cudaFree(p);
  q->Xb = q->H1b = q->H2b = q->dZ1b = q->dZ2b = nullptr;
  q->Z = q->dZ1f = q->dZ2f = q->y = q->dy = nullptr;
  q->cap = 0;
}

int ensure_rows(nbv_mlp* q, int rows) {
  if (rows <= q->cap) return NBV_OK;
  free_acts(q);
  const size_t w = (size_t)q->width, r = (size_t)rows;
  if (!dalloc(&q->Xb, r * q->d_in) || !dalloc(&q->H1b, r * w) || !dalloc(&q->H2b, r * w) ||
      !dalloc(&q->dZ1b, r * w) || !dalloc(&q->dZ2b, r * w) || !dalloc(&q->Z, r * w) || !dalloc(&q->dZ1f, r * w) ||
      !dalloc(&q->dZ2f, r * w) || !dalloc(&q->y, r) || !dalloc(&q->dy, r))
    return NBV_ERR_OOM;
  q->cap = rows;
  return NBV_OK;
}

void refresh_bf16(nbv_mlp* q) {
  const int64_t n1 = (int64_t)q->width * q->d_in, n2 = (int64_t)q->width * q->width;
  nbv::k_to_bf16<<<blocks(n1), 256, 0, q->st>>>(q->params + q->oW1, q->W1b, n1);
  nbv::k_to_bf16<<<blocks(n2), 256, 0, q->st>>>(q->params + q->oW2, q->W2b, n2);
}

// splitmix64 (Steele, Lea and Flood): the seeded initial weights
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Forward pass over `rows` descriptors (device FP32 [rows][d_in]) into q->y.
int forward(nbv_mlp* q, const float* x, int rows) {
  const int w = q->width, d = q->d_in;
  cudaStream_t st = q->st;
  nbv::k_to_bf16<<<blocks((int64_t)rows * d), 256, 0, st>>>(x, q->Xb, (int64_t)rows * d);
  nbv::launch_gemm_bf16(q->Xb, d, 1, q->W1b, d, 1, q->Z, w, rows, w, d, q->d_err, st);
  nbv::k_bias_relu<<<blocks((int64_t)rows * w), 256, 0, st>>>(q->Z, q->params + q->ob1, rows, w, q->H1b);
  nbv::launch_gemm_bf16(q->H1b, w, 1, q->W2b, w, 1, q->Z, w, rows, w, w, q->d_err, st);
  nbv::k_bias_relu<<<blocks((int64_t)rows * w), 256, 0, st>>>(q->Z, q->params + q->ob2, rows, w, q->H2b);
  nbv::k_head<<<blocks((int64_t)rows * 32), 256, 0, st>>>(q->H2b, q->params + q->ow3, q->params + q->ob3, rows, w,
                                                          q->y);
  return cudaGetLastError() == cudaSuccess ? NBV_OK : NBV_ERR_CUDA;
}

// Forward + backward of the mean squared error against t (device [rows]);
// gradients into q->grads, loss into q->d_loss.
int backward(nbv_mlp* q, const float* x, const float* t, int rows) {
  int rc = forward(q, x, rows);
  if (rc != NBV_OK) return rc;
  const int w = q->width, d = q->d_in;
  cudaStream_t st = q->st;
  float* g = q->grads;
  nbv::k_mse<<<1, 256, 0, st>>>(q->y, t, rows, q->d_loss);
  nbv::k_head_grad<<<blocks((int64_t)rows * w), 256, 0, st>>>(q->y, t, rows, w, q->params + q->ow3, q->H2b, q->dy,
                                                               q->dZ2f, q->dZ2b);
  // d w3 = sum_m dy_m h2_m, d b3 = sum_m dy_m, d b2 = sum_m dZ2_m
  nbv::k_colsum<<<blocks(w), 256, 0, st>>>(nullptr, q->H2b, q->dy, rows, w, g + q->ow3);
  nbv::k_colsum<<<1, 32, 0, st>>>(q->dy, nullptr, nullptr, rows, 1, g + q->ob3);
  nbv::k_colsum<<<blocks(w), 256, 0, st>>>(q->dZ2f, nullptr, nullptr, rows, w, g + q->ob2);
  // d W2 [o][i] = sum_m dZ2[m][o] h1[m][i]
  nbv::launch_gemm_bf16(q->dZ2b, 1, w, q->H1b, 1, w, g + q->oW2, w, w, w, rows, q->d_err, st);
  // d h1 [m][i] = sum_o dZ2[m][o] W2[o][i], then the relu mask
  nbv::launch_gemm_bf16(q->dZ2b, w, 1, q->W2b, 1, w, q->Z, w, rows, w, w, q->d_err, st);
  nbv::k_relu_grad<<<blocks((int64_t)rows * w), 256, 0, st>>>(q->Z, q->H1b, (int64_t)rows * w, q->dZ1f, q->dZ1b);
  nbv::k_colsum<<<blocks(w), 256, 0, st>>>(q->dZ1f, nullptr, nullptr, rows, w, g + q->ob1);
  // d W1 [o][i] = sum_m dZ1[m][o] x[m][i]
  nbv::launch_gemm_bf16(q->dZ1b, 1, w, q->Xb, 1, d, g + q->oW1, d, w, d, rows, q->d_err, st);
  return cudaGetLastError() == cudaSuccess ? NBV_OK : NBV_ERR_CUDA;
}

int check_err(nbv_mlp* q) {
  int h = 0;
  if (cudaMemcpyAsync(&h, q->d_err, sizeof(int), cudaMemcpyDeviceToHost, q->st) != cudaSuccess) return NBV_ERR_CUDA;
  if (cudaStreamSynchronize(q->st) != cudaSuccess) return NBV_ERR_CUDA;
  return h ? NBV_ERR_TIMEOUT : NBV_OK;
}

}  // namespace

extern "C" {

int nbv_mlp_create(int d_in, int width, uint64_t seed, void* cuda_stream, nbv_mlp** out) {
  if (!out) return NBV_ERR_ARG;
  *out = nullptr;
  if (d_in < 1 || d_in > 4096 || width < 16 || width > 256 || width % 16 != 0) return NBV_ERR_ARG;
  nbv_mlp* q = new nbv_mlp();
  q->d_in = d_in;
  q->width = width;
  q->st = static_cast<cudaStream_t>(cuda_stream);
  q->oW1 = 0;
  q->ob1 = q->oW1 + (int64_t)width * d_in;
  q->oW2 = q->ob1 + width;
  q->ob2 = q->oW2 + (int64_t)width * width;
  q->ow3 = q->ob2 + width;
  q->ob3 = q->ow3 + width;
  q->P = q->ob3 + 1;
  std::vector<float> h((size_t)q->P, 0.0f);
  uint64_t s = seed;
  auto uni = [&](double a) { return (float)(a * (2.0 * ((double)(splitmix(s) >> 11) * 0x1.0p-53) - 1.0)); };
  for (int64_t i = 0; i < (int64_t)width * d_in; ++i) h[q->oW1 + i] = uni(std::sqrt(6.0 / d_in));
  for (int64_t i = 0; i < (int64_t)width * width; ++i) h[q->oW2 + i] = uni(std::sqrt(6.0 / width));
  for (int i = 0; i < width; ++i) h[q->ow3 + i] = uni(std::sqrt(3.0 / width));
  bool ok = dalloc(&q->params, q->P) && dalloc(&q->grads, q->P) && dalloc(&q->m, q->P) && dalloc(&q->v, q->P) &&
            dalloc(&q->W1b, (size_t)width * d_in) && dalloc(&q->W2b, (size_t)width * width) &&
            dalloc(&q->d_err, 1) && dalloc(&q->d_loss, 1);
  if (ok) {
    ok = cudaMemcpyAsync(q->params, h.data(), sizeof(float) * q->P, cudaMemcpyHostToDevice, q->st) == cudaSuccess &&
         cudaMemsetAsync(q->grads, 0, sizeof(float) * q->P, q->st) == cudaSuccess &&
         cudaMemsetAsync(q->m, 0, sizeof(float) * q->P, q->st) == cudaSuccess &&
         cudaMemsetAsync(q->v, 0, sizeof(float) * q->P, q->st) == cudaSuccess &&
         cudaMemsetAsync(q->d_err, 0, sizeof(int), q->st) == cudaSuccess;
    refresh_bf16(q);
    ok = ok && cudaStreamSynchronize(q->st) == cudaSuccess;
  }
  if (!ok) {
    nbv_mlp_destroy(q);
    return NBV_ERR_OOM;
  }
  *out = q;
  return NBV_OK;
}

void nbv_mlp_destroy(nbv_mlp* q) {
  if (!q) return;
  cudaStreamSynchronize(q->st);
  free_acts(q);
  void* ps[] = {q->params, q->grads, q->m, q->v, q->W1b, q->W2b, q->d_err, q->d_loss};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete q;
}

int64_t nbv_mlp_num_params(const nbv_mlp* q) { return q ? q->P : 0; }

int nbv_mlp_get_params(nbv_mlp* q, float* out) {
  if (!q || !out) return NBV_ERR_ARG;
  if (cudaMemcpyAsync(out, q->params, sizeof(float) * q->P, cudaMemcpyDeviceToDevice, q->st) != cudaSuccess)
    return NBV_ERR_CUDA;
  return NBV_OK;
}

int nbv_mlp_set_params(nbv_mlp* q, const float* in) {
  if (!q || !in) return NBV_ERR_ARG;
  if (cudaMemcpyAsync(q->params, in, sizeof(float) * q->P, cudaMemcpyDeviceToDevice, q->st) != cudaSuccess)
    return NBV_ERR_CUDA;
  refresh_bf16(q);
  return cudaGetLastError() == cudaSuccess ? NBV_OK : NBV_ERR_CUDA;
}

int nbv_mlp_forward(nbv_mlp* q, const float* x, int rows, float* y) {
  if (!q || (rows > 0 && (!x || !y)) || rows < 0) return NBV_ERR_ARG;
  if (rows == 0) return NBV_OK;
  int rc = ensure_rows(q, rows);
  if (rc != NBV_OK) return rc;
  rc = forward(q, x, rows);
  if (rc != NBV_OK) return rc;
  if (cudaMemcpyAsync(y, q->y, sizeof(float) * rows, cudaMemcpyDeviceToDevice, q->st) != cudaSuccess)
    return NBV_ERR_CUDA;
  return check_err(q);
}

int nbv_mlp_gradients(nbv_mlp* q, const float* x, const float* t, int rows, float* grads, double* loss) {
  if (!q || rows < 1 || !x || !t) return NBV_ERR_ARG;
  int rc = ensure_rows(q, rows);
  if (rc != NBV_OK) return rc;
  rc = backward(q, x, t, rows);
  if (rc != NBV_OK) return rc;
  if (grads && cudaMemcpyAsync(grads, q->grads, sizeof(float) * q->P, cudaMemcpyDeviceToDevice, q->st) != cudaSuccess)
    return NBV_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, q->d_loss, sizeof(double), cudaMemcpyDeviceToHost, q->st) != cudaSuccess)
    return NBV_ERR_CUDA;
  return check_err(q);
}

int nbv_mlp_train_step(nbv_mlp* q, const float* x, const float* t, int rows, float lr, double* loss) {
  if (!q || rows < 1 || !x || !t || !(lr > 0.0f)) return NBV_ERR_ARG;
  int rc = ensure_rows(q, rows);
  if (rc != NBV_OK) return rc;
  rc = backward(q, x, t, rows);
  if (rc != NBV_OK) return rc;
  q->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)q->step)), c2 = (float)(1.0 - std::pow(0.999, (double)q->step));
  nbv::k_adam<<<blocks(q->P), 256, 0, q->st>>>(q->params, q->grads, q->m, q->v, q->P, lr, b1, b2, 1e-8f, c1, c2);
  refresh_bf16(q);
  if (cudaGetLastError() != cudaSuccess) return NBV_ERR_CUDA;
  if (loss) {
    if (cudaMemcpyAsync(loss, q->d_loss, sizeof(double), cudaMemcpyDeviceToHost, q->st) != cudaSuccess)
      return NBV_ERR_CUDA;
    return check_err(q);
  }
  return NBV_OK;
}

int nbv_gemm_bf16(const uint16_t* A, int64_t a_sm, int64_t a_sk, const uint16_t* B, int64_t b_sn, int64_t b_sk,
                  float* D, int64_t ldd, int M, int N, int K, int* d_err, void* cuda_stream) {
  if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!D || (K > 0 && (!A || !B))))) return NBV_ERR_ARG;
  nbv::launch_gemm_bf16(A, a_sm, a_sk, B, b_sn, b_sk, D, ldd, M, N, K, d_err, static_cast<cudaStream_t>(cuda_stream));
  return cudaGetLastError() == cudaSuccess ? NBV_OK : NBV_ERR_CUDA;
}

}  // extern "C"
