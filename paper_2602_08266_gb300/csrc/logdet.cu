// Information gain from the structured 2D blocks (Eqs. 5-12).
//
// For Gaussian g, output f in {rgb, d, o} and view v, the Gauss-Newton block
// in the raw parameters theta_f is A^f_vg = M^T B^f_vg M, where B is the 2D
// block the compositing kernel reduced (in u = (mx, my, A, B, C, sigma,
// colour | z | p_1..p_K)) and M = d u / d theta_f is the projection
// Jacobian of that view (recomputed here, never stored).
//
// Training state (once per NBV step):
//   H^f_g = lambda I + c_g sum_t M_t^T B_t M_t          (Eqs. 6, 9 with C_g = c_g I)
// Jacobi-scaled, H~ = D^-1/2 H D^-1/2, and Cholesky-factorised in double
// precision, H~ = L L^T; L^-1 (the colour SH blocks inverted in double, the
// other triangles in single precision from the double factor) is kept in
// single precision.
//
// Per view, by Sylvester's determinant identity,
//   log det(H + c A) - log det H = log det(I_u + c W B),
//   W = M H^-1 M^T = Z^T Z,  Z = L^-1 D^-1/2 M^T,
// a sparse l x u product and a u x u determinant instead of an l x l
// factorisation (u = 9 against l = 59 for colour at SH degree 3). The
// columns of D^-1/2 M^T are sparse by parameter block: the geometric rows
// (mean, scale, rotation, opacity) are dense, an SH row feeds one colour
// channel only, an object-logit row feeds the probability columns only.
// The gains of all Gaussians summed give IG_f(T, v) (block-diagonal
// determinant, Sec. III-B.1); the training mean normalises each output
// (Eq. 10) and the weighted sum (Eq. 11) is maximised (Eq. 5).
#include <math.h>

#include <type_traits>

#include "nbv_internal.cuh"

namespace nbv {
namespace {


struct GJac {
  float Jm[2][3];    // d(mx,my)/d mu
  float Jc[3][10];   // d(A,B,C)/d(mu, log s, q)
  float Jz[3];       // d z / d mu
  float dsig;        // d sigma / d rho
  float Jrgb[3][3];  // d rgb / d mu
  float live[3];     // 1 where the colour is not clamped at 0
  float Y[16];       // SH basis at the view direction
};

struct SHC {
  float c0, c1, c2a, c2b, c2c, c3a, c3b, c3c, c3d, c3e;
};
__device__ __forceinline__ SHC shc() {
  SHC k;
  k.c0 = (float)(0.5 / 1.7724538509055160273);
  k.c1 = (float)0.48860251190291992159;
  k.c2a = (float)(0.5 * 3.8729833462074168852 / 1.7724538509055160273);
  k.c2b = (float)(0.25 * 2.2360679774997896964 / 1.7724538509055160273);
  k.c2c = (float)(0.25 * 3.8729833462074168852 / 1.7724538509055160273);
  k.c3a = (float)(0.25 * 2.3601743597065740);
  k.c3b = (float)(0.5 * 5.7812228852811080);
  k.c3c = (float)(0.25 * 1.8281831978578629);
  k.c3d = (float)(0.25 * 1.4927053303604616);
  k.c3e = (float)(0.25 * 5.7812228852811080);
  return k;
}

// Real SH values and gradients (of the polynomial forms) at direction (x,y,z).
__device__ __forceinline__ void sh_val_grad(int deg, float x, float y, float z, float* Y, float (*G)[3]) {
  const SHC k = shc();
#pragma unroll
  for (int i = 0; i < 16; ++i) { Y[i] = 0.0f; G[i][0] = G[i][1] = G[i][2] = 0.0f; }
  Y[0] = k.c0;
  if (deg < 1) return;
  Y[1] = -k.c1 * y; G[1][1] = -k.c1;
  Y[2] = k.c1 * z;  G[2][2] = k.c1;
  Y[3] = -k.c1 * x; G[3][0] = -k.c1;
  if (deg < 2) return;
  Y[4] = k.c2a * x * y;  G[4][0] = k.c2a * y; G[4][1] = k.c2a * x;
  Y[5] = -k.c2a * y * z; G[5][1] = -k.c2a * z; G[5][2] = -k.c2a * y;
  Y[6] = k.c2b * (2.0f * z * z - x * x - y * y);
  G[6][0] = -2.0f * k.c2b * x; G[6][1] = -2.0f * k.c2b * y; G[6][2] = 4.0f * k.c2b * z;
  Y[7] = -k.c2a * x * z; G[7][0] = -k.c2a * z; G[7][2] = -k.c2a * x;
  Y[8] = k.c2c * (x * x - y * y); G[8][0] = 2.0f * k.c2c * x; G[8][1] = -2.0f * k.c2c * y;
  if (deg < 3) return;
  Y[9] = -k.c3a * y * (3.0f * x * x - y * y);
  G[9][0] = -6.0f * k.c3a * x * y; G[9][1] = -k.c3a * (3.0f * x * x - 3.0f * y * y);
  Y[10] = k.c3b * x * y * z;
  G[10][0] = k.c3b * y * z; G[10][1] = k.c3b * x * z; G[10][2] = k.c3b * x * y;
  Y[11] = -k.c3c * y * (4.0f * z * z - x * x - y * y);
  G[11][0] = 2.0f * k.c3c * x * y; G[11][1] = -k.c3c * (4.0f * z * z - x * x - 3.0f * y * y);
  G[11][2] = -8.0f * k.c3c * y * z;
  Y[12] = k.c3d * z * (2.0f * z * z - 3.0f * x * x - 3.0f * y * y);
  G[12][0] = -6.0f * k.c3d * x * z; G[12][1] = -6.0f * k.c3d * y * z;
  G[12][2] = k.c3d * (6.0f * z * z - 3.0f * x * x - 3.0f * y * y);
  Y[13] = -k.c3c * x * (4.0f * z * z - x * x - y * y);
  G[13][0] = -k.c3c * (4.0f * z * z - 3.0f * x * x - y * y); G[13][1] = 2.0f * k.c3c * x * y;
  G[13][2] = -8.0f * k.c3c * x * z;
  Y[14] = k.c3e * z * (x * x - y * y);
  G[14][0] = 2.0f * k.c3e * x * z; G[14][1] = -2.0f * k.c3e * y * z; G[14][2] = k.c3e * (x * x - y * y);
  Y[15] = -k.c3a * x * (x * x - 3.0f * y * y);
  G[15][0] = -k.c3a * (3.0f * x * x - 3.0f * y * y); G[15][1] = 6.0f * k.c3a * x * y;
}

// Projection Jacobians of Gaussian g in view cam (values in single precision).
// DEG >= 0 fixes the SH degree at compile time (everything stays in
// registers); DEG = -1 reads it from c.
template <int DEG>
__device__ __forceinline__ void compute_gjac_t(const DevScene& s, const Consts& c, const DevCam& cam, int64_t g,
                                               GJac& J) {
  const int deg = DEG >= 0 ? DEG : c.deg;
  const int nb = (deg + 1) * (deg + 1);
  const float4 ms = s.mu_sig[g], ss = s.scale_skip[g], qq = s.qn[g], ax = s.aux[g];
  const float* R = cam.R;
  const float mu[3] = {ms.x, ms.y, ms.z};
  float tc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) tc[i] = R[3 * i] * mu[0] + R[3 * i + 1] * mu[1] + R[3 * i + 2] * mu[2] + cam.t[i];
  const float x = tc[0], y = tc[1], z = tc[2];
  const float iz = 1.0f / z, iz2 = iz * iz;
  // mean: d(mx,my)/d t, then * R
  const float dmx[3] = {cam.fx * iz, 0.0f, -cam.fx * x * iz2};
  const float dmy[3] = {0.0f, cam.fy * iz, -cam.fy * y * iz2};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    J.Jm[0][m] = dmx[0] * R[m] + dmx[1] * R[3 + m] + dmx[2] * R[6 + m];
    J.Jm[1][m] = dmy[0] * R[m] + dmy[1] * R[3 + m] + dmy[2] * R[6 + m];
    J.Jz[m] = R[6 + m];
  }
  // perspective Jacobian with the guard band
  const float limx = c.guard * (0.5f * (float)cam.W / cam.fx);
  const float limy = c.guard * (0.5f * (float)cam.H / cam.fy);
  const float xr = x * iz, yr = y * iz;
  const bool clx = fabsf(xr) > limx, cly = fabsf(yr) > limy;
  const float xz = fminf(limx, fmaxf(-limx, xr)), yz = fminf(limy, fmaxf(-limy, yr));
  const float j00 = cam.fx * iz, j02 = -cam.fx * xz * iz;
  const float j11 = cam.fy * iz, j12 = -cam.fy * yz * iz;
  float T0[3], T1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T0[i] = j00 * R[i] + j02 * R[6 + i];
    T1[i] = j11 * R[3 + i] + j12 * R[6 + i];
  }
  // derivatives of j00, j02, j11, j12 w.r.t. t = (x, y, z)
  float dj00[3] = {0.0f, 0.0f, -cam.fx * iz2};
  float dj02[3], dj12[3];
  if (clx) { dj02[0] = 0.0f; dj02[1] = 0.0f; dj02[2] = -j02 * iz; }
  else { dj02[0] = -cam.fx * iz2; dj02[1] = 0.0f; dj02[2] = 2.0f * cam.fx * x * iz2 * iz; }
  float dj11[3] = {0.0f, 0.0f, -cam.fy * iz2};
  if (cly) { dj12[0] = 0.0f; dj12[1] = 0.0f; dj12[2] = -j12 * iz; }
  else { dj12[0] = 0.0f; dj12[1] = -cam.fy * iz2; dj12[2] = 2.0f * cam.fy * y * iz2 * iz; }
  // rotation of the Gaussian and Sigma3
  const float qw = qq.x, qx = qq.y, qy = qq.z, qz = qq.w;
  const float Rq[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - qw * qz), 2.0f * (qx * qz + qw * qy),
                       2.0f * (qx * qy + qw * qz), 1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - qw * qx),
                       2.0f * (qx * qz - qw * qy), 2.0f * (qy * qz + qw * qx), 1.0f - 2.0f * (qx * qx + qy * qy)};
  const float s2[3] = {ss.x * ss.x, ss.y * ss.y, ss.z * ss.z};
  float S3[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      S3[3 * i + j] = Rq[3 * i] * s2[0] * Rq[3 * j] + Rq[3 * i + 1] * s2[1] * Rq[3 * j + 1] +
                      Rq[3 * i + 2] * s2[2] * Rq[3 * j + 2];
  float ST0[3], ST1[3];  // Sigma3 T0^T, Sigma3 T1^T
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ST0[i] = S3[3 * i] * T0[0] + S3[3 * i + 1] * T0[1] + S3[3 * i + 2] * T0[2];
    ST1[i] = S3[3 * i] * T1[0] + S3[3 * i + 1] * T1[1] + S3[3 * i + 2] * T1[2];
  }
  const float a = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + c.dilation;
  const float b = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
  const float cc = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + c.dilation;
  const float det = a * cc - b * b;
  const float A = cc / det, B = -b / det, C = a / det;
  // d conic = -Q dSigma2 Q
  auto dconic = [&](float da, float db, float dc, float* out) {
    out[0] = -(A * A * da + 2.0f * A * B * db + B * B * dc);
    out[1] = -(A * B * da + (A * C + B * B) * db + B * C * dc);
    out[2] = -(B * B * da + 2.0f * B * C * db + C * C * dc);
  };
  // w.r.t. camera-space t, then mu
  float dabc_t[3][3];
#pragma unroll
  for (int n = 0; n < 3; ++n) {
    float dT0[3], dT1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dT0[i] = dj00[n] * R[i] + dj02[n] * R[6 + i];
      dT1[i] = dj11[n] * R[3 + i] + dj12[n] * R[6 + i];
    }
    const float da = 2.0f * (dT0[0] * ST0[0] + dT0[1] * ST0[1] + dT0[2] * ST0[2]);
    const float db = dT0[0] * ST1[0] + dT0[1] * ST1[1] + dT0[2] * ST1[2] +
                     dT1[0] * ST0[0] + dT1[1] * ST0[1] + dT1[2] * ST0[2];
    const float dc = 2.0f * (dT1[0] * ST1[0] + dT1[1] * ST1[1] + dT1[2] * ST1[2]);
    dconic(da, db, dc, dabc_t[n]);
  }
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int e = 0; e < 3; ++e)
      J.Jc[e][m] = dabc_t[0][e] * R[m] + dabc_t[1][e] * R[3 + m] + dabc_t[2][e] * R[6 + m];
  // w.r.t. log-scales: dSigma3 = 2 s_k^2 r_k r_k^T
  float u0[3], u1[3];   // T0 . r_k, T1 . r_k
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    u0[k] = T0[0] * Rq[k] + T0[1] * Rq[3 + k] + T0[2] * Rq[6 + k];
    u1[k] = T1[0] * Rq[k] + T1[1] * Rq[3 + k] + T1[2] * Rq[6 + k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float o[3];
    dconic(2.0f * s2[k] * u0[k] * u0[k], 2.0f * s2[k] * u0[k] * u1[k], 2.0f * s2[k] * u1[k] * u1[k], o);
#pragma unroll
    for (int e = 0; e < 3; ++e) J.Jc[e][3 + k] = o[e];
  }
  // w.r.t. the normalised quaternion, then the raw one
  const float dR[4][9] = {
      {0.0f, -2.0f * qz, 2.0f * qy, 2.0f * qz, 0.0f, -2.0f * qx, -2.0f * qy, 2.0f * qx, 0.0f},
      {0.0f, 2.0f * qy, 2.0f * qz, 2.0f * qy, -4.0f * qx, -2.0f * qw, 2.0f * qz, 2.0f * qw, -4.0f * qx},
      {-4.0f * qy, 2.0f * qx, 2.0f * qw, 2.0f * qx, 0.0f, 2.0f * qz, -2.0f * qw, 2.0f * qz, -4.0f * qy},
      {-4.0f * qz, -2.0f * qw, 2.0f * qx, 2.0f * qw, -4.0f * qz, 2.0f * qy, 2.0f * qx, 2.0f * qy, 0.0f}};
  float dq_hat[4][3];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float v0[3], v1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v0[k] = T0[0] * dR[e][k] + T0[1] * dR[e][3 + k] + T0[2] * dR[e][6 + k];
      v1[k] = T1[0] * dR[e][k] + T1[1] * dR[e][3 + k] + T1[2] * dR[e][6 + k];
    }
    float da = 0.0f, db = 0.0f, dc = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      da += 2.0f * v0[k] * s2[k] * u0[k];
      db += s2[k] * (v0[k] * u1[k] + u0[k] * v1[k]);
      dc += 2.0f * v1[k] * s2[k] * u1[k];
    }
    dconic(da, db, dc, dq_hat[e]);
  }
  const float qh[4] = {qw, qx, qy, qz};
  const float inv_n = 1.0f / ax.z;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int e3 = 0; e3 < 3; ++e3) {
      float acc = 0.0f;
#pragma unroll
      for (int e = 0; e < 4; ++e) acc += ((e == i ? 1.0f : 0.0f) - qh[e] * qh[i]) * inv_n * dq_hat[e][e3];
      J.Jc[e3][6 + i] = acc;
    }
  J.dsig = ms.w * (1.0f - ms.w);
  // colour: SH at the view direction, d rgb / d mu through the direction
  float dv[3] = {mu[0] - cam.campos[0], mu[1] - cam.campos[1], mu[2] - cam.campos[2]};
  const float il = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const float d[3] = {dv[0] * il, dv[1] * il, dv[2] * il};
  float G[16][3];
  sh_val_grad(deg, d[0], d[1], d[2], J.Y, G);
  const float* shg = s.sh + (size_t)g * nb * 3;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float val = 0.5f, gr[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < nb; ++k) {
      const float co = shg[3 * k + ch];
      val += J.Y[k] * co;
      gr[0] += G[k][0] * co; gr[1] += G[k][1] * co; gr[2] += G[k][2] * co;
    }
    J.live[ch] = val < 0.0f ? 0.0f : 1.0f;
    const float gd = gr[0] * d[0] + gr[1] * d[1] + gr[2] * d[2];
#pragma unroll
    for (int m = 0; m < 3; ++m) J.Jrgb[ch][m] = J.live[ch] * (gr[m] - gd * d[m]) * il;
  }
}

__device__ void compute_gjac(const DevScene& s, const Consts& c, const DevCam& cam, int64_t g, GJac& J) {
  compute_gjac_t<-1>(s, c, cam, g, J);
}

__host__ __device__ __forceinline__ int out_l(int f, const Consts& c) {
  return f == 0 ? kNG + 3 * c.nb : (f == 1 ? kNG : kNG + c.KC);
}
__host__ __device__ __forceinline__ int out_u(int f, const Consts& c) {
  return f == 0 ? 9 : (f == 1 ? 7 : 6 + c.K);
}

// Dense B (u x u) of output f from the structured block.
__device__ __forceinline__ void build_B(int f, const float* blk, const Consts& c, float* Bm, int lane) {
  const int u = out_u(f, c);
  const int qoff = f == 0 ? kOffQrgb : (f == 1 ? kOffQd : kOffQo);
  const float W2 = blk[kOffW2];
  for (int i = lane; i < u * u; i += 32) {
    const int r = i / u, cc = i - r * u;
    float v;
    if (r < 6 && cc < 6) v = r >= cc ? blk[qoff + tri(r, cc)] : blk[qoff + tri(cc, r)];
    else if (r >= 6 && cc >= 6) {
      if (f == 2) v = W2 * ((r == cc ? 1.0f : 0.0f) + 1.0f);
      else v = r == cc ? W2 : 0.0f;
    } else {
      const int big = r >= 6 ? r : cc, small = r >= 6 ? cc : r;
      const int xo = f == 0 ? kOffXrgb : (f == 1 ? kOffXd : kOffXo);
      v = blk[xo + 6 * (big - 6) + small];
    }
    Bm[i] = v;
  }
  __syncwarp();
}

// --------------------------------------------------------- training factors
// Decode the linear index t of a packed lower triangle into (row, col): a
// table lookup (row << 16 | col) for every triangle of up to kTriRows rows
// (all the factors: l <= 11 + 128), computed beyond.
constexpr int kTriRows = 140;
constexpr int kTriMax = kTriRows * (kTriRows + 1) / 2;
__device__ uint32_t g_tri[kTriMax];

__global__ void k_tri_init() {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kTriMax) return;
  int r = 0;
  while (tri(r + 1, 0) <= t) ++r;      // 140 steps at most, once per library context
  g_tri[t] = ((uint32_t)r << 16) | (uint32_t)(t - tri(r, 0));
}

__device__ __forceinline__ void tri_decode(int t, int& r, int& cc) {
  if (t < kTriMax) {
    const uint32_t v = __ldg(&g_tri[t]);
    r = (int)(v >> 16);
    cc = (int)(v & 0xFFFFu);
    return;
  }
  r = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (tri(r + 1, 0) <= t) ++r;
  while (tri(r, 0) > t) --r;
  cc = t - tri(r, 0);
}

// Entries of the projection Jacobian M (u x 11) on the geometric parameters
// (mean, log-scale, quaternion, opacity logit), by row:
// rows 0-1 mean2D, 2-4 conic, 5 sigma (shared by the three outputs).
__device__ __forceinline__ float m_geo(const GJac& J, int v, int a) {
  if (v < 2) return a < 3 ? J.Jm[v][a] : 0.0f;
  if (v < 5) return a < 10 ? J.Jc[v - 2][a] : 0.0f;
  return a == 10 ? J.dsig : 0.0f;
}
// Entry (u, v) of a 6 x 6 block stored packed lower.
__device__ __forceinline__ float q6(const float* q, int u, int v) { return u >= v ? q[tri(u, v)] : q[tri(v, u)]; }

// The colour sums H0 are stored by blocks, without the SH entries of
// different channels (always zero): geometric x geometric (packed 11-triangle,
// 66), SH (k, ch) x geometric b at 66 + (3 k + ch) 11 + b, and SH x SH of one
// channel at 66 + 33 nb + ch T + tri(k, k2), T = nb (nb + 1) / 2.
__host__ __device__ __forceinline__ int h0_sg(int ish, int b) { return kNG * (kNG + 1) / 2 + ish * kNG + b; }
__host__ __device__ __forceinline__ int h0_ss(int nb, int ch, int k, int k2) {
  return kNG * (kNG + 1) / 2 + kNG * 3 * nb + ch * (nb * (nb + 1) / 2) + tri(k, k2);
}

// Per-warp shared memory of the factor kernel: doubles (the scaled matrix
// being factorised and the scaling), then floats.
struct FactLayout {
  int l0, l1, l2, nt0, nt1, nt2;
  int off_A, off_X, off_R, d_per_warp;     // doubles: scaling and floors (2 (l0 + l1 + l2)), then these
  int off_H1, off_H2, off_J, off_GB, off_XG, off_xs, off_E, off_T, off_col, f_per_warp;
};
constexpr int kTrainChunk = 8;   // training views whose Jacobians are held at once

FactLayout fact_layout(const Consts& c) {
  FactLayout y{};
  y.l0 = kNG + 3 * c.nb;
  y.l1 = kNG;
  y.l2 = kNG + c.KC;
  y.nt0 = rgb_L_size(c.nb);       // the structured colour sums (same count as the stored factor)
  y.nt1 = y.l1 * (y.l1 + 1) / 2;
  y.nt2 = y.l2 * (y.l2 + 1) / 2;
  const int T = c.nb * (c.nb + 1) / 2, n3 = 3 * c.nb;
  auto mx = [](int a, int b) { return a > b ? a : b; };
  y.off_A = 2 * (y.l0 + y.l1 + y.l2);
  y.off_X = y.off_A + 3 * T;
  y.off_R = y.off_X + mx(3 * T, kNG * (n3 + 1));      // coupling rows padded to an odd stride
  y.d_per_warp = y.off_R + mx(kNG * (n3 + 1) + kNG * (kNG + 1), y.nt2);
  auto r4 = [](int x) { return (x + 3) & ~3; };
  y.off_H1 = r4(y.nt0);
  y.off_H2 = y.off_H1 + r4(y.nt1);
  y.off_J = y.off_H2 + r4(y.nt2);
  y.off_GB = y.off_J + r4(kTrainChunk * (int)(sizeof(GJac) / 4));
  y.off_XG = y.off_GB + 9 * kNG + 1;
  y.off_xs = y.off_XG + r4(c.K * kNG);
  y.off_E = y.off_xs + 12;
  // T_c (11 x 3 nb) lives only inside the factorisation, after the Jacobians
  // and block scratch of the accumulation are done with: it takes their
  // space when it fits (one more warp per block at SH degree 3)
  const int tsz = r4(kNG * 3 * c.nb);
  int end = y.off_E + 68;
  if (tsz <= y.off_xs - y.off_J) {
    y.off_T = y.off_J;
  } else {
    y.off_T = end;
    end += tsz;
  }
  y.off_col = end;
  y.f_per_warp = y.off_col + r4(mx(y.l2, 2 * kNG));
  return y;
}

// Adds one training view's blocks A = M^T B M of the three outputs to the
// warp's sums H0 (colour), H1 (depth), H2 (object; geometric-geometric
// part, plus XG += X_o G for the logit rows, finished per Gaussian), using
// the block structure of M: geometric rows (mean2D, conic, sigma) over the
// 11 geometric parameters; colour rows over the mean (view direction) and,
// channel by channel, over the SH coefficients (live_ch Y_k); the depth row
// over the mean; the probability rows over the object logits only (view
// independent).
__device__ __forceinline__ void add_view_blocks(const GJac& J, const float* __restrict__ blk, const Consts& c,
                                                float* H0, float* H1, float* H2, float* GB, float* XG,
                                                int lane) {
  const float W2 = blk[kOffW2];
  const int nb = c.nb, K = c.K;
  // colour: GB = B_rgb M (9 x 11)
  for (int e = lane; e < 9 * kNG; e += 32) {
    const int u = e / kNG, a = e - kNG * u;
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const float buv = u < 6 ? q6(blk + kOffQrgb, u, v) : blk[kOffXrgb + 6 * (u - 6) + v];
      acc += buv * m_geo(J, v, a);
    }
    if (a < 3) {
#pragma unroll
      for (int v = 6; v < 9; ++v) {
        const float buv = u < 6 ? blk[kOffXrgb + 6 * (v - 6) + u] : (u == v ? W2 : 0.0f);
        acc += buv * J.Jrgb[v - 6][a];
      }
    }
    GB[e] = acc;
  }
  __syncwarp();
  for (int e = lane; e < kNG * (kNG + 1) / 2; e += 32) {   // geometric x geometric
    int a, b;
    tri_decode(e, a, b);
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) acc += m_geo(J, v, a) * GB[v * kNG + b];
    if (a < 3) {
#pragma unroll
      for (int v = 6; v < 9; ++v) acc += J.Jrgb[v - 6][a] * GB[v * kNG + b];
    }
    H0[e] += acc;
  }
  for (int e = lane; e < 3 * nb * kNG; e += 32) {          // SH x geometric
    const int ish = e / kNG, b = e - kNG * ish;
    const int k = ish / 3, ch = ish - 3 * k;
    H0[h0_sg(ish, b)] += J.live[ch] * J.Y[k] * GB[(6 + ch) * kNG + b];
  }
  for (int e = lane; e < 3 * (nb * (nb + 1) / 2); e += 32) {   // SH x SH, same channel only
    const int ch = e % 3;
    int k, k2;
    tri_decode(e / 3, k, k2);
    H0[h0_ss(nb, ch, k, k2)] += W2 * J.live[ch] * J.Y[k] * J.Y[k2];
  }
  __syncwarp();
  // depth: GB = B_d M (7 x 11), H1 = M^T GB
  for (int e = lane; e < 7 * kNG; e += 32) {
    const int u = e / kNG, a = e - kNG * u;
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const float buv = u < 6 ? q6(blk + kOffQd, u, v) : blk[kOffXd + v];
      acc += buv * m_geo(J, v, a);
    }
    if (a < 3) acc += (u < 6 ? blk[kOffXd + u] : W2) * J.Jz[a];
    GB[e] = acc;
  }
  __syncwarp();
  for (int e = lane; e < kNG * (kNG + 1) / 2; e += 32) {
    int a, b;
    tri_decode(e, a, b);
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) acc += m_geo(J, v, a) * GB[v * kNG + b];
    if (a < 3) acc += J.Jz[a] * GB[6 * kNG + b];
    H1[e] += acc;
  }
  __syncwarp();
  // object, geometric part: GB = Q_o G (6 x 11), H2 += G^T GB; XG += X_o G (K x 11)
  for (int e = lane; e < 6 * kNG; e += 32) {
    const int u = e / kNG, a = e - kNG * u;
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) acc += q6(blk + kOffQo, u, v) * m_geo(J, v, a);
    GB[e] = acc;
  }
  for (int e = lane; e < K * kNG; e += 32) {
    const int j = e / kNG, a = e - kNG * j;
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) acc += blk[kOffXo + 6 * j + v] * m_geo(J, v, a);
    XG[e] += acc;
  }
  __syncwarp();
  for (int e = lane; e < kNG * (kNG + 1) / 2; e += 32) {
    int a, b;
    tri_decode(e, a, b);
    float acc = 0.0f;
#pragma unroll
    for (int v = 0; v < 6; ++v) acc += m_geo(J, v, a) * GB[v * kNG + b];
    H2[e] += acc;
  }
  __syncwarp();
}

// x^-1/2 in double precision by Newton's iteration y <- y (3 - x y^2) / 2,
// started from the single-precision estimate (two steps: about 2^-22 ->
// 2^-44 -> below double rounding). x must lie in the normal float range.
__device__ __forceinline__ double rsqrt_d(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}

// Up to four packed lower matrices that one warp factorises (or inverts)
// together: the pivots of a step are taken by lanes 0-3 at once and the
// element updates of all matrices are spread over the warp, so the serial
// chain of a step is paid once for the set. n = 0 marks an unused slot.
struct MatSet {
  double* P0;
  double* P1;
  double* P2;
  double* P3;
  const double* f0;     // pivot floors by row (see chol_set_d)
  const double* f1;
  const double* f2;
  const double* f3;
  int n0, n1, n2, n3;
};

__device__ __forceinline__ double* ms_P(const MatSet& s, int q) {
  return q == 0 ? s.P0 : (q == 1 ? s.P1 : (q == 2 ? s.P2 : s.P3));
}
__device__ __forceinline__ const double* ms_f(const MatSet& s, int q) {
  return q == 0 ? s.f0 : (q == 1 ? s.f1 : (q == 2 ? s.f2 : s.f3));
}
__device__ __forceinline__ int ms_n(const MatSet& s, int q) {
  return q == 0 ? s.n0 : (q == 1 ? s.n1 : (q == 2 ? s.n2 : s.n3));
}
__device__ __forceinline__ int ms_nmax(const MatSet& s) { return max(max(s.n0, s.n1), max(s.n2, s.n3)); }

// Which of four consecutive ranges of sizes c[0..3] the index e falls in;
// e becomes the offset inside it.
__device__ __forceinline__ int range_of(const int (&c)[4], int& e) {
  int q = 0;
  if (e >= c[0]) {
    e -= c[0];
    q = 1;
    if (e >= c[1]) {
      e -= c[1];
      q = 2;
      if (e >= c[2]) {
        e -= c[2];
        q = 3;
      }
    }
  }
  return q;
}

// Cholesky factorisation of the set in double precision, in place; the
// diagonal slot keeps 1 / L_kk (all that the inversion needs of it).
// Each matrix is a Jacobi-scaled damped Hessian D^-1/2 (lambda I + A) D^-1/2
// with A positive semi-definite, so pivot k is at least lambda / H_kk (the
// floor f[k]). Rounding in the single-precision sums of A can push a pivot
// of a nearly unobserved direction below that bound, even below zero; such a
// pivot is raised to the bound. A non-finite pivot sets *err.
__device__ void chol_set_d(const MatSet& s, int* err, int lane) {
  const int nmax = ms_nmax(s);
  for (int k = 0; k < nmax; ++k) {
    if (lane < 4 && k < ms_n(s, lane)) {
      double* P = ms_P(s, lane);
      double dkk = P[tri(k, k)];
      if (!isfinite(dkk)) atomicExch(err, 1);
      const double fk = ms_f(s, lane)[k];
      if (!(dkk >= fk)) dkk = fk;
      P[tri(k, k)] = rsqrt_d(fmax(dkk, 1e-30));
    }
    __syncwarp();
    int cs[4], ct[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = max(ms_n(s, q) - k - 1, 0);
      cs[q] = r;
      ct[q] = r * (r + 1) / 2;
    }
    const int ns = cs[0] + cs[1] + cs[2] + cs[3];
    for (int e0 = lane; e0 < ns; e0 += 32) {        // column k below the pivot
      int e = e0;
      const int q = range_of(cs, e);
      double* P = ms_P(s, q);
      P[tri(k + 1 + e, k)] *= P[tri(k, k)];
    }
    __syncwarp();
    const int nt = ct[0] + ct[1] + ct[2] + ct[3];
    for (int e0 = lane; e0 < nt; e0 += 32) {        // trailing triangles
      int e = e0;
      const int q = range_of(ct, e);
      double* P = ms_P(s, q);
      int ii, jj;
      tri_decode(e, ii, jj);
      const int i = k + 1 + ii, j = k + 1 + jj;
      P[tri(i, j)] -= P[tri(i, k)] * P[tri(j, k)];
    }
    __syncwarp();
  }
}

// X_q = L_q^-1 (packed lower) for the factors chol_set_d left, right-looking:
//   X_kk = 1 / L_kk,  X_kj = -X_kk acc_kj (j < k),  acc_ij += L_ik X_kj (i > k, j <= k).
// For single-precision X the column L_.k is converted once per step into
// col (sum of the set's n floats).
template <typename TX>
__device__ void inv_set(const MatSet& s, TX* X0, TX* X1, TX* X2, TX* X3, float* col, int lane) {
  const int nn[4] = {s.n0, s.n1, s.n2, s.n3};
  int tt[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) tt[q] = nn[q] * (nn[q] + 1) / 2;
  auto Xq = [&](int q) { return q == 0 ? X0 : (q == 1 ? X1 : (q == 2 ? X2 : X3)); };
  const int ntot = tt[0] + tt[1] + tt[2] + tt[3];
  for (int e0 = lane; e0 < ntot; e0 += 32) {
    int e = e0;
    const int q = range_of(tt, e);
    Xq(q)[e] = (TX)0;
  }
  auto cb = [&](int q) {                      // offset of matrix q's column in col
    return q == 0 ? 0 : (q == 1 ? nn[0] : (q == 2 ? nn[0] + nn[1] : nn[0] + nn[1] + nn[2]));
  };
  __syncwarp();
  const int nmax = ms_nmax(s);
  for (int k = 0; k < nmax; ++k) {
    int ca[4], cc[4], cu[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool live = k < nn[q];
      ca[q] = live ? k + 1 : 0;                 // row k of X
      cc[q] = live ? nn[q] - k - 1 : 0;         // column k of L below the diagonal
      cu[q] = cc[q] * (k + 1);                  // updates of the rows below
    }
    const int na = ca[0] + ca[1] + ca[2] + ca[3];
    const int nc = std::is_same<TX, float>::value ? cc[0] + cc[1] + cc[2] + cc[3] : 0;
    for (int e0 = lane; e0 < na + nc; e0 += 32) {
      if (e0 < na) {
        int e = e0;
        const int q = range_of(ca, e);
        const TX xkk = (TX)ms_P(s, q)[tri(k, k)];
        TX* X = Xq(q);
        X[tri(k, e)] = e == k ? xkk : -xkk * X[tri(k, e)];
      } else {
        int e = e0 - na;
        const int q = range_of(cc, e);
        col[cb(q) + k + 1 + e] = (float)ms_P(s, q)[tri(k + 1 + e, k)];
      }
    }
    __syncwarp();
    const int nu = cu[0] + cu[1] + cu[2] + cu[3];
    // e / (k + 1) as floor((e + 1/2) / (k + 1)) in single precision: exact for
    // e < 2^13, k < 140 (the error is below 2^-10, the distance to the next
    // integer at least 1 / 280)
    const float rk = 1.0f / (float)(k + 1);
    for (int e0 = lane; e0 < nu; e0 += 32) {
      int e = e0;
      const int q = range_of(cu, e);
      const int i = k + 1 + (int)(((float)e + 0.5f) * rk), j = e - (i - k - 1) * (k + 1);
      TX* X = Xq(q);
      TX lik;
      if constexpr (std::is_same<TX, float>::value) lik = col[cb(q) + i];
      else lik = ms_P(s, q)[tri(i, k)];
      X[tri(i, j)] += lik * X[tri(k, j)];
    }
    __syncwarp();
  }
}

// All three outputs' training factors of one Gaussian, stored in the forms
// Factors describes. H0, H1, H2: the sums sum_t A_t of colour (by blocks,
// see h0_sg / h0_ss; SH (k, ch) is parameter 11 + 3 k + ch), depth and
// object (packed; floats; H2 and H1 are reused as outputs, H0 as scratch
// once read). Each H = lambda I + c_g H_sum
// is Jacobi-scaled, H~ = D^-1/2 H D^-1/2, and Cholesky-factorised in double
// precision. Colour goes by blocks with the parameters ordered [SH of
// channel 0, 1, 2 | geometric]: the three SH blocks are independent, so H~ =
// L L^T needs their factors L_c, the coupling L_gS = H~_gS L_S^-T and the
// factor of the geometric Schur complement H~_gg - L_gS L_gS^T. Order of
// work: the SH blocks and the object matrix together, then the Schur
// complement and the depth matrix together.
__device__ void factorise_all(const FactLayout& y, float cg, const Consts& c, float* H0, float* H1, float* H2,
                              double* D, float* fb, float* L0g, float* L1g, float* L2g, int* err, int lane) {
  const int nb = c.nb, T = nb * (nb + 1) / 2, n3 = 3 * nb, l0 = y.l0, l2 = y.l2, nt2 = y.nt2;
  const int n3p = n3 + 1;   // row stride of H~_gS and L_gS: odd, so rows fall in distinct banks
  const int nd = l0 + kNG + l2;
  const double lam = c.lam, cgd = cg;
  double* dsc0 = D;                  // D^-1/2 of colour (natural order), depth, object
  double* dsc1 = D + l0;
  double* dsc2 = dsc1 + kNG;
  double* flX = D + nd;              // pivot floors lambda / H_kk: SH blocks [ch][k],
  double* flS = flX + n3;            // Schur complement, depth, object
  double* fl1 = flS + kNG;
  double* fl2 = fl1 + kNG;
  double* A = D + y.off_A;           // A_c = L_c^-1 (3 packed nb-triangles)
  double* X = D + y.off_X;           // SH blocks being factorised; then H~_gS rows
  double* R = D + y.off_R;           // object matrix; then L_gS, Schur complement, depth
  float* Ef = fb + y.off_E;
  float* Tf = fb + y.off_T;
  float* col = fb + y.off_col;
  for (int i = lane; i < nd; i += 32) {
    float h;
    int fi;
    if (i < l0) {                 // colour: geometric r -> Schur floors, SH (k, ch) -> [ch][k]
      h = i < kNG ? H0[tri(i, i)] : H0[h0_ss(nb, (i - kNG) % 3, (i - kNG) / 3, (i - kNG) / 3)];
      fi = i < kNG ? n3 + i : ((i - kNG) % 3) * nb + (i - kNG) / 3;
    } else {                      // depth and object rows keep their index (l0 = n3 + 11)
      const int r = i < l0 + kNG ? i - l0 : i - l0 - kNG;
      h = (i < l0 + kNG ? H1 : H2)[tri(r, r)];
      fi = i;
    }
    const double d = rsqrt_d(lam + cgd * (double)h);
    D[i] = d;
    flX[fi] = lam * d * d;
  }
  __syncwarp();
  for (int e = lane; e < 3 * T; e += 32) {
    const int ch = e / T;
    int k, k2;
    tri_decode(e - ch * T, k, k2);
    const int a = kNG + 3 * k + ch, b = kNG + 3 * k2 + ch;
    X[e] = (cgd * (double)H0[h0_ss(nb, ch, k, k2)] + (k == k2 ? lam : 0.0)) * dsc0[a] * dsc0[b];
  }
  for (int e = lane; e < nt2; e += 32) {
    int r, r2;
    tri_decode(e, r, r2);
    R[e] = (cgd * (double)H2[e] + (r == r2 ? lam : 0.0)) * dsc2[r] * dsc2[r2];
  }
  __syncwarp();
  chol_set_d(MatSet{X, X + T, X + 2 * T, R, flX, flX + nb, flX + 2 * nb, fl2, nb, nb, nb, l2}, err, lane);
  inv_set<double>(MatSet{X, X + T, X + 2 * T, nullptr, nullptr, nullptr, nullptr, nullptr, nb, nb, nb, 0},
                  A, A + T, A + 2 * T, (double*)nullptr, col, lane);
  inv_set<float>(MatSet{R, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, l2, 0, 0, 0},
                 H2, (float*)nullptr, (float*)nullptr, (float*)nullptr, col, lane);
  for (int e = lane; e < nt2; e += 32) {             // object: L~ = L^-1 D^-1/2
    int r, r2;
    tri_decode(e, r, r2);
    L2g[e] = (float)((double)H2[e] * dsc2[r2]);
  }
  // colour coupling: H~_gS rows, X[r][ch nb + k2] = H(b, r) D^-1/2_b, b = 11 + 3 k2 + ch
  for (int e = lane; e < kNG * n3; e += 32) {
    const int r = e / n3, q = e - r * n3, ch = q / nb, k2 = q - ch * nb;
    const int b = kNG + 3 * k2 + ch;
    X[r * n3p + q] = (double)H0[h0_sg(3 * k2 + ch, r)] * dsc0[b];
  }
  __syncwarp();
  // L_gS[r][ch nb + k] = c_g D^-1/2_r sum_{k2 <= k} X[r][ch nb + k2] A_c[k][k2]; each
  // lane takes k and nb - 1 - k (nb + 1 terms in all, the same count on every lane)
  double* LgS = R;
  double* S = R + kNG * n3p;
  double* S1 = S + kNG * (kNG + 1) / 2;
  const int hp = (nb + 1) / 2;
  for (int task = lane; task < kNG * 3 * hp; task += 32) {
    const int r = task / (3 * hp), rem = task - r * 3 * hp, ch = rem / hp, p = rem - ch * hp;
    const int k1 = p, k2 = nb - 1 - p;
    const double* hrow = X + r * n3p + ch * nb;
    const double* Ac = A + ch * T;
    double acc = 0.0, acc1 = 0.0;
    for (int it = 0; it <= nb; ++it) {
      if (it == k1 + 1) {
        acc1 = acc;
        acc = 0.0;
      }
      const bool first = it <= k1;
      const int q = first ? it : it - k1 - 1;
      acc = fma(hrow[q], Ac[tri(first ? k1 : k2, q)], acc);
    }
    const double sc = cgd * dsc0[r];
    LgS[r * n3p + ch * nb + k1] = sc * acc1;
    LgS[r * n3p + ch * nb + k2] = sc * acc;
  }
  __syncwarp();
  for (int e = lane; e < kNG * (kNG + 1) / 2; e += 32) {   // H~_gg - L_gS L_gS^T
    int r, r2;
    tri_decode(e, r, r2);
    double acc = (cgd * (double)H0[e] + (r == r2 ? lam : 0.0)) * dsc0[r] * dsc0[r2];
    for (int q = 0; q < n3; ++q) acc -= LgS[r * n3p + q] * LgS[r2 * n3p + q];
    S[e] = acc;
  }
  for (int e = lane; e < kNG * (kNG + 1) / 2; e += 32) {   // depth
    int r, r2;
    tri_decode(e, r, r2);
    S1[e] = (cgd * (double)H1[e] + (r == r2 ? lam : 0.0)) * dsc1[r] * dsc1[r2];
  }
  __syncwarp();
  // the Schur complement is >= lambda D_g^-1 too, so its floors are those of the geometric rows
  chol_set_d(MatSet{S, S1, nullptr, nullptr, flS, fl1, nullptr, nullptr, kNG, kNG, 0, 0}, err, lane);
  inv_set<float>(MatSet{S, S1, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, kNG, kNG, 0, 0}, Ef, H1,
                 (float*)nullptr, (float*)nullptr, col, lane);
  // single-precision copies of A_c and L_gS (H0 is no longer read)
  float* Af = H0;
  float* LgSf = H0 + 3 * T;
  for (int e = lane; e < 3 * T + kNG * n3p; e += 32) Af[e] = (float)(e < 3 * T ? A[e] : LgS[e - 3 * T]);
  __syncwarp();
  for (int e = lane; e < kNG * n3; e += 32) {          // T_c = L_gS,c A_c
    const int r = e / n3, q = e - r * n3, ch = q / nb, k = q - ch * nb;
    float acc = 0.0f;
    for (int k2 = k; k2 < nb; ++k2) acc += LgSf[r * n3p + ch * nb + k2] * Af[ch * T + tri(k2, k)];
    Tf[e] = acc;
  }
  __syncwarp();
  for (int e = lane; e < 3 * T; e += 32) {
    const int ch = e / T;
    int k, k2;
    tri_decode(e - ch * T, k, k2);
    L0g[e] = (float)(A[e] * dsc0[kNG + 3 * k2 + ch]);
  }
  float* Lc = L0g + rgb_off_C(nb);
  for (int e = lane; e < kNG * n3; e += 32) {
    const int r = e / n3, q = e - r * n3, ch = q / nb, k = q - ch * nb;
    float acc = 0.0f;
    for (int r2 = 0; r2 <= r; ++r2) acc += Ef[tri(r, r2)] * Tf[r2 * n3 + q];
    Lc[e] = (float)(-(double)acc * dsc0[kNG + 3 * k + ch]);
  }
  float* Le = L0g + rgb_off_E(nb);
  for (int e = lane; e < kNG * (kNG + 1) / 2; e += 32) {
    int r, r2;
    tri_decode(e, r, r2);
    Le[e] = (float)((double)Ef[e] * dsc0[r2]);
    L1g[e] = (float)((double)H1[e] * dsc1[r2]);
  }
  __syncwarp();
}

// One warp per Gaussian: the projection Jacobians of up to 8 training views
// at once (one lane each), the structured sums of the three outputs' blocks
// over the training views, then each output's training Hessian
// H = lambda I + c_g sum_t M_t^T B_t M_t factorised (Eqs. 6, 9; C_g = c_g I).
__global__ void k_build_factors(DevScene s, Consts c, const DevCam* __restrict__ cams,
                                const float* __restrict__ blocks, int n_train, Factors F, int* err,
                                FactLayout y) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nBp = (block_floats(c.K) + 3) & ~3;
  double* Dw = reinterpret_cast<double*>(smem) + (size_t)warp * y.d_per_warp;
  float* fb = reinterpret_cast<float*>(reinterpret_cast<double*>(smem) + (size_t)nw * y.d_per_warp) +
              (size_t)warp * y.f_per_warp;
  float* H0 = fb;
  float* H1 = fb + y.off_H1;
  float* H2 = fb + y.off_H2;
  GJac* Jw = reinterpret_cast<GJac*>(fb + y.off_J);
  float* GB = fb + y.off_GB;
  float* XG = fb + y.off_XG;
  float* xs = fb + y.off_xs;
  const int K = c.K, KC = c.KC;
  for (int64_t sl = (int64_t)blockIdx.x * nw + warp; sl < s.n_act; sl += (int64_t)gridDim.x * nw) {
    const int64_t g = s.act[sl];          // training blocks and factors are stored by active slot
    const float cg = s.aux[g].y;
    const float* p = s.p + (size_t)g * KC;
    for (int i = lane; i < y.nt0; i += 32) H0[i] = 0.0f;
    for (int i = lane; i < y.nt1; i += 32) H1[i] = 0.0f;
    for (int i = lane; i < y.nt2; i += 32) H2[i] = 0.0f;
    for (int i = lane; i < K * kNG; i += 32) XG[i] = 0.0f;
    float w2sum = 0.0f;
    __syncwarp();
    if (cg > 0.0f) {
      for (int t0 = 0; t0 < n_train; t0 += kTrainChunk) {
        const int t = t0 + lane;
        bool seen = false;
        if (lane < kTrainChunk && t < n_train) {
          seen = blocks[((size_t)t * s.n_act + sl) * nBp + kOffW2] != 0.0f;
          if (seen) compute_gjac(s, c, cams[t], g, Jw[lane]);
        }
        unsigned todo = __ballot_sync(0xffffffffu, seen);
        __syncwarp();
        while (todo) {
          const int src = __ffs(todo) - 1;
          todo &= todo - 1;
          const float* blk = blocks + ((size_t)(t0 + src) * s.n_act + sl) * nBp;
          w2sum += blk[kOffW2];
          add_view_blocks(Jw[src], blk, c, H0, H1, H2, GB, XG, lane);
        }
      }
      // object logit rows: d p_j / d o_b = p_j (delta_jb - p_b) (view independent),
      // B_pp = W2 (I + 1 1^T):
      //   A[o_b][geo a] = sum_j P_jb XG[j][a] = p_b (XG[b][a] [b >= 1] - sum_j p_j XG[j][a])
      //   A[o_b][o_b'] = sum_t W2_t (P^T P + cs cs^T)[b][b'],  cs_b = p_b ([b >= 1] - (1 - p_0))
      for (int a = lane; a < kNG; a += 32) {
        float acc = 0.0f;
        for (int j = 1; j <= K; ++j) acc += p[j] * XG[(j - 1) * kNG + a];
        xs[a] = acc;
      }
      __syncwarp();
      for (int e = lane; e < KC * kNG; e += 32) {
        const int b = e / kNG, a = e - kNG * b;
        const float xb = b >= 1 ? XG[(b - 1) * kNG + a] : 0.0f;
        H2[tri(kNG + b, a)] += p[b] * (xb - xs[a]);
      }
      float s2 = 0.0f;
      for (int j = 1; j <= K; ++j) s2 += p[j] * p[j];
      const float one_m_p0 = 1.0f - p[0];
      for (int e = lane; e < KC * (KC + 1) / 2; e += 32) {
        int b, b2;
        tri_decode(e, b, b2);
        const float pb = p[b], pb2 = p[b2];
        float pp = pb * pb2 * s2;
        if (b >= 1) pp -= pb * pb * pb2;
        if (b2 >= 1) pp -= pb2 * pb2 * pb;
        if (b == b2 && b >= 1) pp += pb * pb;
        const float csb = pb * ((b >= 1 ? 1.0f : 0.0f) - one_m_p0);
        const float csb2 = pb2 * ((b2 >= 1 ? 1.0f : 0.0f) - one_m_p0);
        H2[tri(kNG + b, kNG + b2)] += w2sum * (pp + csb * csb2);
      }
      __syncwarp();
    }
    if (c.crit == 2) {
      // T-optimality has no training prior: the gains read L~ = I
      float* L0g = F.L[0] + (size_t)sl * rgb_L_size(c.nb);
      const int T = rgb_tri_nb(c.nb);
      for (int i = lane; i < rgb_L_size(c.nb); i += 32) {
        float v = 0.0f;
        if (i < 3 * T) {
          int k, k2;
          tri_decode(i % T, k, k2);
          v = k == k2 ? 1.0f : 0.0f;
        } else if (i >= rgb_off_E(c.nb)) {
          int r, r2;
          tri_decode(i - rgb_off_E(c.nb), r, r2);
          v = r == r2 ? 1.0f : 0.0f;
        }
        L0g[i] = v;
      }
      for (int f = 1; f < 3; ++f) {
        const int nt = f == 1 ? y.nt1 : y.nt2;
        float* Lg = F.L[f] + (size_t)sl * nt;
        for (int i = lane; i < nt; i += 32) {
          int r, r2;
          tri_decode(i, r, r2);
          Lg[i] = r == r2 ? 1.0f : 0.0f;
        }
      }
      __syncwarp();
      continue;
    }
    factorise_all(y, cg, c, H0, H1, H2, Dw, fb, F.L[0] + (size_t)sl * rgb_L_size(c.nb), F.L[1] + (size_t)sl * y.nt1,
                  F.L[2] + (size_t)sl * y.nt2, err, lane);
  }
}

// -------------------------------------------------------------- view gains
// Y = M^T of output f (l x u, row-major), built by the warp.
__device__ void build_Y(int f, const GJac& J, const Consts& c, const float* p, float* Y, int lane) {
  const int l = out_l(f, c), u = out_u(f, c);
  for (int i = lane; i < u * l; i += 32) Y[i] = 0.0f;
  __syncwarp();
  if (lane == 0) {
    for (int m = 0; m < 3; ++m) {
      Y[m * u + 0] = J.Jm[0][m];
      Y[m * u + 1] = J.Jm[1][m];
    }
    for (int e = 0; e < 3; ++e)
      for (int k = 0; k < 10; ++k) Y[k * u + 2 + e] = J.Jc[e][k];
    Y[10 * u + 5] = J.dsig;
    if (f == 0) {
      for (int ch = 0; ch < 3; ++ch)
        for (int m = 0; m < 3; ++m) Y[m * u + 6 + ch] = J.Jrgb[ch][m];
    } else if (f == 1) {
      for (int m = 0; m < 3; ++m) Y[m * u + 6] = J.Jz[m];
    }
  }
  if (f == 0) {
    for (int i = lane; i < 3 * c.nb; i += 32) {
      const int k = i / 3, ch = i - 3 * k;
      Y[(kNG + i) * u + 6 + ch] = J.live[ch] * J.Y[k];
    }
  } else if (f == 2) {
    for (int i = lane; i < c.K * c.KC; i += 32) {   // d p_j / d o_b = p_j (delta_jb - p_b)
      const int j = 1 + i / c.KC, bb = i % c.KC;
      Y[(kNG + bb) * u + 5 + j] = p[j] * ((j == bb ? 1.0f : 0.0f) - p[bb]);
    }
  }
  __syncwarp();
}

// Row i of Z = L~ Y for output f with U columns (compile time), using the
// block sparsity of Y. Ls is L~ (packed lower triangle).
template <int F, int U>
__device__ __forceinline__ void z_row(int i, int u, const float* __restrict__ Ls, const float* Y, float* Z) {
  float acc[U];
#pragma unroll
  for (int cc = 0; cc < U; ++cc) acc[cc] = 0.0f;
  const float* __restrict__ Li = Ls + tri(i, 0);
  const int kg = i < kNG - 1 ? i : kNG - 1;
  for (int k = 0; k <= kg; ++k) {               // geometric rows: dense
    const float lk = Li[k];
    const float* y = Y + k * u;
#pragma unroll
    for (int cc = 0; cc < U; ++cc)
      if (cc < u) acc[cc] += lk * y[cc];
  }
  if (F == 0) {                                  // SH rows: one colour column each
    for (int k = kNG; k <= i; k += 3) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch)
        if (k + ch <= i) acc[6 + ch] += Li[k + ch] * Y[(k + ch) * u + 6 + ch];
    }
  } else if (F == 2) {                           // object-logit rows: probability columns
    for (int k = kNG; k <= i; ++k) {
      const float lk = Li[k];
      const float* y = Y + k * u;
#pragma unroll
      for (int cc = 6; cc < U; ++cc)
        if (cc < u) acc[cc] += lk * y[cc];
    }
  }
#pragma unroll
  for (int cc = 0; cc < U; ++cc)
    if (cc < u) Z[i * u + cc] = acc[cc];
}

// log det(I + c W B) for one output; W, B, G are u x u in shared memory.
__device__ __forceinline__ float logdet_IcWB(int u, float cg, const float* W, const float* Bm, float* G, int lane,
                                             int crit = 0) {
  if (crit != 0) {   // trace criteria: c tr(W B)
    float t = 0.0f;
    for (int i = lane; i < u * u; i += 32) {
      const int r = i / u, cc = i - r * u;
      t += W[r * u + cc] * Bm[cc * u + r];
    }
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return cg * t;
  }
  for (int i = lane; i < u * u; i += 32) {
    const int r = i / u, cc = i - r * u;
    float a = 0.0f;
    for (int k = 0; k < u; ++k) a += W[r * u + k] * Bm[k * u + cc];
    G[i] = (r == cc ? 1.0f : 0.0f) + cg * a;
  }
  __syncwarp();
  float ld = 0.0f;
  for (int k = 0; k < u; ++k) {
    float best = -1.0f;
    int bi = k;
    for (int i = k + lane; i < u; i += 32) {
      const float v = fabsf(G[i * u + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o >= 1; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (bi != k) {
      for (int j = lane; j < u; j += 32) {
        const float tmp = G[k * u + j];
        G[k * u + j] = G[bi * u + j];
        G[bi * u + j] = tmp;
      }
    }
    __syncwarp();
    const float piv = G[k * u + k];
    ld += logf(fabsf(piv));
    const float ip = 1.0f / piv;
    for (int i = k + 1 + lane; i < u; i += 32) {
      const float fct = G[i * u + k] * ip;
      for (int j = k + 1; j < u; ++j) G[i * u + j] -= fct * G[k * u + j];
    }
    __syncwarp();
  }
  return ld;
}

// Z = L~ M^T of the colour output (rows in the factor's order: SH of
// channel 0, 1, 2, then geometric; 9 columns), from the block form of L~
// (see Factors): an SH row of channel ch has one nonzero, in column 6 + ch.
__device__ __forceinline__ void z_geo_rgb_row(const GJac& J, const float* Er, const float* Cr, int r, int nb,
                                              float (&z)[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) z[q] = 0.0f;
  for (int k = 0; k <= r; ++k) {
    const float lk = Er[k];
    if (k < 3) {
      z[0] += lk * J.Jm[0][k];
      z[1] += lk * J.Jm[1][k];
      z[6] += lk * J.Jrgb[0][k];
      z[7] += lk * J.Jrgb[1][k];
      z[8] += lk * J.Jrgb[2][k];
    }
    if (k < 10) {
      z[2] += lk * J.Jc[0][k];
      z[3] += lk * J.Jc[1][k];
      z[4] += lk * J.Jc[2][k];
    } else {
      z[5] += lk * J.dsig;
    }
  }
  for (int ch = 0; ch < 3; ++ch) {
    float t = 0.0f;
    for (int k = 0; k < nb; ++k) t += Cr[ch * nb + k] * J.Y[k];
    z[6 + ch] += J.live[ch] * t;
  }
}

__device__ void z_rgb_warp(const GJac& J, const float* Lt, int nb, float* Z, int lane) {
  const int n3 = 3 * nb, l = kNG + n3, T = rgb_tri_nb(nb);
  for (int i = lane; i < l * 9; i += 32) Z[i] = 0.0f;
  __syncwarp();
  for (int row = lane; row < l; row += 32) {
    if (row < n3) {
      const int ch = row / nb, k = row - ch * nb;
      const float* Ak = Lt + ch * T + tri(k, 0);
      float a = 0.0f;
      for (int k2 = 0; k2 <= k; ++k2) a += Ak[k2] * J.Y[k2];
      Z[row * 9 + 6 + ch] = J.live[ch] * a;
    } else {
      const int r = row - n3;
      float z[9];
      z_geo_rgb_row(J, Lt + rgb_off_E(nb) + tri(r, 0), Lt + rgb_off_C(nb) + r * n3, r, nb, z);
#pragma unroll
      for (int q = 0; q < 9; ++q) Z[row * 9 + q] = z[q];
    }
  }
  __syncwarp();
}

// fs: the Gaussian's active slot (the row of its training factors).
template <int F, int U>
__device__ float output_gain(const GJac& J, const Consts& c, const float* p, const Factors& Fa, int64_t fs,
                             const float* blk, float cg, float* Ls, float* Y, float* Z, float* W,
                             float* Bm, float* G, int lane) {
  const int l = out_l(F, c), u = out_u(F, c), nt = l * (l + 1) / 2;
  if (F == 0) {
    z_rgb_warp(J, Fa.L[0] + (size_t)fs * rgb_L_size(c.nb), c.nb, Z, lane);   // ends with __syncwarp
  } else {
    const float* Lg = Fa.L[F] + (size_t)fs * nt;   // rows read straight from global memory (L1)
    build_Y(F, J, c, p, Y, lane);                  // ends with __syncwarp
    for (int i = lane; i < l; i += 32) z_row<F, U>(i, u, Lg, Y, Z);
    __syncwarp();
  }
  for (int i = lane; i < u * (u + 1) / 2; i += 32) {   // W = Z^T Z
    int r = (int)((sqrtf(8.0f * i + 1.0f) - 1.0f) * 0.5f);
    while (tri(r + 1, 0) <= i) ++r;
    while (tri(r, 0) > i) --r;
    const int cc = i - tri(r, 0);
    float a = 0.0f;
    for (int k = 0; k < l; ++k) a += Z[k * u + r] * Z[k * u + cc];
    W[r * u + cc] = a;
    W[cc * u + r] = a;
  }
  build_B(F, blk, c, Bm, lane);                  // ends with __syncwarp
  return logdet_IcWB(u, cg, W, Bm, G, lane, c.crit);
}

template <int UO>
__global__ void __launch_bounds__(128, 3) k_view_gains(DevScene s, Consts c, DevCam cam1, const DevCam* cams,
                                                      const float* __restrict__ blocks, Factors F,
                                                      float* __restrict__ delta, double* __restrict__ partial,
                                                      int nt_max, int lu_max, int uu_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nB = block_floats(c.K), nBp = (nB + 3) & ~3;
  // multi-view launches: view = blockIdx.y (its own blocks and partial sums)
  const DevCam cam = cams ? cams[blockIdx.y] : cam1;
  blocks += (size_t)blockIdx.y * s.n_act * nBp;
  partial += (size_t)blockIdx.y * gridDim.x * nw * 3;
  const size_t per_warp = 2 * (size_t)lu_max + 3 * (size_t)uu_max + 32 * (sizeof(GJac) / 4) + 4;
  float* Ls = nullptr;
  float* Y = reinterpret_cast<float*>(smem) + warp * per_warp;
  float* Z = Y + lu_max;
  float* W = Z + lu_max;
  float* Bm = W + uu_max;
  float* G = Bm + uu_max;
  GJac* Jw = reinterpret_cast<GJac*>(G + uu_max);     // one per lane
  double acc3[3] = {0.0, 0.0, 0.0};
  const int64_t nbatch = (s.n_act + 31) / 32;
  const int64_t gw = (int64_t)blockIdx.x * nw + warp, nwarps = (int64_t)gridDim.x * nw;
  for (int64_t bt = gw; bt < nbatch; bt += nwarps) {
    // every lane takes one active slot of the batch: contributes? projection Jacobians
    const int64_t sll = bt * 32 + lane;
    bool mine = false;
    if (sll < s.n_act) {
      const int64_t gl = s.act[sll];
      mine = blocks[(size_t)sll * nBp + kOffW2] != 0.0f;
      if (mine) compute_gjac(s, c, cam, gl, Jw[lane]);
      else if (delta) { delta[3 * gl] = 0.0f; delta[3 * gl + 1] = 0.0f; delta[3 * gl + 2] = 0.0f; }
    }
    unsigned todo = __ballot_sync(0xffffffffu, mine);
    __syncwarp();
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t sl = bt * 32 + src;
      const int64_t g = s.act[sl];
      const float cg = s.aux[g].y;
      const float* blk = blocks + (size_t)sl * nBp;
      const float* p = s.p + (size_t)g * c.KC;
      const GJac& J = Jw[src];
      const float d0 = output_gain<0, 9>(J, c, p, F, sl, blk, cg, Ls, Y, Z, W, Bm, G, lane);
      const float d1 = output_gain<1, 7>(J, c, p, F, sl, blk, cg, Ls, Y, Z, W, Bm, G, lane);
      const float d2 = output_gain<2, UO>(J, c, p, F, sl, blk, cg, Ls, Y, Z, W, Bm, G, lane);
      if (lane == 0) {
        if (delta) { delta[3 * g] = d0; delta[3 * g + 1] = d1; delta[3 * g + 2] = d2; }
        acc3[0] += d0; acc3[1] += d1; acc3[2] += d2;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    double* out = partial + 3 * ((size_t)blockIdx.x * nw + warp);
    out[0] = acc3[0]; out[1] = acc3[1]; out[2] = acc3[2];
  }
}

// ------------------------------------ multi-view gains, Gaussian-major
// One warp per Gaussian and 32 views per pass (lane = view). L~ of the three
// outputs is staged in the warp's shared memory once per Gaussian and read
// by broadcast. The colour and depth gains of a (view, Gaussian) run in one
// lane, in registers:
//   Z = L~ M^T row by row (M sparse by parameter block), W = Z^T Z,
//   W = Lw Lw^T (Cholesky; a column with no pivot left is dropped, which
//   happens exactly when M has a zero row, e.g. a clamped colour channel),
//   log det(I + c W B) = log det(I + c Lw^T B Lw), the latter SPD with
//   eigenvalues >= 1, factorised without pivoting; its pivots are 1 + x and
//   the sum of log1p(x) is the gain.
// The object gain runs warp-cooperatively per (view, Gaussian): the
// probability columns of M (d p / d o) do not depend on the view, so
// Z_p = L~[:, logits] (d p / d o)^T and W_pp = Z_p^T Z_p are formed once per
// Gaussian; per view only the geometric columns change.

// Packed lower-triangle index with compile-time arguments.
__host__ __device__ constexpr int ptri(int r, int cc) { return r * (r + 1) / 2 + cc; }

// (Every loop below has a constant trip count, with the triangular bounds
// as conditions, so that full unrolling leaves only constant indices and the
// arrays stay in registers.)
template <int U>
__device__ __forceinline__ float logdet_lane(float (&Wm)[ptri(U, 0)], const float (&Bm)[ptri(U, 0)], float cg,
                                             int crit = 0) {
  if (crit != 0) {   // trace criteria: c tr(W B) (W and B symmetric, packed)
    float t = 0.0f;
#pragma unroll
    for (int r = 0; r < U; ++r)
#pragma unroll
      for (int cc = 0; cc < U; ++cc)
        if (cc <= r) t += (cc == r ? 1.0f : 2.0f) * Wm[ptri(r, cc)] * Bm[ptri(r, cc)];
    return cg * t;
  }
  // Wm <- Lw (in place)
#pragma unroll
  for (int j = 0; j < U; ++j) {
    float d = Wm[ptri(j, j)];
#pragma unroll
    for (int m = 0; m < U; ++m)
      if (m < j) d -= Wm[ptri(j, m)] * Wm[ptri(j, m)];
    const bool live = d > 1e-6f * Wm[ptri(j, j)] && d > 0.0f;
    const float ljj = live ? sqrtf(d) : 0.0f;
    const float il = live ? 1.0f / ljj : 0.0f;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      if (i > j) {
        float a = Wm[ptri(i, j)];
#pragma unroll
        for (int m = 0; m < U; ++m)
          if (m < j) a -= Wm[ptri(i, m)] * Wm[ptri(j, m)];
        Wm[ptri(i, j)] = a * il;
      }
    }
    Wm[ptri(j, j)] = ljj;
  }
  // X = c Lw^T B Lw (lower triangle), one column of B Lw at a time
  float X[ptri(U, 0)];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    float t[U];
#pragma unroll
    for (int a = 0; a < U; ++a) {
      float acc = 0.0f;
#pragma unroll
      for (int b = 0; b < U; ++b)
        if (b >= j) acc += (a >= b ? Bm[ptri(a, b)] : Bm[ptri(b, a)]) * Wm[ptri(b, j)];
      t[a] = acc;
    }
#pragma unroll
    for (int i = 0; i < U; ++i) {
      if (i >= j) {
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < U; ++a)
          if (a >= i) acc += Wm[ptri(a, i)] * t[a];
        X[ptri(i, j)] = cg * acc;
      }
    }
  }
  // Cholesky of I + X with the identity kept apart: pivot = 1 + x
  float ld = 0.0f;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    float x = X[ptri(j, j)];
#pragma unroll
    for (int m = 0; m < U; ++m)
      if (m < j) x -= X[ptri(j, m)] * X[ptri(j, m)];
    x = fmaxf(x, -0.999999f);
    ld += log1pf(x);
    const float il = rsqrtf(1.0f + x);
#pragma unroll
    for (int i = 0; i < U; ++i) {
      if (i > j) {
        float a = X[ptri(i, j)];
#pragma unroll
        for (int m = 0; m < U; ++m)
          if (m < j) a -= X[ptri(i, m)] * X[ptri(j, m)];
        X[ptri(i, j)] = a * il;
      }
    }
  }
  return ld;
}

// Colour gain of one (view, Gaussian) in one lane. Lt: the block form of
// L~ of the colour output (see Factors; shared memory, same for every lane).
template <int DEG>
__device__ __forceinline__ float rgb_gain_lane(const GJac& J, const float* __restrict__ Lt,
                                               const float* __restrict__ blk, float cg, int crit) {
  constexpr int NB = (DEG + 1) * (DEG + 1), TN = NB * (NB + 1) / 2, N3 = 3 * NB;
  const float* Cm = Lt + 3 * TN;
  const float* Em = Cm + kNG * N3;
  float Wm[45];
#pragma unroll
  for (int i = 0; i < 45; ++i) Wm[i] = 0.0f;
  // SH rows: channel ch only, W[6 + ch][6 + ch] += live_ch |A_ch Y|^2
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float ss = 0.0f;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      float a = 0.0f;
#pragma unroll
      for (int k2 = 0; k2 < NB; ++k2)
        if (k2 <= k) a += Lt[ch * TN + ptri(k, k2)] * J.Y[k2];
      ss += a * a;
    }
    Wm[ptri(6 + ch, 6 + ch)] += J.live[ch] * ss;
  }
  // geometric rows
#pragma unroll
  for (int r = 0; r < kNG; ++r) {
    const float* Er = Em + ptri(r, 0);
    float z[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) z[q] = 0.0f;
#pragma unroll
    for (int k = 0; k < kNG; ++k) {
      if (k <= r) {
        const float lk = Er[k];
        if (k < 3) {
          z[0] += lk * J.Jm[0][k];
          z[1] += lk * J.Jm[1][k];
          z[6] += lk * J.Jrgb[0][k];
          z[7] += lk * J.Jrgb[1][k];
          z[8] += lk * J.Jrgb[2][k];
        }
        if (k < 10) {
          z[2] += lk * J.Jc[0][k];
          z[3] += lk * J.Jc[1][k];
          z[4] += lk * J.Jc[2][k];
        } else {
          z[5] += lk * J.dsig;
        }
      }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float t = 0.0f;
#pragma unroll
      for (int k = 0; k < NB; ++k) t += Cm[r * N3 + ch * NB + k] * J.Y[k];
      z[6 + ch] += J.live[ch] * t;
    }
#pragma unroll
    for (int rr = 0; rr < 9; ++rr)
#pragma unroll
      for (int cc = 0; cc < 9; ++cc)
        if (cc <= rr) Wm[ptri(rr, cc)] += z[rr] * z[cc];
  }
  float Bm[45];
  const float w2 = blk[kOffW2];
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int cc = 0; cc < 9; ++cc)
      if (cc <= r)
        Bm[ptri(r, cc)] = r < 6 ? blk[kOffQrgb + ptri(r, cc)]
                                : (cc < 6 ? blk[kOffXrgb + 6 * (r - 6) + cc] : (r == cc ? w2 : 0.0f));
  return logdet_lane<9>(Wm, Bm, cg, crit);
}

// Depth gain of one (view, Gaussian) in one lane.
__device__ __forceinline__ float depth_gain_lane(const GJac& J, const float* __restrict__ Lt,
                                                 const float* __restrict__ blk, float cg, int crit) {
  float Wm[28];
#pragma unroll
  for (int i = 0; i < 28; ++i) Wm[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < kNG; ++i) {
    const float* Li = Lt + ptri(i, 0);
    float z[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) z[q] = 0.0f;
#pragma unroll
    for (int k = 0; k < kNG; ++k) {
      if (k > i) continue;
      const float lk = Li[k];
      if (k < 3) {
        z[0] += lk * J.Jm[0][k];
        z[1] += lk * J.Jm[1][k];
        z[6] += lk * J.Jz[k];
      }
      if (k < 10) {
        z[2] += lk * J.Jc[0][k];
        z[3] += lk * J.Jc[1][k];
        z[4] += lk * J.Jc[2][k];
      } else {
        z[5] += lk * J.dsig;
      }
    }
#pragma unroll
    for (int r = 0; r < 7; ++r)
#pragma unroll
      for (int cc = 0; cc < 7; ++cc)
        if (cc <= r) Wm[ptri(r, cc)] += z[r] * z[cc];
  }
  float Bm[28];
#pragma unroll
  for (int r = 0; r < 7; ++r)
#pragma unroll
    for (int cc = 0; cc < 7; ++cc)
      if (cc <= r) Bm[ptri(r, cc)] = r < 6 ? blk[kOffQd + ptri(r, cc)] : (cc < 6 ? blk[kOffXd + cc] : blk[kOffW2]);
  return logdet_lane<7>(Wm, Bm, cg, crit);
}

// Object gain of one (view, Gaussian), rows in registers: lane r < u holds
// row r of G = I + c W B (u = 6 + K <= UO <= 32), formed from W (shared,
// u x u) and the structured block B = [[Q, X^T], [X, W2 (I + 1 1^T)]]:
//   G[r][c<6]  = c (sum_{k<6} W[r][k] Q[k][c] + sum_j W[r][6+j] X[j][c])
//   G[r][6+j]  = c (sum_{k<6} W[r][k] X[j][k] + W2 (W[r][6+j] + sum_i W[r][6+i]))
// (plus the identity), then log|det G| by Gaussian elimination with partial
// pivoting across the lanes: the pivot row is found by a warp arg-max and
// broadcast by shuffles, rows already used as pivots drop out (no swaps).
// After each step every row shifts left by one column, so the pivot column
// is always g[0] and the step is a loop body of its own (compact code: this
// runs once per (view, Gaussian), and fully unrolled steps overflow the
// instruction cache). Qs: Q (6 x 6, full), Xs: X (K x 6) in shared memory.
template <int UO>
__device__ __forceinline__ float obj_logdet_rows(int u, int K, float cg, float w2, const float* W, const float* Qs,
                                                 const float* Xs, int lane, int crit) {
  const int r = lane;
  const bool row = r < u;
  float wr[UO];
#pragma unroll
  for (int k = 0; k < UO; ++k) wr[k] = (row && k < u) ? W[r * u + k] : 0.0f;
  if (crit != 0) {   // trace criteria: c tr(W B) = c sum_r sum_k W[r][k] B[k][r], row r's share
    float br = 0.0f;
    if (row) {
      if (r < 6) {
#pragma unroll
        for (int k = 0; k < UO; ++k)
          if (k < u) br += wr[k] * (k < 6 ? Qs[k * 6 + r] : Xs[(k - 6) * 6 + r]);
      } else {
        const int j = r - 6;
        float sw = 0.0f;
#pragma unroll
        for (int k = 6; k < UO; ++k)
          if (k < u) sw += wr[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) br += wr[k] * Xs[j * 6 + k];
        float wrr = 0.0f;
#pragma unroll
        for (int k = 6; k < UO; ++k)
          if (k == r) wrr = wr[k];
        br += w2 * (wrr + sw);
      }
    }
    for (int o = 16; o >= 1; o >>= 1) br += __shfl_xor_sync(0xffffffffu, br, o);
    return cg * br;
  }
  float sw = 0.0f;
#pragma unroll
  for (int k = 6; k < UO; ++k) sw += wr[k];
  float g[UO];
  {
    // G[r][c < 6]: one pass over k (rows of [Q; X]), W[r][k] read from shared memory
    float a[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    const float* Wr = W + (row ? r : 0) * u;
    for (int k = 0; k < u; ++k) {
      const float wk = row ? Wr[k] : 0.0f;
      const float* bk = k < 6 ? Qs + k * 6 : Xs + (k - 6) * 6;
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) a[cc] += wk * bk[cc];
    }
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) g[cc] = (r == cc ? 1.0f : 0.0f) + cg * a[cc];
  }
#pragma unroll
  for (int j = 0; j < UO - 6; ++j) {
    // Xs holds the K rows of X only: rows j >= K are never read (the
    // template covers up to UO - 6 of them, past the end of the buffer)
    float a = 0.0f;
    if (j < K) {
#pragma unroll
      for (int k = 0; k < 6; ++k) a += wr[k] * Xs[j * 6 + k];
      a += w2 * (wr[6 + j] + sw);
    }
    g[6 + j] = (r == 6 + j ? 1.0f : 0.0f) + (j < K ? cg * a : 0.0f);
  }
  bool done = !row;
  // log |det| = log(mant) + ex log 2: the pivot magnitudes are multiplied into
  // a mantissa in [1, 2) and their binary exponents summed (one multiply and
  // a few integer operations per step instead of a logarithm)
  float mant = 1.0f;
  int ex = 0;
  for (int k = 0; k < u; ++k) {
    // pivot row: the largest |g[0]| among the rows left, by one warp max over
    // keys (|g[0]| with its lowest 5 bits replaced by the inverted lane, so
    // near-ties go to the lower row; |g| >= 0 orders like its bit pattern)
    const unsigned key = done ? 0u : ((__float_as_uint(fabsf(g[0])) & ~31u) | (unsigned)(31 - r));
    const int bl = 31 - (int)(__reduce_max_sync(0xffffffffu, key) & 31u);
    const float piv = __shfl_sync(0xffffffffu, g[0], bl);
    {
      const uint32_t b = __float_as_uint(mant * fabsf(piv));
      ex += (int)((b >> 23) & 0xFFu) - 127;
      mant = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    }
    const bool upd = !done && r != bl;
    const float f = upd ? __fdividef(g[0], piv) : 0.0f;
    const int live = u - k - 1;                 // columns right of the pivot (warp-uniform)
#pragma unroll
    for (int j0 = 0; j0 < UO - 1; j0 += 4) {
      if (j0 < live) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          if (j0 + jj < UO - 1) {
            const float pj = __shfl_sync(0xffffffffu, g[j0 + jj + 1], bl);
            g[j0 + jj] = g[j0 + jj + 1] - f * pj;
          }
        }
      }
    }
    if (r == bl) done = true;
  }
  return logf(mant) + (float)ex * 0.693147180559945309f;
}

// The same for 32 < u <= UO <= 64 rows: lane l holds rows l and l + 32. Row r
// of G = I + c W B is formed from row r of W (shared memory) and the
// structured B: G[r][c < 6] = [r = c] + c sum_k W[r][k] B[k][c] (B's first six
// columns are Q above X), and for j < K
//   G[r][6 + j] = [r = 6 + j] + c (sum_{k<6} W[r][k] X[j][k] + w2 (W[r][6 + j] + sum_{k>=6} W[r][k]))
// (B's probability block is w2 (I + 1 1^T)). Gaussian elimination with
// partial pivoting (the largest |G[.][k]| among the rows left, by one warp
// max over 6-bit row keys; near-ties within 2^-17 relative go to the lower
// row), the rows shifted left by one column per step.
template <int UO>
__device__ __forceinline__ float obj_logdet_rows2(int u, int K, float cg, float w2, const float* W, const float* Qs,
                                                  const float* Xs, int lane, int crit) {
  const int ra = lane, rb = lane + 32;
  const bool rowa = ra < u, rowb = rb < u;
  if (crit != 0) {   // trace criteria: c tr(W B) = c sum_r sum_k W[r][k] B[k][r]
    float br = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h ? rb : ra;
      if (!(h ? rowb : rowa)) continue;
      const float* Wr = W + r * u;
      if (r < 6) {
        for (int k = 0; k < u; ++k) br += Wr[k] * (k < 6 ? Qs[k * 6 + r] : Xs[(k - 6) * 6 + r]);
      } else {
        const int j = r - 6;
        float sw = 0.0f;
        for (int k = 6; k < u; ++k) sw += Wr[k];
        for (int k = 0; k < 6; ++k) br += Wr[k] * Xs[j * 6 + k];
        br += w2 * (Wr[r] + sw);
      }
    }
    for (int o = 16; o >= 1; o >>= 1) br += __shfl_xor_sync(0xffffffffu, br, o);
    return cg * br;
  }
  float ga[UO], gb[UO];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = h ? rb : ra;
    const bool row = h ? rowb : rowa;
    float* g = h ? gb : ga;
    const float* Wr = W + (row ? r : 0) * u;
    float a[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float sw = 0.0f, w6[6];
    for (int k = 0; k < u; ++k) {
      const float wk = row ? Wr[k] : 0.0f;
      if (k >= 6) sw += wk;
      const float* bk = k < 6 ? Qs + k * 6 : Xs + (k - 6) * 6;
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) a[cc] += wk * bk[cc];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) w6[k] = row ? Wr[k] : 0.0f;
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) g[cc] = (r == cc ? 1.0f : 0.0f) + cg * a[cc];
#pragma unroll
    for (int j = 0; j < UO - 6; ++j) {
      float t = 0.0f;
      if (j < K) {
#pragma unroll
        for (int k = 0; k < 6; ++k) t += w6[k] * Xs[j * 6 + k];
        t += w2 * ((row ? Wr[6 + j] : 0.0f) + sw);
      }
      g[6 + j] = (r == 6 + j ? 1.0f : 0.0f) + (j < K ? cg * t : 0.0f);
    }
  }
  bool done_a = !rowa, done_b = !rowb;
  float mant = 1.0f;
  int ex = 0;
  for (int k = 0; k < u; ++k) {
    const unsigned ka = done_a ? 0u : ((__float_as_uint(fabsf(ga[0])) & ~63u) | (unsigned)(63 - ra));
    const unsigned kb = done_b ? 0u : ((__float_as_uint(fabsf(gb[0])) & ~63u) | (unsigned)(63 - rb));
    const int prow = 63 - (int)(__reduce_max_sync(0xffffffffu, max(ka, kb)) & 63u);
    const int bl = prow & 31;
    const bool hb = prow >= 32;                 // the same for the whole warp
    const float piv = hb ? __shfl_sync(0xffffffffu, gb[0], bl) : __shfl_sync(0xffffffffu, ga[0], bl);
    {
      const uint32_t b = __float_as_uint(mant * fabsf(piv));
      ex += (int)((b >> 23) & 0xFFu) - 127;
      mant = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    }
    const float fa_ = (!done_a && ra != prow) ? __fdividef(ga[0], piv) : 0.0f;
    const float fb_ = (!done_b && rb != prow) ? __fdividef(gb[0], piv) : 0.0f;
    const int live = u - k - 1;
#pragma unroll
    for (int j0 = 0; j0 < UO - 1; j0 += 4) {
      if (j0 < live) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          if (j0 + jj < UO - 1) {
            const float pj = hb ? __shfl_sync(0xffffffffu, gb[j0 + jj + 1], bl)
                                : __shfl_sync(0xffffffffu, ga[j0 + jj + 1], bl);
            ga[j0 + jj] = ga[j0 + jj + 1] - fa_ * pj;
            gb[j0 + jj] = gb[j0 + jj + 1] - fb_ * pj;
          }
        }
      }
    }
    if (ra == prow) done_a = true;
    if (rb == prow) done_b = true;
  }
  return logf(mant) + (float)ex * 0.693147180559945309f;
}

struct GmLayout {     // per-warp shared memory (floats)
  int nt0, nt1, nt2;  // packed sizes of L~ per output
  int l2, u2;         // object output sizes
  int off_L1, off_L2, off_Yg, off_s, off_Zp, off_Zg, off_W, off_B, off_G, per_warp;
};

__host__ __device__ inline GmLayout gm_layout(const Consts& c) {
  GmLayout y{};
  const int l0 = kNG + 3 * c.nb, l1 = kNG;
  y.l2 = kNG + c.KC;
  y.u2 = 6 + c.K;
  y.nt0 = rgb_L_size(c.nb);
  (void)l0;
  y.nt1 = l1 * (l1 + 1) / 2;
  y.nt2 = y.l2 * (y.l2 + 1) / 2;
  auto r4 = [](int x) { return (x + 3) & ~3; };
  y.off_L1 = r4(y.nt0);
  y.off_L2 = y.off_L1 + r4(y.nt1);
  y.off_Yg = y.off_L2 + r4(y.nt2);
  y.off_s = y.off_Yg + 66 * 32;
  y.off_Zp = y.off_s + r4(y.l2);
  y.off_Zg = y.off_Zp + r4(y.l2 * c.K);
  y.off_W = y.off_Zg + r4(y.l2 * 6);
  // u <= 40 takes the row eliminations, which read only W, Q (6 x 6) and
  // X (K x 6): B holds those and there is no G workspace; larger u takes
  // logdet_IcWB with a full u x u B and G
  const bool rows = y.u2 <= 40;
  y.off_B = y.off_W + r4(y.u2 * y.u2);
  y.off_G = y.off_B + (rows ? r4(36 + 6 * c.K) : r4(y.u2 * y.u2));
  y.per_warp = y.off_G + (rows ? 0 : r4(y.u2 * y.u2));
  return y;
}

template <int DEG>
__global__ void __launch_bounds__(256, 1) k_gains_gm(DevScene s, Consts c, const DevCam* __restrict__ cams, int nv,
                                                    const float* __restrict__ blocks, Factors F,
                                                    double* __restrict__ partial, int nparts) {
  extern __shared__ __align__(16) float smf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const GmLayout y = gm_layout(c);
  float* base = smf + (size_t)warp * y.per_warp;
  float* L0 = base;
  float* L1 = base + y.off_L1;
  float* L2 = base + y.off_L2;
  float* Yg = base + y.off_Yg;    // [66][32]: geometric rows of M^T per lane (view)
  float* srow = base + y.off_s;
  float* Zp = base + y.off_Zp;    // [l2][K]
  float* Zg = base + y.off_Zg;    // [l2][6]
  float* Wo = base + y.off_W;     // [u2][u2]
  float* Bo = base + y.off_B;
  float* Go = base + y.off_G;
  const int nBp = (block_floats(c.K) + 3) & ~3;
  const int K = c.K, KC = c.KC, l2 = y.l2, u2 = y.u2;
  const int v0 = 32 * blockIdx.y;
  const int v = v0 + lane;
  const bool vok = v < nv;
  const DevCam* camp = cams + (vok ? v : 0);
  double acc[3] = {0.0, 0.0, 0.0};
  const int slot = blockIdx.x * nw + warp;
  for (int64_t sl = slot; sl < s.n_act; sl += (int64_t)gridDim.x * nw) {
    const int64_t g = s.act[sl];                       // active: c_g > 0
    const float cg = s.aux[g].y;
    const float* blk = blocks + ((size_t)v * s.n_act + sl) * nBp;
    const bool mine = vok && blk[kOffW2] != 0.0f;
    const unsigned todo_all = __ballot_sync(0xffffffffu, mine);
    if (todo_all == 0u) continue;
    // stage L~ of the three outputs
    {
      const float* g0 = F.L[0] + (size_t)sl * y.nt0;
      const float* g1 = F.L[1] + (size_t)sl * y.nt1;
      const float* g2 = F.L[2] + (size_t)sl * y.nt2;
      for (int i = lane; i < y.nt0; i += 32) L0[i] = g0[i];
      for (int i = lane; i < y.nt1; i += 32) L1[i] = g1[i];
      for (int i = lane; i < y.nt2; i += 32) L2[i] = g2[i];
    }
    const float* p = s.p + (size_t)g * KC;
    __syncwarp();
    // view-independent object pieces: s_i, Z_p, W_pp (into Wo's lower-right block)
    for (int i = lane; i < l2; i += 32) {
      float a = 0.0f;
      for (int b = 0; kNG + b <= i && b < KC; ++b) a += L2[tri(i, kNG + b)] * p[b];
      srow[i] = a;
    }
    __syncwarp();
    for (int t = lane; t < l2 * K; t += 32) {
      const int i = t / K, j = t - i * K;
      const float lij = (kNG + 1 + j <= i) ? L2[tri(i, kNG + 1 + j)] : 0.0f;
      Zp[t] = p[1 + j] * (lij - srow[i]);
    }
    __syncwarp();
    for (int t = lane; t < K * K; t += 32) {
      const int a = t / K, b = t - a * K;
      if (b > a) continue;
      float w = 0.0f;
      for (int i = 0; i < l2; ++i) w += Zp[i * K + a] * Zp[i * K + b];
      Wo[(6 + a) * u2 + 6 + b] = w;
      Wo[(6 + b) * u2 + 6 + a] = w;
    }
    // per lane: projection Jacobians, geometric rows of M^T for the object pass
    GJac J;
    if (mine) {
      compute_gjac_t<DEG>(s, c, *camp, g, J);
#pragma unroll
      for (int q = 0; q < 66; ++q) {
        const int k = q / 6, cc = q - 6 * (q / 6);
        float val = 0.0f;
        if (cc < 2) val = k < 3 ? J.Jm[cc][k] : 0.0f;
        else if (cc < 5) val = k < 10 ? J.Jc[cc - 2][k] : 0.0f;
        else val = k == 10 ? J.dsig : 0.0f;
        Yg[q * 32 + lane] = val;
      }
      acc[1] += (double)depth_gain_lane(J, L1, blk, cg, c.crit);
      acc[0] += (double)rgb_gain_lane<DEG>(J, L0, blk, cg, c.crit);
    }
    __syncwarp();
    // object gain, one (view, Gaussian) at a time
    unsigned todo = todo_all;
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const float* bsrc = blocks + ((size_t)(v0 + src) * s.n_act + sl) * nBp;
      for (int i = lane; i < l2; i += 32) {           // Z_g = L~[:, :11] M_g^T
        float zr[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        const int kg = i < kNG - 1 ? i : kNG - 1;
        const float* Li = L2 + tri(i, 0);
        for (int k = 0; k <= kg; ++k) {
          const float lk = Li[k];
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) zr[cc] += lk * Yg[(6 * k + cc) * 32 + src];
        }
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) Zg[i * 6 + cc] = zr[cc];
      }
      __syncwarp();
      for (int t = lane; t < 21 + 6 * K; t += 32) {   // W_gg (packed) and W_gp
        float w = 0.0f;
        int r, cc;
        if (t < 21) {
          tri_decode(t, r, cc);
          for (int i = 0; i < l2; ++i) w += Zg[i * 6 + r] * Zg[i * 6 + cc];
        } else {
          const int q = t - 21;
          r = q / K;
          cc = 6 + (q - r * K);
          for (int i = 0; i < l2; ++i) w += Zg[i * 6 + r] * Zp[i * K + cc - 6];
        }
        Wo[r * u2 + cc] = w;
        Wo[cc * u2 + r] = w;
      }
      float d2;
      if (u2 <= 40) {
        // Q (full 6 x 6) and X of this view's block into shared memory
        for (int i = lane; i < 36 + 6 * K; i += 32)
          Bo[i] = i < 36 ? q6(bsrc + kOffQo, i / 6, i % 6) : bsrc[kOffXo + i - 36];
        __syncwarp();
        const float w2 = bsrc[kOffW2];
        d2 = u2 <= 24   ? obj_logdet_rows<24>(u2, K, cg, w2, Wo, Bo, Bo + 36, lane, c.crit)
             : u2 <= 32 ? obj_logdet_rows<32>(u2, K, cg, w2, Wo, Bo, Bo + 36, lane, c.crit)
                        : obj_logdet_rows2<40>(u2, K, cg, w2, Wo, Bo, Bo + 36, lane, c.crit);
        __syncwarp();
      } else {
        build_B(2, bsrc, c, Bo, lane);                 // ends with __syncwarp
        d2 = logdet_IcWB(u2, cg, Wo, Bo, Go, lane, c.crit);
      }
      if (lane == src) acc[2] += (double)d2;
    }
    __syncwarp();
  }
  if (vok) {
    double* out = partial + ((size_t)v * nparts + slot) * 3;
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = acc[2];
  }
}

__global__ void k_reduce_partial(const double* __restrict__ partial, int nblocks, double* out3) {
  __shared__ double sm[3][256];
  const int tid = threadIdx.x;
  partial += (size_t)blockIdx.x * nblocks * 3;     // one block per view
  out3 += 3 * blockIdx.x;
  double a[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < nblocks; i += 256)
    for (int f = 0; f < 3; ++f) a[f] += partial[3 * i + f];
  for (int f = 0; f < 3; ++f) sm[f][tid] = a[f];
  __syncthreads();
  for (int h = 128; h >= 1; h >>= 1) {
    if (tid < h)
      for (int f = 0; f < 3; ++f) sm[f][tid] += sm[f][tid + h];
    __syncthreads();
  }
  if (tid < 3) out3[tid] = sm[tid][0];
}

__global__ void k_final_scores(const double* __restrict__ igc, const double* __restrict__ igt,
                               int n_cand, int n_train, Consts c, float* __restrict__ out4,
                               int* best, float* best_score, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double nrm[3] = {0.0, 0.0, 0.0};
  for (int t = 0; t < n_train; ++t)
    for (int f = 0; f < 3; ++f) nrm[f] += igt[3 * t + f];
  for (int f = 0; f < 3; ++f) nrm[f] /= (double)n_train;
  const bool empty = !(nrm[0] != 0.0 && nrm[1] != 0.0 && nrm[2] != 0.0);
  *err = empty ? 1 : 0;
  int bi = -1;
  float bs = 0.0f;
  for (int v = 0; v < n_cand; ++v) {
    double tot = empty ? (double)NAN
                       : igc[3 * v] / nrm[0] + (double)c.beta_d * igc[3 * v + 1] / nrm[1] +
                             (double)c.beta_o * igc[3 * v + 2] / nrm[2];
    out4[4 * v] = (float)igc[3 * v];
    out4[4 * v + 1] = (float)igc[3 * v + 1];
    out4[4 * v + 2] = (float)igc[3 * v + 2];
    out4[4 * v + 3] = (float)tot;
    if (!empty && (bi < 0 || tot > (double)bs)) { bi = v; bs = (float)tot; }
  }
  *best = bi;
  *best_score = bs;
}

// Gradients of the raw parameters of each projected Gaussian from the
// gradients of its projected quantities (one thread per Gaussian): the
// transpose of the projection Jacobian M applied to
// (mean2D, conic, sigma, colour, z), and the softmax Jacobian to the
// probability gradients.
__global__ void k_project_backward(DevScene s, Consts c, DevCam cam, const float* __restrict__ gacc, int gw,
                                   const int4* __restrict__ rect, float* __restrict__ g_mu,
                                   float* __restrict__ g_logs, float* __restrict__ g_q, float* __restrict__ g_rho,
                                   float* __restrict__ g_sh, float* __restrict__ g_obj) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= s.n || rect[g].x < 0) return;
  const float* a = gacc + (size_t)g * gw;
  bool any = false;
  for (int q = 0; q < gw; ++q) any |= a[q] != 0.0f;
  if (!any) return;
  GJac J;
  compute_gjac(s, c, cam, g, J);
  const float gm0 = a[0], gm1 = a[1], gcon[3] = {a[2], a[3], a[4]}, gsig = a[5];
  const float gcol[3] = {a[6], a[7], a[8]}, gz = a[9];
  for (int m = 0; m < 3; ++m) {
    float v = J.Jm[0][m] * gm0 + J.Jm[1][m] * gm1 + J.Jz[m] * gz;
    for (int e = 0; e < 3; ++e) v += J.Jc[e][m] * gcon[e];
    for (int ch = 0; ch < 3; ++ch) v += J.Jrgb[ch][m] * gcol[ch];
    g_mu[3 * g + m] += v;
  }
  for (int k = 0; k < 3; ++k) {
    float v = 0.0f;
    for (int e = 0; e < 3; ++e) v += J.Jc[e][3 + k] * gcon[e];
    g_logs[3 * g + k] += v;
  }
  for (int i = 0; i < 4; ++i) {
    float v = 0.0f;
    for (int e = 0; e < 3; ++e) v += J.Jc[e][6 + i] * gcon[e];
    g_q[4 * g + i] += v;
  }
  g_rho[g] += J.dsig * gsig;
  for (int k = 0; k < c.nb; ++k)
    for (int ch = 0; ch < 3; ++ch) g_sh[((size_t)g * c.nb + k) * 3 + ch] += J.live[ch] * J.Y[k] * gcol[ch];
  const float* p = s.p + (size_t)g * c.KC;
  float pg = 0.0f;
  for (int k = 1; k < c.KC; ++k) pg += p[k] * a[10 + k];
  for (int b = 0; b < c.KC; ++b) g_obj[(size_t)g * c.KC + b] += p[b] * ((b >= 1 ? a[10 + b] : 0.0f) - pg);
}

struct GainsDims { int nt_max, lu_max, uu_max; };

GainsDims gains_dims(const Consts& c) {
  GainsDims d{0, 0, 0};
  for (int f = 0; f < 3; ++f) {
    const int l = out_l(f, c), u = out_u(f, c);
    if (l * (l + 1) / 2 > d.nt_max) d.nt_max = l * (l + 1) / 2;
    if (l * u > d.lu_max) d.lu_max = l * u;
    if (u * u > d.uu_max) d.uu_max = u * u;
  }
  d.nt_max = (d.nt_max + 3) & ~3;
  d.lu_max = (d.lu_max + 3) & ~3;
  d.uu_max = (d.uu_max + 3) & ~3;
  return d;
}

size_t gains_smem_per_warp(const GainsDims& d) {
  return (2 * (size_t)d.lu_max + 3 * (size_t)d.uu_max + 32 * (sizeof(GJac) / 4) + 4) * sizeof(float);
}

int warps_for(size_t per_warp) {
  const size_t budget = 200 * 1024;
  int w = (int)(budget / per_warp);
  return w < 1 ? 1 : (w > 4 ? 4 : w);
}

}  // namespace


int launch_tri_table_init(cudaStream_t st) {
  k_tri_init<<<(kTriMax + 255) / 256, 256, 0, st>>>();
  return 1;
}

int launch_build_factors(const DevScene& s, const Consts& c, const DevCam* cams, const float* blocks,
                         int n_train, const Factors& f, int* d_err, cudaStream_t st) {
  const FactLayout y = fact_layout(c);
  const size_t pw = (size_t)y.d_per_warp * sizeof(double) + (size_t)y.f_per_warp * sizeof(float);
  int nw = (int)((220 * 1024) / pw);
  nw = nw < 1 ? 1 : (nw > 12 ? 12 : nw);
  const size_t sm = pw * nw;
  cudaFuncSetAttribute(k_build_factors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (s.n_act <= 0) return 0;
  const int64_t nblk = (s.n_act + nw - 1) / nw;
  const int64_t gcap = (int64_t)device_sm_count() * 32;
  const int grid = (int)(nblk < gcap ? nblk : gcap);
  k_build_factors<<<grid, 32 * nw, sm, st>>>(s, c, cams, blocks, n_train, f, d_err, y);
  return 1;
}

template <int UO>
void launch_gains_k(const DevScene& s, const Consts& c, const DevCam& cam, const DevCam* cams, int nv,
                    const float* blocks, const Factors& f, float* delta, double* partial, int grid, int nw,
                    size_t sm, const GainsDims& d, cudaStream_t st) {
  cudaFuncSetAttribute(k_view_gains<UO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_view_gains<UO><<<dim3(grid, nv), 32 * nw, sm, st>>>(s, c, cam, cams, blocks, f, delta, partial, d.nt_max,
                                                        d.lu_max, d.uu_max);
}

template <class L>
void dispatch_uo(int K, L&& fn) {
  const int uo = 6 + K;
  if (uo <= 24) fn(std::integral_constant<int, 24>{});
  else if (uo <= 40) fn(std::integral_constant<int, 40>{});
  else if (uo <= 72) fn(std::integral_constant<int, 72>{});
  else fn(std::integral_constant<int, 136>{});
}

int launch_view_gains(const DevScene& s, const Consts& c, const DevCam& cam, const float* blocks,
                      const Factors& f, float* delta, double* partial, int nblocks_cap,
                      int* nblocks_used, cudaStream_t st) {
  const GainsDims d = gains_dims(c);
  const size_t pw = gains_smem_per_warp(d);
  const int nw = warps_for(pw);
  const size_t sm = pw * nw;
  const int64_t nblk = ((s.n_act + 31) / 32 + nw - 1) / nw;
  int grid = (int)(nblk < nblocks_cap ? nblk : nblocks_cap);
  if (grid < 1) grid = 1;
  *nblocks_used = grid * nw;        // one partial sum per warp
  dispatch_uo(c.K, [&](auto uo) {
    launch_gains_k<decltype(uo)::value>(s, c, cam, nullptr, 1, blocks, f, delta, partial, grid, nw, sm, d, st);
  });
  return 1;
}

int launch_views_gains(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const float* blocks,
                       const Factors& f, double* partial, int parts_cap, int* nparts, cudaStream_t st) {
  const GainsDims d = gains_dims(c);
  const size_t pw = gains_smem_per_warp(d);
  const int nw = warps_for(pw);
  const size_t sm = pw * nw;
  const int64_t nblk = ((s.n_act + 31) / 32 + nw - 1) / nw;
  int grid = (int)(nblk < parts_cap / nw ? nblk : parts_cap / nw);
  if (grid < 1) grid = 1;
  *nparts = grid * nw;
  DevCam dummy{};
  dispatch_uo(c.K, [&](auto uo) {
    launch_gains_k<decltype(uo)::value>(s, c, dummy, cams, nv, blocks, f, nullptr, partial, grid, nw, sm, d, st);
  });
  return 1;
}

int launch_views_gains_gm(const DevScene& s, const Consts& c, const DevCam* cams, int nv, const float* blocks,
                          const Factors& f, double* partial, int parts_cap, int* nparts, cudaStream_t st) {
  if (nv <= 0) return 0;
  const GmLayout y = gm_layout(c);
  const size_t pw = (size_t)y.per_warp * sizeof(float);
  int nw = (int)((size_t)(220 * 1024) / pw);
  if (nw < 1) return -1;                      // does not fit: caller uses the view-major kernel
  if (nw > 8) nw = 8;
  const int nsm = device_sm_count();
  const int nchunk = (nv + 31) / 32;
  int grid = (int)((s.n_act + nw - 1) / nw);
  // a few blocks per SM over all chunks (16 per SM, for a better-balanced
  // last wave, measured slower: 6.4 -> 7.7 ms on the batching workload)
  const int want = (nsm * 4 + nchunk - 1) / nchunk;
  if (grid > want) grid = want;
  if (grid * nw > parts_cap) grid = parts_cap / nw;
  if (grid < 1) grid = 1;
  *nparts = grid * nw;
  const size_t sm = pw * nw;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<dim3(grid, nchunk), 32 * nw, sm, st>>>(s, c, cams, nv, blocks, f, partial, *nparts);
  };
  switch (c.deg) {
    case 0: go(k_gains_gm<0>); break;
    case 1: go(k_gains_gm<1>); break;
    case 2: go(k_gains_gm<2>); break;
    default: go(k_gains_gm<3>); break;
  }
  return 1;
}

int launch_project_backward(const DevScene& s, const Consts& c, const DevCam& cam, const float* gacc, int gw,
                            const int4* rect, float* g_means, float* g_logs, float* g_quats, float* g_rho,
                            float* g_sh, float* g_obj, cudaStream_t st) {
  if (s.n <= 0) return 0;
  k_project_backward<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(s, c, cam, gacc, gw, rect, g_means, g_logs,
                                                                    g_quats, g_rho, g_sh, g_obj);
  return 1;
}

int launch_reduce_gains_views(const double* partial, int nparts, int nv, double* out3, cudaStream_t st) {
  if (nv <= 0) return 0;
  k_reduce_partial<<<nv, 256, 0, st>>>(partial, nparts, out3);
  return 1;
}

int launch_reduce_gains(const double* partial, int nblocks, double* out3, cudaStream_t st) {
  k_reduce_partial<<<1, 256, 0, st>>>(partial, nblocks, out3);
  return 1;
}

int launch_final_scores(const double* ig_cand, const double* ig_train, int n_cand, int n_train,
                        const Consts& c, float* out4, int* best, float* best_score, int* err,
                        cudaStream_t st) {
  k_final_scores<<<1, 32, 0, st>>>(ig_cand, ig_train, n_cand, n_train, c, out4, best, best_score, err);
  return 1;
}

}  // namespace nbv
