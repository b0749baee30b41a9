/*
 * CPU oracle of the object-aware Gaussian-splat next-best-view score.
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only code that may load or call this
 * library. The GPU product path never calls it and shares no code with it.
 *
 * It is plain and slow on purpose: every quantity is computed the way the
 * paper defines it, in double precision, in the paper's order:
 *
 *   object vector      O' = sum_i softmax(o_i) alpha_i T_i             Eq. 1
 *   background residual O = O' + e0 (1 - 1^T O')                       Eq. 2
 *   information gain   IG(T,c) = f(T u c) - f(T), NBV = argmax         Eq. 5
 *   log-det criterion  f(V) = log det(sum_v J_v^T J_v)                 Eq. 6
 *   block diagonal     one l x l block per Gaussian                    Sec. III-B.1
 *   confidence         c_g = max_k(p_gk)^-a_obj sigma_g^-a_opa         Eq. 7
 *                      C_g = c_g I_l,  H := J^T C J                    Eqs. 8-9
 *   per-output scaling IG_f / mean_t IG_f(T,t), f in {rgb,d,o}         Eq. 10
 *   weighted sum       IG_rgb + b_d IG_d + b_o IG_o                    Eq. 11
 *   object-centric     c_g,obj = p_g,obj^-a_obj sigma^-a_opa if
 *                      argmax_k p_gk = obj, else 0                     Eq. 12
 *
 * The rasterizer follows the standard 3D Gaussian Splatting forward pass the
 * paper builds on (Sec. IV-A.2): EWA projection with a 0.3 px dilation,
 * 3-sigma screen radius, tile binning, per-tile depth sort, front-to-back
 * compositing with the 1/255 alpha cut-off, the 0.99 alpha clamp and the
 * 1e-4 transmittance stop.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - C_g scales the parameter-space block: H_g = lambda I + c_g sum_v A_vg,
 *    A_vg = sum_pixels sum_channels J J^T, lambda = damping (config).
 *  - Parameters are the raw ones: mu, log-scale, unnormalised quaternion,
 *    opacity logit, SH coefficients, object logits.
 *  - Depth output D = sum_i w_i z_i (camera-space z, not normalised).
 *  - Pixel centre at (px+0.5, py+0.5).
 *  - Tie-break of the depth sort: (float bits of z, Gaussian index).
 *  - A tile lists every splat whose 3-sigma rectangle covers it (the plain
 *    binning rule of 3D Gaussian Splatting; no culling inside the rectangle).
 *  - Discrete decisions (culling, tile rectangle, alpha cut-off, alpha
 *    clamp, transmittance stop) are taken in single
 *    precision, the precision the GPU kernel works in; every value is
 *    computed in double. The
 *    single-precision decision path uses only correctly rounded + - * / sqrt
 *    in a fixed order, so a GPU that follows the same order reproduces every
 *    decision except the transmittance stop, whose running product also
 *    depends on exp; for that one the oracle reports a per-pixel margin.
 *
 * The Jacobian of the projection is taken by forward-mode dual numbers
 * through the projection itself, so it is the derivative of exactly the
 * function that is rendered.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double c) : v(c) { for (int i = 0; i < N; ++i) d[i] = 0.0; }  // NOLINT
  static Dual var(double c, int i) { Dual r(c); r.d[i] = 1.0; return r; }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> Dual<N> dsqrt(const Dual<N>& a) {
  double s = std::sqrt(a.v); Dual<N> r(s);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * s); return r; }
template <int N> Dual<N> dexp(const Dual<N>& a) {
  double e = std::exp(a.v); Dual<N> r(e);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * e; return r; }
inline double dsqrt(double a) { return std::sqrt(a); }
inline double dexp(double a) { return std::exp(a); }
template <int N> double val(const Dual<N>& a) { return a.v; }
inline double val(double a) { return a; }

constexpr int NG = 11;  // geometric parameters: mu(3) log-scale(3) quaternion(4) opacity logit(1)
using DG = Dual<NG>;

// ------------------------------------------------------------ configuration
struct Hyper {
  float alpha_obj, alpha_opa, beta_d, beta_o, lambda;
  float near_z, alpha_min, alpha_max, t_min, dilation, guard;
  int tile_w, tile_h;
  int crit;   // 0: log det (Eq. 6); 1: tr(H_T^-1 c A_v); 2: tr(c A_v) (T-optimality)
};

struct Cam32 {
  float R[9], t[3], fx, fy, cx, cy;
  int W, H;
};

struct Scene {
  int64_t n;
  int K, deg, nb, target;
  Hyper hp;
  std::vector<float> mu, logs, q, rho, sh, obj;   // raw inputs (float, as given)
  // decision-path (single precision) per-Gaussian values
  std::vector<float> scale32, qn32, sigma32, pw_skip32, pw_clamp32;
  // value-path (double) per-Gaussian values
  std::vector<double> sigma64, p64, conf;
  // training state of orc_prepare: H_T blocks (l x l per Gaussian) and log det H_T
  std::vector<double> H[3], ldH;
  bool prepared = false;
};

// --------------------------------------------------- real spherical harmonics
// Y_lm on the unit sphere written as polynomials in (x,y,z):
//   m = 0 : K_l0 * P_l(z)
//   m > 0 : sqrt2 K_lm (-1)^m (d^m P_l/dz^m)(z) Re (x + i y)^m
//   m < 0 : sqrt2 K_l|m| (-1)^m (d^|m| P_l/dz^|m|)(z) Im (x + i y)^|m|
//   K_lm  = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
// i.e. the real harmonics built from the associated Legendre functions with
// the Condon-Shortley phase. Index k = l*l + l + m.
static std::vector<double> legendre_coeffs(int l) {
  // Bonnet recursion on coefficient arrays: (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}
  std::vector<double> p0{1.0}, p1{0.0, 1.0};
  if (l == 0) return p0;
  for (int n = 1; n < l; ++n) {
    std::vector<double> p2(n + 2, 0.0);
    for (int i = 0; i <= n; ++i) p2[i + 1] += (2.0 * n + 1.0) * p1[i];
    for (int i = 0; i < (int)p0.size(); ++i) p2[i] -= n * p0[i];
    for (auto& c : p2) c /= (n + 1.0);
    p0 = p1; p1 = p2;
  }
  return p1;
}

static double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

template <class S>
void sh_basis(int deg, const S dir[3], S* Y) {
  for (int l = 0; l <= deg; ++l) {
    std::vector<double> P = legendre_coeffs(l);
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      // d^am/dz^am of P
      std::vector<double> Q = P;
      for (int k = 0; k < am; ++k) {
        std::vector<double> dq(Q.size() > 1 ? Q.size() - 1 : 1, 0.0);
        for (size_t i = 1; i < Q.size(); ++i) dq[i - 1] = Q[i] * (double)i;
        Q = dq;
      }
      S qz = S(0.0), zp = S(1.0);
      for (size_t i = 0; i < Q.size(); ++i) { qz = qz + Q[i] * zp; zp = zp * dir[2]; }
      S re = S(1.0), im = S(0.0);
      for (int k = 0; k < am; ++k) {
        S nre = re * dir[0] - im * dir[1];
        S nim = re * dir[1] + im * dir[0];
        re = nre; im = nim;
      }
      double Klm = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - am) / factorial(l + am));
      S y;
      if (m == 0) y = Klm * qz;
      else {
        double sgn = (am % 2) ? -1.0 : 1.0;
        y = (std::sqrt(2.0) * Klm * sgn) * qz * (m > 0 ? re : im);
      }
      Y[l * l + l + m] = y;
    }
  }
}

// --------------------------------------- single-precision decision path (A1)
// Every step is one correctly rounded float operation, in this order.
struct Key32 {
  int valid;
  int x0, x1, y0, y1;
  float radius;
  uint32_t zbits;
  float mx, my, A, B, C;
};

static Key32 key_path32(const Scene& s, int64_t g, const Cam32& c) {
  Key32 k{};
  k.valid = 0;
  const float* m = &s.mu[3 * g];
  const float* sc = &s.scale32[3 * g];
  const float* qn = &s.qn32[4 * g];
  const float* R = c.R;
  float tx = ((R[0] * m[0] + R[1] * m[1]) + R[2] * m[2]) + c.t[0];
  float ty = ((R[3] * m[0] + R[4] * m[1]) + R[5] * m[2]) + c.t[1];
  float tz = ((R[6] * m[0] + R[7] * m[1]) + R[8] * m[2]) + c.t[2];
  if (!(tz > s.hp.near_z)) return k;
  float mx = c.fx * (tx / tz) + c.cx;
  float my = c.fy * (ty / tz) + c.cy;
  float limx = s.hp.guard * ((0.5f * (float)c.W) / c.fx);
  float limy = s.hp.guard * ((0.5f * (float)c.H) / c.fy);
  float xz = std::fmin(limx, std::fmax(-limx, tx / tz));
  float yz = std::fmin(limy, std::fmax(-limy, ty / tz));
  float txp = xz * tz, typ = yz * tz;
  float tz2 = tz * tz;
  float j00 = c.fx / tz, j02 = -((c.fx * txp) / tz2);
  float j11 = c.fy / tz, j12 = -((c.fy * typ) / tz2);
  float T0[3], T1[3];
  for (int i = 0; i < 3; ++i) {
    T0[i] = j00 * R[0 + i] + j02 * R[6 + i];
    T1[i] = j11 * R[3 + i] + j12 * R[6 + i];
  }
  float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  float Rq[9];
  Rq[0] = 1.0f - 2.0f * (y * y + z * z);
  Rq[1] = 2.0f * (x * y - w * z);
  Rq[2] = 2.0f * (x * z + w * y);
  Rq[3] = 2.0f * (x * y + w * z);
  Rq[4] = 1.0f - 2.0f * (x * x + z * z);
  Rq[5] = 2.0f * (y * z - w * x);
  Rq[6] = 2.0f * (x * z - w * y);
  Rq[7] = 2.0f * (y * z + w * x);
  Rq[8] = 1.0f - 2.0f * (x * x + y * y);
  float V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[3 * i + j] = Rq[3 * i + j] * sc[j];
  float Sg[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Sg[3 * i + j] = (V[3 * i + 0] * V[3 * j + 0] + V[3 * i + 1] * V[3 * j + 1]) + V[3 * i + 2] * V[3 * j + 2];
  float U0[3], U1[3];
  for (int j = 0; j < 3; ++j) {
    U0[j] = (T0[0] * Sg[0 + j] + T0[1] * Sg[3 + j]) + T0[2] * Sg[6 + j];
    U1[j] = (T1[0] * Sg[0 + j] + T1[1] * Sg[3 + j]) + T1[2] * Sg[6 + j];
  }
  float a = ((U0[0] * T0[0] + U0[1] * T0[1]) + U0[2] * T0[2]) + s.hp.dilation;
  float b = (U0[0] * T1[0] + U0[1] * T1[1]) + U0[2] * T1[2];
  float cc = ((U1[0] * T1[0] + U1[1] * T1[1]) + U1[2] * T1[2]) + s.hp.dilation;
  float det = a * cc - b * b;
  if (!(det > 0.0f)) return k;
  float A = cc / det, B = -b / det, C = a / det;
  float mid = 0.5f * (a + cc);
  float lam = mid + std::sqrt(std::fmax(0.1f, mid * mid - det));
  float r = std::ceil(3.0f * std::sqrt(lam));
  int GX = (c.W + s.hp.tile_w - 1) / s.hp.tile_w;
  int GY = (c.H + s.hp.tile_h - 1) / s.hp.tile_h;
  float twf = (float)s.hp.tile_w, thf = (float)s.hp.tile_h;
  float fx0 = std::floor((mx - r) / twf), fx1 = std::floor((mx + r) / twf) + 1.0f;
  float fy0 = std::floor((my - r) / thf), fy1 = std::floor((my + r) / thf) + 1.0f;
  int x0 = (int)std::fmin(std::fmax(fx0, 0.0f), (float)GX);
  int x1 = (int)std::fmin(std::fmax(fx1, 0.0f), (float)GX);
  int y0 = (int)std::fmin(std::fmax(fy0, 0.0f), (float)GY);
  int y1 = (int)std::fmin(std::fmax(fy1, 0.0f), (float)GY);
  if (x0 >= x1 || y0 >= y1) return k;
  k.valid = 1;
  k.x0 = x0; k.x1 = x1; k.y0 = y0; k.y1 = y1;
  k.radius = r;
  std::memcpy(&k.zbits, &tz, 4);
  k.mx = mx; k.my = my; k.A = A; k.B = B; k.C = C;
  return k;
}

// The pixel-level decision quantity: the exponent of the splat at a pixel centre.
static inline float power32(const Key32& k, int px, int py) {
  float dx = k.mx - ((float)px + 0.5f);
  float dy = k.my - ((float)py + 0.5f);
  float dxx = dx * dx, dyy = dy * dy, dxy = dx * dy;
  float qf = k.A * dxx + k.C * dyy;
  return (-0.5f * qf) - k.B * dxy;
}

// ----------------------------------------------- double-precision value path
struct CamD {
  double R[9], t[3], fx, fy, cx, cy, campos[3];
  int W, H;
};

static CamD to_camd(const Cam32& c) {
  CamD d;
  for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
  d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.W = c.W; d.H = c.H;
  for (int i = 0; i < 3; ++i)  // camera centre -R^T t
    d.campos[i] = -(d.R[0 + i] * d.t[0] + d.R[3 + i] * d.t[1] + d.R[6 + i] * d.t[2]);
  return d;
}

template <class S>
struct Geo { S mx, my, A, B, C, sigma, z; S dir[3]; };

template <class S>
Geo<S> project_geo(const S mu[3], const S logs[3], const S q[4], const S& rho, const CamD& c,
                   double dilation, double guard) {
  Geo<S> g;
  g.sigma = S(1.0) / (S(1.0) + dexp(-rho));
  S tc[3];
  for (int i = 0; i < 3; ++i) tc[i] = c.R[3 * i] * mu[0] + c.R[3 * i + 1] * mu[1] + c.R[3 * i + 2] * mu[2] + c.t[i];
  g.z = tc[2];
  g.mx = c.fx * tc[0] / tc[2] + c.cx;
  g.my = c.fy * tc[1] / tc[2] + c.cy;
  double limx = guard * 0.5 * c.W / c.fx, limy = guard * 0.5 * c.H / c.fy;
  S xz = tc[0] / tc[2], yz = tc[1] / tc[2];
  if (val(xz) > limx) xz = S(limx);
  if (val(xz) < -limx) xz = S(-limx);
  if (val(yz) > limy) yz = S(limy);
  if (val(yz) < -limy) yz = S(-limy);
  // Jacobian of (fx x/z, fy y/z) at the (guard-band clamped) point
  S j00 = c.fx / tc[2], j02 = -(c.fx * xz) / tc[2];
  S j11 = c.fy / tc[2], j12 = -(c.fy * yz) / tc[2];
  S T0[3], T1[3];
  for (int k = 0; k < 3; ++k) {
    T0[k] = j00 * c.R[k] + j02 * c.R[6 + k];
    T1[k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
  }
  S nrm = dsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
  S Rq[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
             2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
             2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
  S s2[3];
  for (int k = 0; k < 3; ++k) { S e = dexp(logs[k]); s2[k] = e * e; }
  S Sg[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S acc = S(0.0);
      for (int k = 0; k < 3; ++k) acc = acc + Rq[3 * i + k] * s2[k] * Rq[3 * j + k];
      Sg[3 * i + j] = acc;
    }
  S a = S(dilation), b = S(0.0), cc = S(dilation);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a = a + T0[i] * Sg[3 * i + j] * T0[j];
      b = b + T0[i] * Sg[3 * i + j] * T1[j];
      cc = cc + T1[i] * Sg[3 * i + j] * T1[j];
    }
  S det = a * cc - b * b;
  g.A = cc / det;
  g.B = -b / det;
  g.C = a / det;
  S dv[3];
  for (int i = 0; i < 3; ++i) dv[i] = mu[i] - c.campos[i];
  S len = dsqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  for (int i = 0; i < 3; ++i) g.dir[i] = dv[i] / len;
  return g;
}

// Everything the compositing and the Jacobians need about one (view, Gaussian).
struct Rec64 {
  double mx, my, A, B, C, sigma, z, rgb[3];
  double Mgeo[6][NG];   // d{mx,my,A,B,C,z}/d(geo params)
  double dsig;          // d sigma / d rho
  double drgb_dmu[3][3];
  int rgb_live[3];      // 0 where the colour is clamped at 0
  double Y[16];
};

static Rec64 value_path(const Scene& s, int64_t gi, const CamD& c) {
  Rec64 r{};
  DG mu[3], logs[3], q[4], rho;
  for (int i = 0; i < 3; ++i) mu[i] = DG::var(s.mu[3 * gi + i], i);
  for (int i = 0; i < 3; ++i) logs[i] = DG::var(s.logs[3 * gi + i], 3 + i);
  for (int i = 0; i < 4; ++i) q[i] = DG::var(s.q[4 * gi + i], 6 + i);
  rho = DG::var(s.rho[gi], 10);
  Geo<DG> g = project_geo<DG>(mu, logs, q, rho, c, s.hp.dilation, s.hp.guard);
  r.mx = g.mx.v; r.my = g.my.v; r.A = g.A.v; r.B = g.B.v; r.C = g.C.v; r.sigma = g.sigma.v; r.z = g.z.v;
  const DG* rows[6] = {&g.mx, &g.my, &g.A, &g.B, &g.C, &g.z};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < NG; ++j) r.Mgeo[i][j] = rows[i]->d[j];
  r.dsig = g.sigma.d[10];
  DG Y[16];
  sh_basis<DG>(s.deg, g.dir, Y);
  for (int k = 0; k < s.nb; ++k) r.Y[k] = Y[k].v;
  for (int ch = 0; ch < 3; ++ch) {
    DG acc = DG(0.5);
    for (int k = 0; k < s.nb; ++k) acc = acc + Y[k] * (double)s.sh[(gi * s.nb + k) * 3 + ch];
    if (acc.v < 0.0) {
      r.rgb[ch] = 0.0; r.rgb_live[ch] = 0;
      for (int j = 0; j < 3; ++j) r.drgb_dmu[ch][j] = 0.0;
    } else {
      r.rgb[ch] = acc.v; r.rgb_live[ch] = 1;
      for (int j = 0; j < 3; ++j) r.drgb_dmu[ch][j] = acc.d[j];
    }
  }
  return r;
}

// ------------------------------------------------------------ per-view setup
struct ViewData {
  Cam32 c32;
  CamD cd;
  int GX, GY;
  std::vector<Key32> keys;
  std::vector<Rec64> recs;
  std::vector<std::vector<int32_t>> lists;  // per tile, sorted Gaussian ids
};

static void build_view(const Scene& s, const Cam32& c, ViewData& v, bool with_values) {
  v.c32 = c;
  v.cd = to_camd(c);
  v.GX = (c.W + s.hp.tile_w - 1) / s.hp.tile_w;
  v.GY = (c.H + s.hp.tile_h - 1) / s.hp.tile_h;
  v.keys.resize(s.n);
  for (int64_t g = 0; g < s.n; ++g) v.keys[g] = key_path32(s, g, c);
  if (with_values) {
    v.recs.assign(s.n, Rec64{});
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < s.n; ++g)
      if (v.keys[g].valid) v.recs[g] = value_path(s, g, v.cd);
  }
  // tile lists: every Gaussian whose rectangle covers the tile, sorted by
  // (depth bits, Gaussian index)
  v.lists.assign((size_t)v.GX * v.GY, {});
  for (int64_t g = 0; g < s.n; ++g) {
    const Key32& k = v.keys[g];
    if (!k.valid) continue;
    for (int ty = k.y0; ty < k.y1; ++ty)
      for (int tx = k.x0; tx < k.x1; ++tx) v.lists[(size_t)ty * v.GX + tx].push_back((int32_t)g);
  }
  for (auto& L : v.lists)
    std::stable_sort(L.begin(), L.end(), [&](int32_t a, int32_t b) {
      if (v.keys[a].zbits != v.keys[b].zbits) return v.keys[a].zbits < v.keys[b].zbits;
      return a < b;
    });
}

// ------------------------------------------------ compositing one pixel (A3)
struct Step { int32_t g; double alpha, T; int clamped; };

struct PixelOut {
  double rgb[3], depth, alpha;
  std::vector<double> obj;
  int n_contrib;      // list entries up to and including the last blended one
  float margin;       // min relative distance of T(1-a) to the stop threshold
  std::vector<Step> steps;
};

static void composite_pixel(const Scene& s, const ViewData& v, int px, int py, PixelOut& o) {
  const int KC = s.K + 1;
  const auto& L = v.lists[(size_t)(py / s.hp.tile_h) * v.GX + (px / s.hp.tile_w)];
  o.rgb[0] = o.rgb[1] = o.rgb[2] = 0.0;
  o.depth = 0.0;
  o.obj.assign(KC, 0.0);
  o.steps.clear();
  o.n_contrib = 0;
  o.margin = 1e30f;
  float T32 = 1.0f;
  double T = 1.0;
  for (size_t idx = 0; idx < L.size(); ++idx) {
    const int32_t g = L[idx];
    const Key32& k = v.keys[g];
    // decisions, single precision
    float pw = power32(k, px, py);
    if (pw > 0.0f) continue;
    if (pw < s.pw_skip32[g]) continue;
    int clamped = pw >= s.pw_clamp32[g];
    float a32 = clamped ? s.hp.alpha_max : s.sigma32[g] * (float)std::exp((double)pw);
    float testT32 = T32 * (1.0f - a32);
    float mg = std::fabs(testT32 - s.hp.t_min) / s.hp.t_min;
    o.margin = std::min(o.margin, mg);
    if (testT32 < s.hp.t_min) break;
    // values, double precision
    const Rec64& r = v.recs[g];
    double dx = r.mx - (px + 0.5), dy = r.my - (py + 0.5);
    double power = -0.5 * (r.A * dx * dx + r.C * dy * dy) - r.B * dx * dy;
    double alpha = clamped ? (double)s.hp.alpha_max : r.sigma * std::exp(power);
    double w = alpha * T;
    for (int ch = 0; ch < 3; ++ch) o.rgb[ch] += w * r.rgb[ch];
    o.depth += w * r.z;
    for (int kk = 0; kk < KC; ++kk) o.obj[kk] += w * s.p64[(size_t)g * KC + kk];     // Eq. 1
    o.steps.push_back(Step{g, alpha, T, clamped});
    T *= (1.0 - alpha);
    T32 = testT32;
    o.n_contrib = (int)idx + 1;
  }
  o.alpha = 1.0 - T;
  double sum = 0.0;
  for (int kk = 0; kk < KC; ++kk) sum += o.obj[kk];
  o.obj[0] += 1.0 - sum;                                                          // Eq. 2
}

// ------------------------------------ Jacobian blocks of one view (Eqs. 6, 9)
// A^f_g += J J^T over every pixel and every channel of output f, with
// J = d out / d theta_g, theta_g the raw parameters the output depends on:
//   rgb: [mu, log s, q, rho, sh (nb x 3, [k][ch])]      l = 11 + 3 nb
//   d  : [mu, log s, q, rho]                            l = 11
//   o  : [mu, log s, q, rho, o (K+1)]                   l = 12 + K
struct Blocks {
  int lr, ld, lo;
  std::vector<int64_t> slot;   // Gaussian -> block index or -1
  std::vector<double> Ar, Ad, Ao;
};

static void accumulate_view_blocks(const Scene& s, const ViewData& v, Blocks& B,
                                   std::vector<float>* margins, int row_stride = 1) {
  const int KC = s.K + 1, nb = s.nb;
  const int lr = B.lr, ld = B.ld, lo = B.lo;
  const int ur = 9, ud = 7, uo = 6 + KC;
  std::vector<omp_lock_t> locks;
#ifdef _OPENMP
  locks.resize(s.n);
  for (auto& l : locks) omp_init_lock(&l);
#endif
  const int W = v.c32.W, H = v.c32.H;
#pragma omp parallel
  {
    PixelOut o;
    std::vector<double> Mr(ur * lr), Md(ud * ld), Mo(uo * lo), gu(uo), J(std::max(lr, lo));
    std::vector<double> Rrgb(3), Ro(KC);
#pragma omp for schedule(dynamic, 1)
    for (int py = 0; py < H; py += row_stride) {
      for (int px = 0; px < W; ++px) {
        composite_pixel(s, v, px, py, o);
        if (margins) (*margins)[(size_t)py * W + px] = o.margin;
        // suffix sums R_i = sum_{j>i} w_j x_j, built back to front
        double Rd = 0.0, RA = 0.0;
        for (int ch = 0; ch < 3; ++ch) Rrgb[ch] = 0.0;
        for (int kk = 0; kk < KC; ++kk) Ro[kk] = 0.0;
        for (int i = (int)o.steps.size() - 1; i >= 0; --i) {
          const Step& st = o.steps[i];
          const int64_t g = st.g;
          const Rec64& r = v.recs[g];
          const double* p = &s.p64[(size_t)g * KC];
          const double w = st.alpha * st.T, om = 1.0 - st.alpha;
          // d out / d alpha_i = T_i x_i - R_i / (1 - alpha_i)
          double s_rgb[3], s_d, s_A;
          std::vector<double> s_o(KC);
          for (int ch = 0; ch < 3; ++ch) s_rgb[ch] = st.T * r.rgb[ch] - Rrgb[ch] / om;
          s_d = st.T * r.z - Rd / om;
          s_A = st.T - RA / om;
          for (int kk = 0; kk < KC; ++kk) s_o[kk] = st.T * p[kk] - Ro[kk] / om;
          s_o[0] -= s_A;  // O_0 = O'_0 + 1 - sum_k O'_k
          // d alpha / d (mx, my, A, B, C, sigma); zero when alpha is clamped
          double da[6] = {0, 0, 0, 0, 0, 0};
          if (!st.clamped) {
            double dx = r.mx - (px + 0.5), dy = r.my - (py + 0.5);
            da[0] = st.alpha * (-(r.A * dx + r.B * dy));
            da[1] = st.alpha * (-(r.B * dx + r.C * dy));
            da[2] = st.alpha * (-0.5 * dx * dx);
            da[3] = st.alpha * (-dx * dy);
            da[4] = st.alpha * (-0.5 * dy * dy);
            da[5] = st.alpha / r.sigma;
          }
          // M = d u / d theta for each output
          std::fill(Mr.begin(), Mr.end(), 0.0);
          std::fill(Md.begin(), Md.end(), 0.0);
          std::fill(Mo.begin(), Mo.end(), 0.0);
          for (int row = 0; row < 5; ++row)
            for (int j = 0; j < NG; ++j) {
              Mr[row * lr + j] = r.Mgeo[row][j];
              Md[row * ld + j] = r.Mgeo[row][j];
              Mo[row * lo + j] = r.Mgeo[row][j];
            }
          Mr[5 * lr + 10] = r.dsig; Md[5 * ld + 10] = r.dsig; Mo[5 * lo + 10] = r.dsig;
          for (int ch = 0; ch < 3; ++ch) {
            if (!r.rgb_live[ch]) continue;
            for (int j = 0; j < 3; ++j) Mr[(6 + ch) * lr + j] = r.drgb_dmu[ch][j];
            for (int kk = 0; kk < nb; ++kk) Mr[(6 + ch) * lr + NG + kk * 3 + ch] = r.Y[kk];
          }
          for (int j = 0; j < NG; ++j) Md[6 * ld + j] = r.Mgeo[5][j];
          for (int a = 0; a < KC; ++a)           // softmax Jacobian diag(p) - p p^T
            for (int b = 0; b < KC; ++b)
              Mo[(6 + a) * lo + NG + b] = (a == b ? p[a] : 0.0) - p[a] * p[b];
          const int64_t sl = B.slot[g];
          if (sl >= 0) {
#ifdef _OPENMP
            omp_set_lock(&locks[g]);
#endif
            // rgb: three channels, u = [mx,my,A,B,C,sigma,r,g,b]
            double* Ar = &B.Ar[(size_t)sl * lr * lr];
            for (int ch = 0; ch < 3; ++ch) {
              for (int u = 0; u < ur; ++u) gu[u] = 0.0;
              for (int u = 0; u < 6; ++u) gu[u] = s_rgb[ch] * da[u];
              gu[6 + ch] = w;
              for (int j = 0; j < lr; ++j) {
                double acc = 0.0;
                for (int u = 0; u < ur; ++u) acc += gu[u] * Mr[u * lr + j];
                J[j] = acc;
              }
              for (int i2 = 0; i2 < lr; ++i2)
                for (int j = 0; j <= i2; ++j) Ar[i2 * lr + j] += J[i2] * J[j];
            }
            // depth: u = [mx,my,A,B,C,sigma,z]
            double* Ad = &B.Ad[(size_t)sl * ld * ld];
            for (int u = 0; u < 6; ++u) gu[u] = s_d * da[u];
            gu[6] = w;
            for (int j = 0; j < ld; ++j) {
              double acc = 0.0;
              for (int u = 0; u < ud; ++u) acc += gu[u] * Md[u * ld + j];
              J[j] = acc;
            }
            for (int i2 = 0; i2 < ld; ++i2)
              for (int j = 0; j <= i2; ++j) Ad[i2 * ld + j] += J[i2] * J[j];
            // objects: K+1 channels, u = [mx,my,A,B,C,sigma,p_0..p_K]
            double* Ao = &B.Ao[(size_t)sl * lo * lo];
            for (int kk = 0; kk < KC; ++kk) {
              for (int u = 0; u < 6; ++u) gu[u] = s_o[kk] * da[u];
              for (int b = 0; b < KC; ++b) {
                double d = (b == kk) ? w : 0.0;     // d O'_k / d p_b
                if (kk == 0) d -= w;                 // residual into channel 0
                gu[6 + b] = d;
              }
              for (int j = 0; j < lo; ++j) {
                double acc = 0.0;
                for (int u = 0; u < uo; ++u) acc += gu[u] * Mo[u * lo + j];
                J[j] = acc;
              }
              for (int i2 = 0; i2 < lo; ++i2)
                for (int j = 0; j <= i2; ++j) Ao[i2 * lo + j] += J[i2] * J[j];
            }
#ifdef _OPENMP
            omp_unset_lock(&locks[g]);
#endif
          }
          // extend the suffix sums with entry i
          for (int ch = 0; ch < 3; ++ch) Rrgb[ch] += w * r.rgb[ch];
          Rd += w * r.z;
          RA += w;
          for (int kk = 0; kk < KC; ++kk) Ro[kk] += w * p[kk];
        }
      }
    }
  }
#ifdef _OPENMP
  for (auto& l : locks) omp_destroy_lock(&l);
#endif
}

static void symmetrize(std::vector<double>& A, int64_t nblk, int l) {
  for (int64_t b = 0; b < nblk; ++b) {
    double* M = &A[(size_t)b * l * l];
    for (int i = 0; i < l; ++i)
      for (int j = i + 1; j < l; ++j) M[i * l + j] = M[j * l + i];
  }
}

// log det of a symmetric positive definite matrix by the Cholesky factorisation
static double logdet_spd(std::vector<double>& M, int l) {
  double ld = 0.0;
  for (int j = 0; j < l; ++j) {
    double d = M[j * l + j];
    for (int k = 0; k < j; ++k) d -= M[j * l + k] * M[j * l + k];
    if (!(d > 0.0)) return std::nan("");
    double L = std::sqrt(d);
    M[j * l + j] = L;
    ld += 2.0 * std::log(L);
    for (int i = j + 1; i < l; ++i) {
      double x = M[i * l + j];
      for (int k = 0; k < j; ++k) x -= M[i * l + k] * M[j * l + k];
      M[i * l + j] = x / L;
    }
  }
  return ld;
}

static Cam32 read_cam(const float* cam, const int* wh) {
  Cam32 c;
  for (int i = 0; i < 9; ++i) c.R[i] = cam[i];
  for (int i = 0; i < 3; ++i) c.t[i] = cam[9 + i];
  c.fx = cam[12]; c.fy = cam[13]; c.cx = cam[14]; c.cy = cam[15];
  c.W = wh[0]; c.H = wh[1];
  return c;
}

static void alloc_blocks(const Scene& s, Blocks& B, const uint8_t* mask) {
  B.lr = NG + 3 * s.nb; B.ld = NG; B.lo = NG + s.K + 1;
  B.slot.assign(s.n, -1);
  int64_t m = 0;
  for (int64_t g = 0; g < s.n; ++g)
    if (!mask || mask[g]) B.slot[g] = m++;
  B.Ar.assign((size_t)m * B.lr * B.lr, 0.0);
  B.Ad.assign((size_t)m * B.ld * B.ld, 0.0);
  B.Ao.assign((size_t)m * B.lo * B.lo, 0.0);
}

}  // namespace

// ============================================================== C interface
extern "C" {

// Scene set-up (A0). hp = {alpha_obj, alpha_opa, beta_d, beta_o, lambda, near,
// alpha_min, alpha_max, t_min, dilation, guard, tile_w, tile_h, criterion}.
void* orc_scene_create(int64_t n, int K, int sh_degree, const float* means, const float* log_scales,
                       const float* quats, const float* opacity, const float* sh, const float* obj,
                       const float* hp, int target) {
  Scene* s = new Scene();
  s->n = n; s->K = K; s->deg = sh_degree; s->nb = (sh_degree + 1) * (sh_degree + 1); s->target = target;
  s->hp = Hyper{hp[0], hp[1], hp[2], hp[3], hp[4], hp[5], hp[6], hp[7], hp[8], hp[9], hp[10],
                (int)hp[11], (int)hp[12], (int)hp[13]};
  const int KC = K + 1;
  s->mu.assign(means, means + 3 * n);
  s->logs.assign(log_scales, log_scales + 3 * n);
  s->q.assign(quats, quats + 4 * n);
  s->rho.assign(opacity, opacity + n);
  s->sh.assign(sh, sh + (size_t)n * s->nb * 3);
  s->obj.assign(obj, obj + (size_t)n * KC);
  s->scale32.resize(3 * n); s->qn32.resize(4 * n); s->sigma32.resize(n);
  s->pw_skip32.resize(n); s->pw_clamp32.resize(n);
  s->sigma64.resize(n); s->p64.resize((size_t)n * KC); s->conf.resize(n);
  for (int64_t g = 0; g < n; ++g) {
    for (int k = 0; k < 3; ++k) s->scale32[3 * g + k] = (float)std::exp((double)log_scales[3 * g + k]);
    const float* q = &quats[4 * g];
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    float nr = std::sqrt(n2);
    for (int k = 0; k < 4; ++k) s->qn32[4 * g + k] = q[k] / nr;
    double sig = 1.0 / (1.0 + std::exp(-(double)opacity[g]));
    s->sigma64[g] = sig;
    float sig32 = (float)sig;
    s->sigma32[g] = sig32;
    // alpha = sigma exp(power) < alpha_min  <=>  power < log(alpha_min / sigma)
    s->pw_skip32[g] = (float)std::log((double)s->hp.alpha_min / (double)sig32);
    s->pw_clamp32[g] = (float)std::log((double)s->hp.alpha_max / (double)sig32);
    // p = softmax(o)
    const float* o = &obj[(size_t)g * KC];
    double mx = o[0];
    int am = 0;
    for (int k = 1; k < KC; ++k) if (o[k] > o[am]) am = k;
    for (int k = 1; k < KC; ++k) mx = std::max(mx, (double)o[k]);
    double z = 0.0;
    for (int k = 0; k < KC; ++k) z += std::exp((double)o[k] - mx);
    double pmax = 0.0;
    for (int k = 0; k < KC; ++k) {
      double p = std::exp((double)o[k] - mx) / z;
      s->p64[(size_t)g * KC + k] = p;
      pmax = std::max(pmax, p);
    }
    // confidence, Eq. 7 (whole scene) or Eq. 12 (target object)
    double cg;
    if (target < 0) {
      cg = std::pow(pmax, -(double)s->hp.alpha_obj) * std::pow(sig, -(double)s->hp.alpha_opa);
    } else {
      cg = (am == target) ? std::pow(s->p64[(size_t)g * KC + target], -(double)s->hp.alpha_obj) *
                                std::pow(sig, -(double)s->hp.alpha_opa)
                          : 0.0;
    }
    s->conf[g] = cg;
  }
  return s;
}

void orc_scene_destroy(void* h) { delete static_cast<Scene*>(h); }

void orc_confidence(void* h, double* out) {
  Scene* s = static_cast<Scene*>(h);
  std::memcpy(out, s->conf.data(), sizeof(double) * s->n);
}

// Single-precision decision path of one view: rect [x0,x1)x[y0,y1) (all -1
// when culled), radius, depth bits, mean2D and conic.
void orc_project32(void* h, const float* cam, const int* wh, int32_t* rect, float* radius,
                   uint32_t* zbits, float* mean2d, float* conic) {
  Scene* s = static_cast<Scene*>(h);
  Cam32 c = read_cam(cam, wh);
  for (int64_t g = 0; g < s->n; ++g) {
    Key32 k = key_path32(*s, g, c);
    if (!k.valid) {
      rect[4 * g] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = -1;
      radius[g] = 0.0f; zbits[g] = 0; mean2d[2 * g] = mean2d[2 * g + 1] = 0.0f;
      conic[3 * g] = conic[3 * g + 1] = conic[3 * g + 2] = 0.0f;
      continue;
    }
    rect[4 * g] = k.x0; rect[4 * g + 1] = k.x1; rect[4 * g + 2] = k.y0; rect[4 * g + 3] = k.y1;
    radius[g] = k.radius; zbits[g] = k.zbits;
    mean2d[2 * g] = k.mx; mean2d[2 * g + 1] = k.my;
    conic[3 * g] = k.A; conic[3 * g + 1] = k.B; conic[3 * g + 2] = k.C;
  }
}

// Double-precision projected values: per Gaussian {mx,my,A,B,C,sigma,z,r,g,b}.
void orc_project64(void* h, const float* cam, const int* wh, double* vals) {
  Scene* s = static_cast<Scene*>(h);
  Cam32 c = read_cam(cam, wh);
  CamD cd = to_camd(c);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t g = 0; g < s->n; ++g) {
    Rec64 r = value_path(*s, g, cd);
    double* o = &vals[10 * g];
    o[0] = r.mx; o[1] = r.my; o[2] = r.A; o[3] = r.B; o[4] = r.C; o[5] = r.sigma; o[6] = r.z;
    o[7] = r.rgb[0]; o[8] = r.rgb[1]; o[9] = r.rgb[2];
  }
}

// Tile lists of one view: offsets[t]..offsets[t+1] index ids[]. Returns the
// total entry count; writes ids only if it fits in cap.
int64_t orc_tile_lists(void* h, const float* cam, const int* wh, int64_t* offsets, int32_t* ids,
                       int64_t cap) {
  Scene* s = static_cast<Scene*>(h);
  ViewData v;
  build_view(*s, read_cam(cam, wh), v, false);
  int64_t tot = 0;
  for (size_t t = 0; t < v.lists.size(); ++t) { offsets[t] = tot; tot += (int64_t)v.lists[t].size(); }
  offsets[v.lists.size()] = tot;
  if (tot <= cap) {
    int64_t o = 0;
    for (auto& L : v.lists) for (int32_t g : L) ids[o++] = g;
  }
  return tot;
}

// The splats of each tile's list that some image pixel of the tile cannot
// skip: those with 1/255-cut-off exponent thr <= power <= 0 (the skip test of
// compositing, single precision) at one of the tile's pixel centres inside
// the image. A list that drops others changes no pixel. Same layout as
// orc_tile_lists (offsets [ntiles + 1], ids in list order); returns the total.
int64_t orc_tile_needed(void* h, const float* cam, const int* wh, int64_t* offsets, int32_t* ids, int64_t cap) {
  Scene* s = static_cast<Scene*>(h);
  Cam32 c = read_cam(cam, wh);
  ViewData v;
  build_view(*s, c, v, false);
  const int TW = s->hp.tile_w, TH = s->hp.tile_h;
  std::vector<std::vector<int32_t>> need(v.lists.size());
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < (int64_t)v.lists.size(); ++t) {
    const int tx = (int)(t % v.GX), ty = (int)(t / v.GX);
    for (int32_t g : v.lists[t]) {
      const Key32& k = v.keys[g];
      bool pass = false;
      for (int py = ty * TH; py < std::min((ty + 1) * TH, c.H) && !pass; ++py)
        for (int px = tx * TW; px < std::min((tx + 1) * TW, c.W); ++px) {
          const float pw = power32(k, px, py);
          if (!(pw > 0.0f) && !(pw < s->pw_skip32[g])) { pass = true; break; }
        }
      if (pass) need[t].push_back(g);
    }
  }
  int64_t tot = 0;
  for (size_t t = 0; t < need.size(); ++t) { offsets[t] = tot; tot += (int64_t)need[t].size(); }
  offsets[need.size()] = tot;
  if (tot <= cap) {
    int64_t o = 0;
    for (auto& L : need) for (int32_t g : L) ids[o++] = g;
  }
  return tot;
}

// Render one view in double precision. obj is [H][W][K+1]; n_contrib and
// margin are per pixel.
void orc_render(void* h, const float* cam, const int* wh, double* rgb, double* depth, double* alpha,
                double* obj, int32_t* n_contrib, float* margin) {
  Scene* s = static_cast<Scene*>(h);
  ViewData v;
  build_view(*s, read_cam(cam, wh), v, true);
  const int KC = s->K + 1, W = wh[0], H = wh[1];
#pragma omp parallel
  {
    PixelOut o;
#pragma omp for schedule(dynamic, 4)
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        composite_pixel(*s, v, px, py, o);
        size_t i = (size_t)py * W + px;
        for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = o.rgb[ch];
        depth[i] = o.depth; alpha[i] = o.alpha;
        for (int k = 0; k < KC; ++k) obj[i * KC + k] = o.obj[k];
        n_contrib[i] = o.n_contrib; margin[i] = o.margin;
      }
  }
}

// Per Gaussian, the sum over the view's pixels of w^2 = (alpha T)^2 of its
// blended splats (how strongly the view observes it).
void orc_view_w2(void* h, const float* cam, const int* wh, double* w2) {
  Scene* s = static_cast<Scene*>(h);
  ViewData v;
  build_view(*s, read_cam(cam, wh), v, true);
  const int W = wh[0], H = wh[1];
  for (int64_t g = 0; g < s->n; ++g) w2[g] = 0.0;
#pragma omp parallel
  {
    PixelOut o;
    std::vector<double> acc(s->n, 0.0);
#pragma omp for schedule(dynamic, 4)
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        composite_pixel(*s, v, px, py, o);
        for (const Step& st : o.steps) {
          const double w = st.alpha * st.T;
          acc[st.g] += w * w;
        }
      }
#pragma omp critical
    for (int64_t g = 0; g < s->n; ++g) w2[g] += acc[g];
  }
}

// Jacobian blocks A^f_g of one view for the Gaussians with mask[g] != 0
// (mask may be NULL for all), written densely in the order of g.
void orc_view_blocks(void* h, const float* cam, const int* wh, const uint8_t* mask, double* Ar,
                     double* Ad, double* Ao) {
  Scene* s = static_cast<Scene*>(h);
  ViewData v;
  build_view(*s, read_cam(cam, wh), v, true);
  Blocks B;
  alloc_blocks(*s, B, mask);
  accumulate_view_blocks(*s, v, B, nullptr);
  int64_t m = (int64_t)(B.Ad.size() / (B.ld * B.ld));
  symmetrize(B.Ar, m, B.lr); symmetrize(B.Ad, m, B.ld); symmetrize(B.Ao, m, B.lo);
  std::memcpy(Ar, B.Ar.data(), B.Ar.size() * sizeof(double));
  std::memcpy(Ad, B.Ad.data(), B.Ad.size() * sizeof(double));
  std::memcpy(Ao, B.Ao.data(), B.Ao.size() * sizeof(double));
}

// Training state (Eqs. 6, 9): H_T,g = lambda I + c_g sum_t A_t,g and its log
// det, for every Gaussian and output. Returns 0, or -2 if a block is not
// positive definite. row_stride > 1 keeps every row_stride-th pixel row only
// (a bounded sample for timing; 1 = the definition).
static int prepare_state(Scene* s, int n_train, const float* tcams, const int* twh, int row_stride) {
  Blocks HB;
  alloc_blocks(*s, HB, nullptr);
  const int ls[3] = {HB.lr, HB.ld, HB.lo};
  for (int t = 0; t < n_train; ++t) {
    ViewData v;
    build_view(*s, read_cam(tcams + 16 * t, twh + 2 * t), v, true);
    accumulate_view_blocks(*s, v, HB, nullptr, row_stride);
  }
  std::vector<double>* Hs[3] = {&HB.Ar, &HB.Ad, &HB.Ao};
  for (int f = 0; f < 3; ++f) symmetrize(*Hs[f], s->n, ls[f]);
  for (int f = 0; f < 3; ++f) {
    const int l = ls[f];
    for (int64_t g = 0; g < s->n; ++g) {
      double* M = &(*Hs[f])[(size_t)g * l * l];
      for (int i = 0; i < l * l; ++i) M[i] *= s->conf[g];
      for (int i = 0; i < l; ++i) M[i * l + i] += (double)s->hp.lambda;
    }
  }
  s->ldH.assign((size_t)s->n * 3, 0.0);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
  for (int64_t g = 0; g < s->n; ++g)
    for (int f = 0; f < 3; ++f) {
      const int l = ls[f];
      std::vector<double> M((*Hs[f]).begin() + (size_t)g * l * l, (*Hs[f]).begin() + (size_t)(g + 1) * l * l);
      s->ldH[3 * g + f] = logdet_spd(M, l);
      if (std::isnan(s->ldH[3 * g + f])) bad++;
    }
  for (int f = 0; f < 3; ++f) s->H[f].swap(*Hs[f]);
  s->prepared = (bad == 0);
  return bad ? -2 : 0;
}

// trace(H^-1 A) for symmetric positive definite H (l x l): H = L L^T by
// Cholesky, X = L^-1 A L^-T by two triangular solves, trace of X.
static double trace_solve(const double* Hg, const double* A, int l) {
  std::vector<double> L(Hg, Hg + (size_t)l * l), Y((size_t)l * l);
  logdet_spd(L, l);                                   // leaves the factor in the lower triangle
  // Y = L^-1 A (column by column)
  for (int c = 0; c < l; ++c)
    for (int i = 0; i < l; ++i) {
      double x = A[i * l + c];
      for (int k = 0; k < i; ++k) x -= L[i * l + k] * Y[k * l + c];
      Y[i * l + c] = x / L[i * l + i];
    }
  // trace(L^-1 A L^-T) = sum_i (L^-1 Y^T)_ii with Y^T = A L^-T ... = sum over i of row i of
  // L^-1 applied to column i of Y^T: solve L z = (row i of Y)^T and take z_i
  double tr = 0.0;
  std::vector<double> z(l);
  for (int i = 0; i < l; ++i) {
    for (int r = 0; r < l; ++r) {
      double x = Y[i * l + r];
      for (int k = 0; k < r; ++k) x -= L[r * l + k] * z[k];
      z[r] = x / L[r * l + r];
    }
    tr += z[i];
  }
  return tr;
}

// IG_f(T, v) = sum_g [log det(H_T,g + c_g A_v,g) - log det H_T,g] (Eqs. 5, 6, 9),
// or, for the criterion variants, sum_g tr(H_T,g^-1 c_g A_v,g) (the first-order
// term of that log det: an expected-information criterion in the manner of
// FisherRF) or sum_g tr(c_g A_v,g) (T-optimality).
static int score_view(Scene* s, const Cam32& c, double* out3, double* dg, int row_stride) {
  const int ls[3] = {NG + 3 * s->nb, NG, NG + s->K + 1};
  ViewData v;
  build_view(*s, c, v, true);
  Blocks AB;
  alloc_blocks(*s, AB, nullptr);
  accumulate_view_blocks(*s, v, AB, nullptr, row_stride);
  std::vector<double>* As[3] = {&AB.Ar, &AB.Ad, &AB.Ao};
  for (int f = 0; f < 3; ++f) symmetrize(*As[f], s->n, ls[f]);
  std::vector<double> dl((size_t)s->n * 3, 0.0);
  int nbad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : nbad)
  for (int64_t g = 0; g < s->n; ++g)
    for (int f = 0; f < 3; ++f) {
      const int l = ls[f];
      const double* A = &(*As[f])[(size_t)g * l * l];
      bool zero = true;
      for (int i = 0; i < l * l && zero; ++i) zero = (A[i] == 0.0);
      if (zero || s->conf[g] == 0.0) { dl[3 * g + f] = 0.0; continue; }
      if (s->hp.crit == 2) {
        double tr = 0.0;
        for (int i = 0; i < l; ++i) tr += A[i * l + i];
        dl[3 * g + f] = s->conf[g] * tr;
        continue;
      }
      if (s->hp.crit == 1) {
        dl[3 * g + f] = s->conf[g] * trace_solve(&s->H[f][(size_t)g * l * l], A, l);
        continue;
      }
      std::vector<double> M(s->H[f].begin() + (size_t)g * l * l, s->H[f].begin() + (size_t)(g + 1) * l * l);
      for (int i = 0; i < l * l; ++i) M[i] += s->conf[g] * A[i];
      double ld = logdet_spd(M, l);
      if (std::isnan(ld)) nbad++;
      dl[3 * g + f] = ld - s->ldH[3 * g + f];
    }
  for (int f = 0; f < 3; ++f) {
    double acc = 0.0;
    for (int64_t g = 0; g < s->n; ++g) acc += dl[3 * g + f];
    out3[f] = acc;
  }
  if (dg) std::memcpy(dg, dl.data(), dl.size() * sizeof(double));
  return nbad ? -2 : 0;
}

// Build and keep the training state (see prepare_state).
int orc_prepare(void* h, int n_train, const float* tcams, const int* twh, int row_stride) {
  return prepare_state(static_cast<Scene*>(h), n_train, tcams, twh, row_stride < 1 ? 1 : row_stride);
}

// Raw gains of n views against the kept training state: ig [n][3].
int orc_score_views(void* h, int n, const float* cams, const int* wh, double* ig, int row_stride) {
  Scene* s = static_cast<Scene*>(h);
  if (!s->prepared) return -3;
  for (int i = 0; i < n; ++i)
    if (score_view(s, read_cam(cams + 16 * i, wh + 2 * i), &ig[3 * i], nullptr, row_stride < 1 ? 1 : row_stride))
      return -2;
  return 0;
}

// The whole score (Eqs. 5-12): training views build H_T; every training view
// and every candidate is scored; scores are normalised per output by the
// training mean and weighted. ig_train [n_train][3], ig_cand [n_cand][3],
// score [n_cand]. If delta != NULL it receives the per-Gaussian log-det
// gains [n][3] of candidate `dv`. Returns the argmax candidate (lowest index
// on ties), -1 if a normaliser is zero, -2 if a block is not positive definite.
int orc_score(void* h, int n_train, const float* tcams, const int* twh, int n_cand,
              const float* ccams, const int* cwh, double* ig_train, double* ig_cand, double* score,
              double* delta, int dv) {
  Scene* s = static_cast<Scene*>(h);
  if (prepare_state(s, n_train, tcams, twh, 1)) return -2;
  for (int t = 0; t < n_train; ++t)
    if (score_view(s, read_cam(tcams + 16 * t, twh + 2 * t), &ig_train[3 * t], nullptr, 1)) return -2;
  double norm[3] = {0, 0, 0};
  for (int f = 0; f < 3; ++f) {
    for (int t = 0; t < n_train; ++t) norm[f] += ig_train[3 * t + f];
    norm[f] /= n_train;
  }
  for (int c = 0; c < n_cand; ++c)
    if (score_view(s, read_cam(ccams + 16 * c, cwh + 2 * c), &ig_cand[3 * c], (delta && c == dv) ? delta : nullptr, 1))
      return -2;
  if (norm[0] == 0.0 || norm[1] == 0.0 || norm[2] == 0.0) {
    for (int c = 0; c < n_cand; ++c) score[c] = std::nan("");
    return -1;
  }
  const double bd = s->hp.beta_d, bo = s->hp.beta_o;
  int best = -1;
  for (int c = 0; c < n_cand; ++c) {
    score[c] = ig_cand[3 * c] / norm[0] + bd * ig_cand[3 * c + 1] / norm[1] + bo * ig_cand[3 * c + 2] / norm[2];
    if (best < 0 || score[c] > score[best]) best = c;
  }
  return best;
}

// Test support for finite differences: record, for every pixel of one view,
// which Gaussians were blended and whether each was clamped; then render
// another (perturbed) scene with exactly those discrete decisions, so that
// central differences see only the smooth part the Jacobian describes.
struct Frozen {
  int W, H;
  std::vector<std::vector<std::pair<int32_t, int>>> steps;
};

void* orc_freeze(void* h, const float* cam, const int* wh) {
  Scene* s = static_cast<Scene*>(h);
  ViewData v;
  build_view(*s, read_cam(cam, wh), v, true);
  Frozen* fz = new Frozen();
  fz->W = wh[0]; fz->H = wh[1];
  fz->steps.resize((size_t)fz->W * fz->H);
  PixelOut o;
  for (int py = 0; py < fz->H; ++py)
    for (int px = 0; px < fz->W; ++px) {
      composite_pixel(*s, v, px, py, o);
      auto& st = fz->steps[(size_t)py * fz->W + px];
      for (const Step& x : o.steps) st.emplace_back(x.g, x.clamped);
    }
  return fz;
}

void orc_frozen_destroy(void* f) { delete static_cast<Frozen*>(f); }

void orc_render_frozen(void* h, void* f, const float* cam, const int* wh, double* rgb, double* depth,
                       double* alpha, double* obj) {
  Scene* s = static_cast<Scene*>(h);
  Frozen* fz = static_cast<Frozen*>(f);
  CamD cd = to_camd(read_cam(cam, wh));
  const int KC = s->K + 1;
  std::vector<Rec64> recs(s->n);
  for (int64_t g = 0; g < s->n; ++g) recs[g] = value_path(*s, g, cd);
  for (int py = 0; py < fz->H; ++py)
    for (int px = 0; px < fz->W; ++px) {
      size_t i = (size_t)py * fz->W + px;
      double T = 1.0, c3[3] = {0, 0, 0}, d = 0.0;
      std::vector<double> ob(KC, 0.0);
      for (auto& st : fz->steps[i]) {
        const Rec64& r = recs[st.first];
        double dx = r.mx - (px + 0.5), dy = r.my - (py + 0.5);
        double power = -0.5 * (r.A * dx * dx + r.C * dy * dy) - r.B * dx * dy;
        double a = st.second ? (double)s->hp.alpha_max : r.sigma * std::exp(power);
        double w = a * T;
        for (int ch = 0; ch < 3; ++ch) c3[ch] += w * r.rgb[ch];
        d += w * r.z;
        for (int k = 0; k < KC; ++k) ob[k] += w * s->p64[(size_t)st.first * KC + k];
        T *= 1.0 - a;
      }
      double sum = 0.0;
      for (int k = 0; k < KC; ++k) sum += ob[k];
      ob[0] += 1.0 - sum;
      for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = c3[ch];
      depth[i] = d; alpha[i] = 1.0 - T;
      for (int k = 0; k < KC; ++k) obj[i * KC + k] = ob[k];
    }
}

// Real spherical harmonics at unit directions, for tests: Y [n][(deg+1)^2].
void orc_sh_basis(int deg, int64_t n, const double* dirs, double* Y) {
  const int nb = (deg + 1) * (deg + 1);
  for (int64_t i = 0; i < n; ++i) sh_basis<double>(deg, &dirs[3 * i], &Y[(size_t)i * nb]);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
