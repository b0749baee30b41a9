// Host checks of the float-float arithmetic in csrc/df64.cuh (built by
// tests/test_df64.py with g++ -ffp-contract=off). Prints one "name value"
// line per measured quantity; the Python side holds the bounds.
//
// References are computed in long double (64-bit significand on x86-64,
// 113 bits where long double is quad precision), both finer than df64's
// 48 bits.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "df64.cuh"

using nbv::df64;
using namespace nbv;   // the df64 operators
using LD = long double;

static LD val(df64 x) { return (LD)x.hi + (LD)x.lo; }

static df64 from_ld(LD x) {
  const float hi = (float)x;
  const float lo = (float)(x - (LD)hi);
  df64 r;
  nbv::df_fast_two_sum(hi, lo, r.hi, r.lo);
  return r;
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> E(-30, 30);
  auto rnd = [&]() { return (float)std::ldexp(U(rng), E(rng)); };

  // error-free transformations: exact in long double
  long bad_sum = 0, bad_prod = 0, bad_fast = 0;
  for (int i = 0; i < 200000; ++i) {
    const float a = rnd(), b = rnd();
    float s, e;
    nbv::df_two_sum(a, b, s, e);
    if ((LD)s + (LD)e != (LD)a + (LD)b) ++bad_sum;
    const float x = std::fabs(a) >= std::fabs(b) ? a : b, y = std::fabs(a) >= std::fabs(b) ? b : a;
    nbv::df_fast_two_sum(x, y, s, e);
    if ((LD)s + (LD)e != (LD)x + (LD)y) ++bad_fast;
    nbv::df_two_prod(a, b, s, e);
    if ((LD)s + (LD)e != (LD)a * (LD)b) ++bad_prod;
  }
  std::printf("two_sum_inexact %ld\nfast_two_sum_inexact %ld\ntwo_prod_inexact %ld\n", bad_sum, bad_fast, bad_prod);

  // add, mul, fms against long double: relative error (add: relative to the
  // larger operand, which bounds it under cancellation)
  LD e_add = 0, e_mul = 0, e_fms = 0, e_rsq = 0;
  for (int i = 0; i < 100000; ++i) {
    const df64 x = from_ld((LD)U(rng) * std::ldexp(1.0L, E(rng) / 3) * (1 + (LD)U(rng) * 1e-9L));
    const df64 y = from_ld((LD)U(rng) * std::ldexp(1.0L, E(rng) / 3) * (1 + (LD)U(rng) * 1e-9L));
    const df64 z = from_ld((LD)U(rng) * std::ldexp(1.0L, E(rng) / 3));
    const LD X = val(x), Y = val(y), Z = val(z);
    const LD sc = std::fmax(std::fabs(X), std::fabs(Y));
    if (sc > 0) e_add = std::fmax(e_add, std::fabs(val(nbv::df_add(x, y)) - (X + Y)) / sc);
    if (X * Y != 0) e_mul = std::fmax(e_mul, std::fabs(val(nbv::df_mul(x, y)) - X * Y) / std::fabs(X * Y));
    const LD f = Z - X * Y, fs = std::fmax(std::fabs(Z), std::fabs(X * Y));
    if (fs > 0) e_fms = std::fmax(e_fms, std::fabs(val(nbv::df_fms(z, x, y)) - f) / fs);
    const LD P = std::ldexp(std::fabs((LD)U(rng)) + 0.01L, E(rng));
    const df64 p = from_ld(P);
    const LD R = 1.0L / std::sqrt(val(p));
    e_rsq = std::fmax(e_rsq, std::fabs(val(nbv::df_rsqrt(p)) - R) / R);
  }
  std::printf("add_rel_err_log2 %.3f\nmul_rel_err_log2 %.3f\nfms_rel_err_log2 %.3f\nrsqrt_rel_err_log2 %.3f\n",
              (double)std::log2(e_add), (double)std::log2(e_mul), (double)std::log2(e_fms),
              (double)std::log2(e_rsq));

  // Cholesky + inverse of Jacobi-scaled damped matrices lambda I + G G^T
  // (rank-deficient G, so that the damping decides the small pivots), in
  // df64 and in long double; the inverse factors rounded to float compared.
  const int n = 28, m = 200;
  std::normal_distribution<double> N(0.0, 1.0);
  long equal = 0, equal_f = 0, total = 0;
  double worst = 0.0, worst_f = 0.0;
  for (int q = 0; q < m; ++q) {
    const int r = 20;
    std::vector<LD> G((size_t)n * r), H((size_t)n * n);
    for (int i = 0; i < n; ++i) {
      const LD s = std::ldexp(1.0L, (int)(N(rng) * 6));      // row scales over ~2^+-12
      for (int k = 0; k < r; ++k) G[i * r + k] = s * (LD)N(rng);
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        LD a = i == j ? 0.1L : 0.0L;
        for (int k = 0; k < r; ++k) a += G[i * r + k] * G[j * r + k];
        H[i * n + j] = (LD)(float)a;                         // the sums arrive in single precision
      }
    std::vector<LD> d(n);
    for (int i = 0; i < n; ++i) d[i] = 1.0L / std::sqrt(H[i * n + i]);
    // reference in long double
    std::vector<LD> L((size_t)n * n, 0.0L), Li((size_t)n * n, 0.0L);
    for (int k = 0; k < n; ++k) {
      LD p = H[k * n + k] * d[k] * d[k];
      for (int t = 0; t < k; ++t) p -= L[k * n + t] * L[k * n + t];
      L[k * n + k] = std::sqrt(p);
      for (int i = k + 1; i < n; ++i) {
        LD a = H[i * n + k] * d[i] * d[k];
        for (int t = 0; t < k; ++t) a -= L[i * n + t] * L[k * n + t];
        L[i * n + k] = a / L[k * n + k];
      }
    }
    for (int j = 0; j < n; ++j) {
      Li[j * n + j] = 1.0L / L[j * n + j];
      for (int i = j + 1; i < n; ++i) {
        LD a = 0.0L;
        for (int t = j; t < i; ++t) a += L[i * n + t] * Li[t * n + j];
        Li[i * n + j] = -a / L[i * n + i];
      }
    }
    // df64: right-looking factorisation keeping 1 / L_kk, then the inverse
    std::vector<df64> P((size_t)n * n), X((size_t)n * n, df64{0.0f, 0.0f}), dd(n);
    for (int i = 0; i < n; ++i) dd[i] = nbv::df_rsqrt(from_ld(H[i * n + i]));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j)
        P[i * n + j] = nbv::df_mul(nbv::df_mul(from_ld(H[i * n + j]), dd[i]), dd[j]);
    std::vector<df64> inv(n);
    for (int k = 0; k < n; ++k) {
      inv[k] = nbv::df_rsqrt(P[k * n + k]);
      for (int i = k + 1; i < n; ++i) P[i * n + k] = nbv::df_mul(P[i * n + k], inv[k]);
      for (int i = k + 1; i < n; ++i)
        for (int j = k + 1; j <= i; ++j) P[i * n + j] -= P[i * n + k] * P[j * n + k];   // operator form
    }
    for (int k = 0; k < n; ++k) {
      for (int j = 0; j < k; ++j) X[k * n + j] = nbv::df_neg(nbv::df_mul(inv[k], X[k * n + j]));
      X[k * n + k] = inv[k];
      for (int i = k + 1; i < n; ++i)
        for (int j = 0; j <= k; ++j) X[i * n + j] += P[i * n + k] * X[k * n + j];
    }
    // the same factorisation in plain single precision, to show what the
    // comparison detects
    std::vector<float> Pf((size_t)n * n), Xf((size_t)n * n, 0.0f), df(n), invf(n);
    for (int i = 0; i < n; ++i) df[i] = 1.0f / std::sqrt((float)H[i * n + i]);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j) Pf[i * n + j] = (float)H[i * n + j] * df[i] * df[j];
    for (int k = 0; k < n; ++k) {
      invf[k] = 1.0f / std::sqrt(std::fmax(Pf[k * n + k], 1e-30f));
      for (int i = k + 1; i < n; ++i) Pf[i * n + k] *= invf[k];
      for (int i = k + 1; i < n; ++i)
        for (int j = k + 1; j <= i; ++j) Pf[i * n + j] -= Pf[i * n + k] * Pf[j * n + k];
    }
    for (int k = 0; k < n; ++k) {
      for (int j = 0; j < k; ++j) Xf[k * n + j] = -invf[k] * Xf[k * n + j];
      Xf[k * n + k] = invf[k];
      for (int i = k + 1; i < n; ++i)
        for (int j = 0; j <= k; ++j) Xf[i * n + j] += Pf[i * n + k] * Xf[k * n + j];
    }
    for (int i = 0; i < n; ++i) {
      LD rs = 0.0L;
      for (int j = 0; j <= i; ++j) rs = std::fmax(rs, std::fabs(Li[i * n + j] * d[j]));
      for (int j = 0; j <= i; ++j) {
        const float want = (float)(Li[i * n + j] * d[j]);
        const float got = nbv::df_to_float(nbv::df_mul(X[i * n + j], dd[j]));
        const float gotf = Xf[i * n + j] * df[j];
        ++total;
        if (want == got) ++equal;
        if (want == gotf) ++equal_f;
        worst = std::fmax(worst, (double)(std::fabs((LD)got - (LD)want) / rs));
        worst_f = std::fmax(worst_f, (double)(std::fabs((LD)gotf - (LD)want) / rs));
      }
    }
  }
  std::printf("factor_equal_fraction %.6f\nfactor_worst_rel_row %.3e\n", (double)equal / (double)total, worst);
  std::printf("float_equal_fraction %.6f\nfloat_worst_rel_row %.3e\n", (double)equal_f / (double)total, worst_f);
  return 0;
}
