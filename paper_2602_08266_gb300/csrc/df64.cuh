// Float-float arithmetic ("df64"): a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi) / 2, about 48 significant bits, computed on
// the FP32 pipes. On this part the FP64 pipe issues about one warp
// instruction per 16 SM cycles against four FP32 warp instructions per cycle,
// so a factorisation that needs more than single precision runs several
// times faster in df64 than in double even at ten to twenty FP32 operations
// per df64 operation.
//
// Building blocks (error-free transformations):
//   df_two_sum       s + e = a + b exactly              Knuth, TAOCP vol. 2, 4.2.2
//   df_fast_two_sum  the same for |a| >= |b|            Dekker (1971)
//   df_two_prod      p + e = a b exactly, e by one FMA  Dekker (1971), FMA form
// The addition renormalises twice (the variant that keeps its relative error
// near 2^-47 under cancellation, needed by elimination updates); the
// reciprocal square root takes the single-precision estimate through two
// Newton steps y <- y + y (1 - x y^2) / 2 evaluated in df64.
//
// Host and device share the code (the host build is used by the CPU tests).
// Device code uses the round-to-nearest intrinsics so that no sum of a
// product is contracted into an FMA; host code must be compiled with
// -ffp-contract=off for the same reason.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace nbv {

struct df64 {
  float hi, lo;
};

DF_HD float df_add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DF_HD float df_sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DF_HD float df_mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DF_HD float df_fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

DF_HD df64 df_from_float(float x) { return df64{x, 0.0f}; }

DF_HD void df_two_sum(float a, float b, float& s, float& e) {
  s = df_add_rn(a, b);
  const float bb = df_sub_rn(s, a);
  e = df_add_rn(df_sub_rn(a, df_sub_rn(s, bb)), df_sub_rn(b, bb));
}

DF_HD void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = df_add_rn(a, b);
  e = df_sub_rn(b, df_sub_rn(s, a));
}

DF_HD void df_two_prod(float a, float b, float& p, float& e) {
  p = df_mul_rn(a, b);
  e = df_fma_rn(a, b, -p);
}

DF_HD df64 df_neg(df64 x) { return df64{-x.hi, -x.lo}; }

DF_HD df64 df_add(df64 x, df64 y) {
  float s1, s2, t1, t2;
  df_two_sum(x.hi, y.hi, s1, s2);
  df_two_sum(x.lo, y.lo, t1, t2);
  s2 = df_add_rn(s2, t1);
  df_fast_two_sum(s1, s2, s1, s2);
  s2 = df_add_rn(s2, t2);
  df_fast_two_sum(s1, s2, s1, s2);
  return df64{s1, s2};
}

DF_HD df64 df_sub(df64 x, df64 y) { return df_add(x, df_neg(y)); }

DF_HD df64 df_mul(df64 x, df64 y) {
  float p, e;
  df_two_prod(x.hi, y.hi, p, e);
  e = df_fma_rn(x.hi, y.lo, e);
  e = df_fma_rn(x.lo, y.hi, e);
  df_fast_two_sum(p, e, p, e);
  return df64{p, e};
}

DF_HD df64 df_mul_f(df64 x, float b) {
  float p, e;
  df_two_prod(x.hi, b, p, e);
  e = df_fma_rn(x.lo, b, e);
  df_fast_two_sum(p, e, p, e);
  return df64{p, e};
}

// a - b c, the elimination update.
DF_HD df64 df_fms(df64 a, df64 b, df64 c) { return df_sub(a, df_mul(b, c)); }

// Nearest float to hi + lo (|lo| <= ulp(hi) / 2, so one rounded add).
DF_HD float df_to_float(df64 x) { return df_add_rn(x.hi, x.lo); }

// x^-1/2 for x > 0 in the normal float range.
DF_HD df64 df_rsqrt(df64 x) {
#ifdef __CUDA_ARCH__
  df64 y = df_from_float(rsqrtf(x.hi));
#else
  df64 y = df_from_float(1.0f / std::sqrt(x.hi));
#endif
  for (int it = 0; it < 2; ++it) {
    const df64 r = df_sub(df_from_float(1.0f), df_mul(x, df_mul(y, y)));
    y = df_add(y, df_mul_f(df_mul(y, r), 0.5f));
  }
  return y;
}

// Operators, so that code written for double reads the same in df64.
DF_HD df64 operator+(df64 a, df64 b) { return df_add(a, b); }
DF_HD df64 operator-(df64 a, df64 b) { return df_sub(a, b); }
DF_HD df64 operator-(df64 a) { return df_neg(a); }
DF_HD df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
DF_HD df64& operator+=(df64& a, df64 b) { return a = df_add(a, b); }
DF_HD df64& operator-=(df64& a, df64 b) { return a = df_sub(a, b); }
DF_HD df64& operator*=(df64& a, df64 b) { return a = df_mul(a, b); }
DF_HD bool operator>=(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
DF_HD bool df_isfinite(df64 a) { return std::isfinite(a.hi) && std::isfinite(a.lo); }
DF_HD df64 df_max(df64 a, df64 b) { return a >= b ? a : b; }

}  // namespace nbv
