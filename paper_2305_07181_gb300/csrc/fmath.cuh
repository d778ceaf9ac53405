// Table-driven float64 log, log1p, exp and expm1 for the residual kernels,
// after P. T. P. Tang (ACM TOMS 15(2), 1989: exponential; 16(4), 1990:
// logarithm).  On GB300 a library float64 log costs ~32 and an exp ~18 fused
// multiply-adds of the FP64 pipe, the resource every kernel here is bound by;
// these versions cost ~12-14.
//
//   log:  x = 2^k m with m in [sqrt(2)/2, sqrt(2)), c = j/128 the nearest grid
//         point, r = (m - c)/c (m - c exact), log x = k ln2 + ln c + log1p(r),
//         |r| < 0.0056, log1p(r) by its Taylor series through r^9
//         (truncation < 2^-60 |r|); ln c and 1/c tabulated.
//   exp:  x = (32 k + j) ln2/32 + r, |r| <= ln2/64, exp x = 2^k 2^(j/32) exp(r),
//         exp(r) - 1 by its Taylor series through r^6 (truncation < 2^-58);
//         2^(j/32) tabulated as a float64 pair.
//   log1p(x) = log(u + c) with u = 1 + x rounded and c = x - (u - 1) the
//   rounding error, carried into r; for |x| < 2^-5 directly by its Taylor
//   series through x^12 (truncation < 2^-63 |x|); expm1 from the exp reduction as
//   (2^k T_hi - 1) + 2^k (T_hi p + T_lo) (the first difference is exact where
//   it cancels), and for |x| < 1/16 by its Taylor series through x^10.
//   Tables: fmath_tables.h (gen_fmath_tables.py).
// Domain: finite normal positive arguments for log (log1p: 1 + x normal
// positive), |x| < 708 for exp/expm1; anything else goes to the CUDA library
// function.  The range tests and the grid point c are formed from the bit
// patterns by integer operations: on GB300 a float64 compare or an
// integer-to-float64 conversion occupies the float64 pipe like an FMA.  Error: a few ulp (tests/test_gpu_fmath.py compares against
// the host's correctly rounded-to-1-ulp libm over random arguments).
#pragma once

#include "fmath_tables.h"

namespace esplit {
namespace fm {

__device__ __forceinline__ double pow2i(int k) {  // 2^k, |k| <= 1022
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// log(x + corr) for x > 0 normal (< 2^1022) and corr a small correction
// (|corr| <= ulp(x)); CORR = false: plain log(x)
template <bool CORR>
__device__ __forceinline__ double log_core(double x, double corr) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const long long f = b & 0xFFFFFFFFFFFFFLL;
  const long long F_SQRT2 = 0x6A09E667F3BCDLL;  // mantissa field of sqrt(2)
  int k, j;
  double m;
  if (f >= F_SQRT2) {  // m = M/2 in [0.707, 1)
    k = e + 1;
    m = __longlong_as_double(f | (1022LL << 52));
    j = 64 + (int)((f + (1LL << 45)) >> 46);
  } else {  // m = M in [1, 1.414)
    k = e;
    m = __longlong_as_double(f | (1023LL << 52));
    j = 128 + (int)((f + (1LL << 44)) >> 45);
  }
  const int t = j - LOG_J0;
  // c = j/128 built from its bits: j in [91, 128] is (j - 64)/64 above 2^-1
  // (j = 128 carries into the exponent: 1.0), j in [128, 181] is (j - 128)/128
  // above 1
  const long long cb = (f >= F_SQRT2) ? (1022LL << 52) + ((long long)(j - 64) << 46)
                                      : (1023LL << 52) + ((long long)(j - 128) << 45);
  const double c = __longlong_as_double(cb);
  const double inv = __ldg(&LOG_INV_C[t]);
  double r = (m - c) * inv;
  if (CORR) r = fma(corr * pow2i(-k), inv, r);
  const double r2 = r * r;
  double q = fma(r, LOG_C9, LOG_C8);
  q = fma(r, q, LOG_C7);
  q = fma(r, q, LOG_C6);
  q = fma(r, q, LOG_C5);
  q = fma(r, q, LOG_C4);
  q = fma(r, q, LOG_C3);
  q = fma(r, q, LOG_C2);
  const double p = fma(r2, q, r);
  const double kd = (double)k;
  const double hi = fma(kd, LN2_HI, __ldg(&LOG_C_HI[t]));
  const double lo = fma(kd, LN2_LO, __ldg(&LOG_C_LO[t]));
  return hi + (lo + p);
}

// normal, positive, below 2^1022: sign 0 and biased exponent field 1..2044
__device__ __forceinline__ bool log_domain(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return b - (1ULL << 52) < (2044ULL << 52);
}

// |x| < y for a positive finite y given by its bit pattern (the patterns of
// non-negative floats order as the values; NaN: false)
__device__ __forceinline__ bool abs_below(double x, unsigned long long y_bits) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL) < y_bits;
}
constexpr unsigned long long BITS_2M5 = 0x3FA0000000000000ULL;  // 2^-5
constexpr unsigned long long BITS_2M4 = 0x3FB0000000000000ULL;  // 2^-4
constexpr unsigned long long BITS_708 = 0x4086200000000000ULL;  // 708.0

__device__ __forceinline__ double log(double x) { return log_domain(x) ? log_core<false>(x, 0.0) : ::log(x); }

__device__ __forceinline__ double log1p(double x) {
  if (abs_below(x, BITS_2M5)) {
    double q = fma(x, LOG_C12, LOG_C11);
    q = fma(x, q, LOG_C10);
    q = fma(x, q, LOG_C9);
    q = fma(x, q, LOG_C8);
    q = fma(x, q, LOG_C7);
    q = fma(x, q, LOG_C6);
    q = fma(x, q, LOG_C5);
    q = fma(x, q, LOG_C4);
    q = fma(x, q, LOG_C3);
    q = fma(x, q, LOG_C2);
    return fma(x * x, q, x);
  }
  const double u = 1.0 + x;
  if (!log_domain(u)) return ::log1p(x);
  const double corr = x - (u - 1.0);
  return log_core<true>(u, corr);
}

// exp reduction: x = N ln2/32 + r; returns p = exp(r) - 1, j = N mod 32, k = N div 32
__device__ __forceinline__ double exp_reduce(double x, int& j, int& k) {
  const double SHIFT = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
  const double tt = fma(x, INV_L32, SHIFT);
  const int N = (int)__double2loint(tt);
  const double nd = tt - SHIFT;
  double r = fma(-nd, L32_HI, x);
  r = fma(-nd, L32_LO, r);
  j = N & 31;
  k = N >> 5;
  double q = fma(r, EXP_E6, EXP_E5);
  q = fma(r, q, EXP_E4);
  q = fma(r, q, EXP_E3);
  q = fma(r, q, EXP_E2);
  return fma(r * r, q, r);
}

__device__ __forceinline__ double exp(double x) {
  if (!abs_below(x, BITS_708)) return ::exp(x);
  int j, k;
  const double p = exp_reduce(x, j, k);
  const double th = __ldg(&EXP_T_HI[j]);
  const double s = th + fma(th, p, __ldg(&EXP_T_LO[j]));
  return s * pow2i(k);
}

__device__ __forceinline__ double expm1(double x) {
  if (abs_below(x, BITS_2M4)) {  // Taylor series through x^10 (truncation < 2^-64 |x|)
    double q = fma(x, EXP_E10, EXP_E9);
    q = fma(x, q, EXP_E8);
    q = fma(x, q, EXP_E7);
    q = fma(x, q, EXP_E6);
    q = fma(x, q, EXP_E5);
    q = fma(x, q, EXP_E4);
    q = fma(x, q, EXP_E3);
    q = fma(x, q, EXP_E2);
    return fma(x * x, q, x);
  }
  if (!abs_below(x, BITS_708)) return ::expm1(x);
  int j, k;
  const double p = exp_reduce(x, j, k);
  const double th = __ldg(&EXP_T_HI[j]);
  const double sc = pow2i(k);
  const double lo = fma(th, p, __ldg(&EXP_T_LO[j])) * sc;
  return fma(th, sc, -1.0) + lo;
}

}  // namespace fm
}  // namespace esplit
