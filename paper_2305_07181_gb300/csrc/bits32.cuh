// float64 <-> float32 conversions by integer operations on the bit patterns.
// On GB300 a float64<->float32 conversion instruction occupies the float64
// pipe; the float32 and FP32-bulk kernels use these instead so that their
// float64 pipe stays free (or free for the float64 work they do have).
#pragma once

#include <cuda_runtime.h>

namespace esplit {

// v = hi + lo with float hi (v's first 24 significant bits, truncated) and
// float lo (the remaining 29 bits, rounded to 24), by integer operations on
// the bit patterns: on GB300 a float64<->float32 conversion occupies the FP64
// pipe, which the kernel's pointwise float64 work already saturates.  |v| below
// 2^-126 gives hi = lo = 0; |v| below 2^-74 loses lo (both far below the
// round-off of the float64 terms these variations are added to).
__device__ __forceinline__ void split_f64(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ffULL);  // biased exponent
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  if (e <= 1023 - 127) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFULL;
  hi = __uint_as_float(sgn | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(mant >> 29));
  const int E = e - 1075;  // weight of the lowest mantissa bit
  if (E < -126) {
    lo = 0.0f;
    return;
  }
  const float lf = __uint2float_rn((unsigned)(mant & 0x1FFFFFFFULL));
  lo = __uint_as_float(sgn | __float_as_uint(__fmul_rn(lf, __uint_as_float((unsigned)(E + 127) << 23))));
}

// float -> double by the bit patterns (normal floats and zero; float
// subnormals, far below the terms these sums are added to, give zero; the
// kernels report non-finite states through their own checks)
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// float32 value of a float64, rounded to nearest (ties away from zero), by
// integer operations: half a float32 unit in the last place is added to the
// bit pattern (a carry out of the mantissa moves into the exponent) and the
// low 29 bits dropped.  Values beyond the float32 range take the conversion
// instruction (overflow to infinity, NaN kept), so non-physical states stay
// detectable; |v| below 2^-126 gives 0.
__device__ __forceinline__ float f32_round(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) + (1ULL << 28);
  const int e = (int)((b >> 52) & 0x7ffULL);
  if (e >= 1023 + 128) return (float)v;
  if (e <= 1023 - 127) return 0.0f;
  return __uint_as_float(((unsigned)(b >> 63) << 31) | ((unsigned)(e - 1023 + 127) << 23) |
                         (unsigned)((b & 0xFFFFFFFFFFFFFULL) >> 29));
}

// (float)(a - b): one float64 subtraction (a single rounding at 2^-53), then
// the bit-pattern rounding to float32
__device__ __forceinline__ float f32_diff(double a, double b) { return f32_round(a - b); }

}  // namespace esplit
