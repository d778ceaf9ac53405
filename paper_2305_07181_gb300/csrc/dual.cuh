// Forward-mode dual numbers with N derivative components, for the exact
// pointwise Jacobians the reverse (VJP) kernels apply transposed.  The
// physics templates of phys.cuh run unchanged on Dual<N>.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "fmath.cuh"

namespace esplit {

template <int N>
struct Dual {
  double v;
  double d[N];
  __host__ __device__ __forceinline__ Dual() {}
  __host__ __device__ __forceinline__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};

template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(double b, const Dual<N>& a) {
  return a + b;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v -= b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(double b, const Dual<N>& a) {
  Dual<N> r = -a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double b, const Dual<N>& a) {
  return a * b;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) {
  return a * (1.0 / b);
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) {
  Dual<N> r;
  double ib = 1.0 / b.v;
  r.v = a * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -r.v * b.d[i] * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) {
  a = a + b;
  return a;
}
template <int N>
__device__ __forceinline__ Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) {
  a = a - b;
  return a;
}
template <int N>
__device__ __forceinline__ Dual<N>& operator*=(Dual<N>& a, const Dual<N>& b) {
  a = a * b;
  return a;
}
template <int N>
__device__ __forceinline__ bool operator>(const Dual<N>& a, double b) {
  return a.v > b;
}
template <int N>
__device__ __forceinline__ bool operator>=(const Dual<N>& a, double b) {
  return a.v >= b;
}
template <int N>
__device__ __forceinline__ bool operator<(const Dual<N>& a, double b) {
  return a.v < b;
}
template <int N>
__device__ __forceinline__ bool operator>(const Dual<N>& a, const Dual<N>& b) {
  return a.v > b.v;
}

template <int N>
__device__ __forceinline__ Dual<N> chain(const Dual<N>& a, double fv, double dfdx) {
  Dual<N> r;
  r.v = fv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = dfdx * a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> t_log(const Dual<N>& a) {
  return chain(a, fm::log(a.v), 1.0 / a.v);
}
template <int N>
__device__ __forceinline__ Dual<N> t_exp(const Dual<N>& a) {
  double e = fm::exp(a.v);
  return chain(a, e, e);
}
template <int N>
__device__ __forceinline__ Dual<N> t_sqrt(const Dual<N>& a) {
  double s = sqrt(a.v);
  return chain(a, s, 0.5 / s);
}
template <int N>
__device__ __forceinline__ Dual<N> t_abs(const Dual<N>& a) {
  // d|x|/dx = sign(x), with sign(0) = 0
  return chain(a, fabs(a.v), a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0));
}
template <int N>
__device__ __forceinline__ Dual<N> t_expm1(const Dual<N>& a) {
  return chain(a, fm::expm1(a.v), fm::exp(a.v));
}
template <int N>
__device__ __forceinline__ Dual<N> t_log1p(const Dual<N>& a) {
  return chain(a, fm::log1p(a.v), 1.0 / (1.0 + a.v));
}
template <int N>
__device__ __forceinline__ bool t_isfinite(const Dual<N>& a) {
  return ::isfinite(a.v);
}

}  // namespace esplit
