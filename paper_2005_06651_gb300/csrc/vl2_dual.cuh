// Forward-mode dual numbers for device code: a value and N tangent components.  Instantiating the device
// flux functions with DualN<N> gives N columns of their local Jacobian at the point (branches are taken on
// the value, so a limiter / fan-region / upwind choice stays frozen, as in any first-order derivative
// of a piecewise-smooth map away from its switching surfaces).
#pragma once
#include <cuda_runtime.h>

namespace vl2 {

template <int N>
struct DualN {
  double v;
  double d[N];
  __device__ __forceinline__ DualN() : v(0.0) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.0;
  }
  __device__ __forceinline__ DualN(double x) : v(x) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.0;
  }
  __device__ __forceinline__ explicit operator double() const { return v; }
};

template <int N>
__device__ __forceinline__ DualN<N> operator+(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v + b.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator-(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v - b.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator-(const DualN<N>& a) {
  DualN<N> r(-a.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator*(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r(a.v * b.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator/(const DualN<N>& a, const DualN<N>& b) {
  const double ib = 1.0 / b.v;
  const double q = a.v * ib;
  DualN<N> r(q);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - q * b.d[k]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> sqrt(const DualN<N>& a) {
  const double s = ::sqrt(a.v);
  const double h = 0.5 / s;
  DualN<N> r(s);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> rsqrt(const DualN<N>& a) {
  const double s = ::rsqrt(a.v);
  const double h = -0.5 * s / a.v;
  DualN<N> r(s);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> fabs(const DualN<N>& a) {
  return (__double_as_longlong(a.v) < 0) ? -a : a;
}
// the integer-pipe sign tests and orderings of the flux functions look at the value
template <int N>
__device__ __forceinline__ long long dbits(const DualN<N>& x) {
  return __double_as_longlong(x.v);
}
template <int N>
__device__ __forceinline__ long long okey(const DualN<N>& x) {
  const long long b = __double_as_longlong(x.v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

}  // namespace vl2
