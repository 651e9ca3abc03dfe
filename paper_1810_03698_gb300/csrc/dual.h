// Forward-mode dual numbers with three partial derivatives, for the position
// derivatives of the adjoint: a kernel evaluates an energy-like expression with the
// site coordinates seeded as duals and reads d(expression)/d(position) exactly
// (no differencing).  Dual3T<double> and Dual3T<float>; a scalar operand is taken
// in the dual's own precision.
#pragma once

#include <cuda_runtime.h>

namespace bp {

template <typename S>
struct Dual3T {
  S v, d0, d1, d2;
};
typedef Dual3T<double> Dual3;

template <typename S>
struct same_t {
  typedef S type;
};

template <typename S>
__device__ __forceinline__ Dual3T<S> dual_of(S v) {
  return {v, S(0), S(0), S(0)};
}
__device__ __forceinline__ Dual3 dual(double v) { return dual_of<double>(v); }
template <typename S>
__device__ __forceinline__ Dual3T<S> seed_of(S v, int k) {
  return {v, k == 0 ? S(1) : S(0), k == 1 ? S(1) : S(0), k == 2 ? S(1) : S(0)};
}
__device__ __forceinline__ Dual3 seed(double v, int k) { return seed_of<double>(v, k); }

template <typename S>
__device__ __forceinline__ Dual3T<S> operator+(Dual3T<S> a, Dual3T<S> b) {
  return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator-(Dual3T<S> a, Dual3T<S> b) {
  return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator-(Dual3T<S> a) {
  return {-a.v, -a.d0, -a.d1, -a.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator*(Dual3T<S> a, Dual3T<S> b) {
  return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator*(Dual3T<S> a, typename same_t<S>::type s) {
  return {a.v * s, a.d0 * s, a.d1 * s, a.d2 * s};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator*(typename same_t<S>::type s, Dual3T<S> a) {
  return a * s;
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator+(Dual3T<S> a, typename same_t<S>::type s) {
  return {a.v + s, a.d0, a.d1, a.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator+(typename same_t<S>::type s, Dual3T<S> a) {
  return a + s;
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator-(Dual3T<S> a, typename same_t<S>::type s) {
  return {a.v - s, a.d0, a.d1, a.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S> operator-(typename same_t<S>::type s, Dual3T<S> a) {
  return {s - a.v, -a.d0, -a.d1, -a.d2};
}
template <typename S>
__device__ __forceinline__ Dual3T<S>& operator+=(Dual3T<S>& a, Dual3T<S> b) {
  a = a + b;
  return a;
}
// 1 / a
template <typename S>
__device__ __forceinline__ Dual3T<S> inv(Dual3T<S> a) {
  const S r = S(1) / a.v, r2 = -r * r;
  return {r, a.d0 * r2, a.d1 * r2, a.d2 * r2};
}
__device__ __forceinline__ Dual3T<double> sqrt(Dual3T<double> a) {
  const double s = ::sqrt(a.v), h = 0.5 / s;
  return {s, a.d0 * h, a.d1 * h, a.d2 * h};
}
__device__ __forceinline__ Dual3T<float> sqrt(Dual3T<float> a) {
  const float s = ::sqrtf(a.v), h = 0.5f / s;
  return {s, a.d0 * h, a.d1 * h, a.d2 * h};
}
__device__ __forceinline__ Dual3T<double> exp(Dual3T<double> a) {
  const double e = ::exp(a.v);
  return {e, a.d0 * e, a.d1 * e, a.d2 * e};
}
// plain overloads, so unqualified calls on doubles inside this namespace still resolve
__host__ __device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
__host__ __device__ __forceinline__ double exp(double a) { return ::exp(a); }
__device__ __forceinline__ double value(Dual3 a) { return a.v; }
__device__ __forceinline__ double value(double a) { return a; }
__device__ __forceinline__ double inv(double a) { return 1.0 / a; }

}  // namespace bp
