// Forward-mode dual numbers with three partial derivatives (FP64), for the position
// derivatives of the adjoint: a kernel evaluates an energy-like expression with the
// site coordinates seeded as duals and reads d(expression)/d(position) exactly
// (no differencing).
#pragma once

#include <cuda_runtime.h>

namespace bp {

struct Dual3 {
  double v, d0, d1, d2;
};

__device__ __forceinline__ Dual3 dual(double v) { return {v, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ Dual3 seed(double v, int k) {
  return {v, k == 0 ? 1.0 : 0.0, k == 1 ? 1.0 : 0.0, k == 2 ? 1.0 : 0.0};
}
__device__ __forceinline__ Dual3 operator+(Dual3 a, Dual3 b) { return {a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
__device__ __forceinline__ Dual3 operator-(Dual3 a, Dual3 b) { return {a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
__device__ __forceinline__ Dual3 operator-(Dual3 a) { return {-a.v, -a.d0, -a.d1, -a.d2}; }
__device__ __forceinline__ Dual3 operator*(Dual3 a, Dual3 b) {
  return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
__device__ __forceinline__ Dual3 operator*(Dual3 a, double s) { return {a.v * s, a.d0 * s, a.d1 * s, a.d2 * s}; }
__device__ __forceinline__ Dual3 operator*(double s, Dual3 a) { return a * s; }
__device__ __forceinline__ Dual3 operator+(Dual3 a, double s) { return {a.v + s, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ Dual3 operator+(double s, Dual3 a) { return a + s; }
__device__ __forceinline__ Dual3 operator-(Dual3 a, double s) { return {a.v - s, a.d0, a.d1, a.d2}; }
__device__ __forceinline__ Dual3 operator-(double s, Dual3 a) { return {s - a.v, -a.d0, -a.d1, -a.d2}; }
__device__ __forceinline__ Dual3& operator+=(Dual3& a, Dual3 b) {
  a = a + b;
  return a;
}
// 1 / a
__device__ __forceinline__ Dual3 inv(Dual3 a) {
  const double r = 1.0 / a.v, r2 = -r * r;
  return {r, a.d0 * r2, a.d1 * r2, a.d2 * r2};
}
__device__ __forceinline__ Dual3 sqrt(Dual3 a) {
  const double s = ::sqrt(a.v), h = 0.5 / s;
  return {s, a.d0 * h, a.d1 * h, a.d2 * h};
}
__device__ __forceinline__ Dual3 exp(Dual3 a) {
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
