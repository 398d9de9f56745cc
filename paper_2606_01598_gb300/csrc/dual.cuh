// Dual numbers (value + directional derivative) for kernels written once over a scalar type
// T: float for a plain pass, Dual for a pass that also carries a tangent (forward-mode
// differentiation). Used by the learned network (net.cu) and the quadrupole Hessian-vector
// product (quad.cu).
#pragma once

#include <cuda_runtime.h>

namespace gbpme {

struct Dual {
  float v, d;
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(float x) : v(x), d(0.f) {}
  __device__ __forceinline__ Dual(float x, float y) : v(x), d(y) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.v * b.d + a.d * b.v); }
__device__ __forceinline__ Dual operator*(float s, Dual a) { return Dual(s * a.v, s * a.d); }
__device__ __forceinline__ Dual operator*(Dual a, float s) { return Dual(s * a.v, s * a.d); }
__device__ __forceinline__ Dual operator+(Dual a, float s) { return Dual(a.v + s, a.d); }
__device__ __forceinline__ Dual operator+(float s, Dual a) { return Dual(a.v + s, a.d); }
__device__ __forceinline__ Dual operator-(float s, Dual a) { return Dual(s - a.v, -a.d); }
__device__ __forceinline__ Dual operator-(Dual a, float s) { return Dual(a.v - s, a.d); }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a.v += b.v; a.d += b.d; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a.v -= b.v; a.d -= b.d; return a; }

__device__ __forceinline__ float rcpT(float a) { return 1.f / a; }
__device__ __forceinline__ Dual rcpT(Dual a) { const float r = 1.f / a.v; return Dual(r, -a.d * r * r); }
__device__ __forceinline__ float sqrtT(float a) { return sqrtf(a); }
__device__ __forceinline__ Dual sqrtT(Dual a) { const float s = sqrtf(a.v); return Dual(s, 0.5f * a.d / s); }
__device__ __forceinline__ void sincosT(float a, float& s, float& c) { sincosf(a, &s, &c); }
__device__ __forceinline__ void sincosT(Dual a, Dual& s, Dual& c) {
  float sv, cv;
  sincosf(a.v, &sv, &cv);
  s = Dual(sv, cv * a.d);
  c = Dual(cv, -sv * a.d);
}
__device__ __forceinline__ float sigmoidT(float a) { return 1.f / (1.f + expf(-a)); }
__device__ __forceinline__ Dual sigmoidT(Dual a) {
  const float s = 1.f / (1.f + expf(-a.v));
  return Dual(s, a.d * s * (1.f - s));
}
template <typename T> __device__ __forceinline__ T siluT(T x) { return x * sigmoidT(x); }
// d silu / dx = s (1 + x (1 - s)), s = sigmoid(x)
template <typename T> __device__ __forceinline__ T dsiluT(T x) {
  const T s = sigmoidT(x);
  return s * (1.f + x * (1.f - s));
}
__device__ __forceinline__ float shfl_xor(float x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
__device__ __forceinline__ Dual shfl_xor(Dual x, int o) {
  return Dual(__shfl_xor_sync(0xffffffffu, x.v, o), __shfl_xor_sync(0xffffffffu, x.d, o));
}
template <typename T> __device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += shfl_xor(x, o);
  return x;
}
__device__ __forceinline__ float rsqrtT(float a) { return rsqrtf(a); }
__device__ __forceinline__ Dual rsqrtT(Dual a) {
  const float r = rsqrtf(a.v);
  return Dual(r, -0.5f * a.d * r * r * r);
}
__device__ __forceinline__ float expT(float a) { return expf(a); }
__device__ __forceinline__ Dual expT(Dual a) {
  const float e = expf(a.v);
  return Dual(e, e * a.d);
}
// erfc'(x) = -2/sqrt(pi) exp(-x^2)
__device__ __forceinline__ float erfcT(float a) { return erfcf(a); }
__device__ __forceinline__ Dual erfcT(Dual a) {
  return Dual(erfcf(a.v), -1.1283791670955126f * expf(-a.v * a.v) * a.d);
}
__device__ __forceinline__ float dval(float x) { return x; }
__device__ __forceinline__ float dval(Dual x) { return x.v; }
__device__ __forceinline__ float dtan(float) { return 0.f; }
__device__ __forceinline__ float dtan(Dual x) { return x.d; }

}  // namespace gbpme
