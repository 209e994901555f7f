// Complex helpers on CUDA vector types (double2 / float2 = re, im).
#pragma once
#include <cuda_runtime.h>

template <typename T2>
struct RealOf;
template <>
struct RealOf<double2> {
  using T = double;
};
template <>
struct RealOf<float2> {
  using T = float;
};

template <typename R>
struct Cplx;
template <>
struct Cplx<double> {
  using T = double2;
};
template <>
struct Cplx<float> {
  using T = float2;
};

__host__ __device__ __forceinline__ double2 mk(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ float2 mk(float re, float im) { return make_float2(re, im); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cjmul(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cjmul(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// c + a * b
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
// 1 / z as conj(z) / |z|^2 (IEEE division of the real scale).
__host__ __device__ __forceinline__ double2 crcp(double2 z) {
  double d = 1.0 / (z.x * z.x + z.y * z.y);
  return make_double2(z.x * d, -z.y * d);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return cmul(a, crcp(b)); }
__host__ __device__ __forceinline__ float2 crcp(float2 z) {
  float d = 1.0f / (z.x * z.x + z.y * z.y);
  return make_float2(z.x * d, -z.y * d);
}
__host__ __device__ __forceinline__ float2 cdiv(float2 a, float2 b) { return cmul(a, crcp(b)); }

__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename T2>
__host__ __device__ __forceinline__ T2 from_d2(double2 a);
template <>
__host__ __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <>
__host__ __device__ __forceinline__ float2 from_d2<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// FP32 arithmetic on vectors stored in either precision (no FP64 work when
// the storage is FP32)
__host__ __device__ __forceinline__ float2 to_f2(float2 a) { return a; }
__host__ __device__ __forceinline__ float2 to_f2(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <typename T2>
__host__ __device__ __forceinline__ T2 from_f2(float2 a);
template <>
__host__ __device__ __forceinline__ float2 from_f2<float2>(float2 a) { return a; }
template <>
__host__ __device__ __forceinline__ double2 from_f2<double2>(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ float2 add_f2(float2 o, float2 x) { return make_float2(o.x + x.x, o.y + x.y); }
__host__ __device__ __forceinline__ double2 add_f2(double2 o, float2 x) { return make_double2(o.x + x.x, o.y + x.y); }

// Convert a double2 coefficient to the vector type T2.
template <typename T2>
__host__ __device__ __forceinline__ T2 cvt(double2 a) {
  return from_d2<T2>(a);
}
