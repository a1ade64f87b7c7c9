// Complex arithmetic on float2 / double2 and small device utilities.
#pragma once

#include <cuda_runtime.h>

namespace mb {

template <typename R> struct V2;
template <> struct V2<float> { typedef float2 T; };
template <> struct V2<double> { typedef double2 T; };

__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }

template <typename T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 &operator+=(float2 &a, float2 b) { a.x += b.x; a.y += b.y; return a; }
__device__ __forceinline__ double2 &operator+=(double2 &a, double2 b) { a.x += b.x; a.y += b.y; return a; }

// complex * complex
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmul_c(float2 a, float2 b) { return cmulc(b, a); }
__device__ __forceinline__ double2 cmul_c(double2 a, double2 b) { return cmulc(b, a); }
// acc += a * b
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += r * a (real r)
__device__ __forceinline__ void rfma(float2 &acc, float r, float2 a) {
    acc.x = fmaf(r, a.x, acc.x);
    acc.y = fmaf(r, a.y, acc.y);
}
__device__ __forceinline__ void rfma(double2 &acc, double r, double2 a) {
    acc.x = fma(r, a.x, acc.x);
    acc.y = fma(r, a.y, acc.y);
}
__device__ __forceinline__ float2 rscale(float r, float2 a) { return make_float2(r * a.x, r * a.y); }
__device__ __forceinline__ double2 rscale(double r, double2 a) { return make_double2(r * a.x, r * a.y); }

}  // namespace mb
