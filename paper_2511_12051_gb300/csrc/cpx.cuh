// Small complex type for device code, templated on the real type so that the
// same phase-linking code runs in single and double precision.
#pragma once

#include <cuda_runtime.h>

namespace plk {

template <class T>
struct __align__(2 * sizeof(T)) cpx {
    T x, y;
};

template <class T>
__device__ __forceinline__ cpx<T> mk(T x, T y) { cpx<T> r; r.x = x; r.y = y; return r; }

template <class T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <class T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <class T>
__device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T>
__device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.x, s * a.y); }
template <class T>
__device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }
template <class T>
__device__ __forceinline__ T norm2(cpx<T> a) { return a.x * a.x + a.y * a.y; }
// c - a * b
template <class T>
__device__ __forceinline__ cpx<T> cfms(cpx<T> a, cpx<T> b, cpx<T> c) {
    return mk(c.x - a.x * b.x + a.y * b.y, c.y - a.x * b.y - a.y * b.x);
}
// c + a * b
template <class T>
__device__ __forceinline__ cpx<T> cfma(cpx<T> a, cpx<T> b, cpx<T> c) {
    return mk(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
// c + a * conj(b)
template <class T>
__device__ __forceinline__ cpx<T> cfma_conj(cpx<T> a, cpx<T> b, cpx<T> c) {
    return mk(c.x + a.x * b.x + a.y * b.y, c.y + a.y * b.x - a.x * b.y);
}

__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }
__device__ __forceinline__ float sqrt_t(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_t(double v) { return sqrt(v); }
__device__ __forceinline__ float atan2_t(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double atan2_t(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float abs_t(float v) { return fabsf(v); }
__device__ __forceinline__ double abs_t(double v) { return fabs(v); }

}  // namespace plk
