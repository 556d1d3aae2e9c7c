// Small complex arithmetic for the device kernels, templated on float/double.
// Built from the CUDA real math functions; the principal square root uses the
// half-angle identities sqrt(z) = t + i y/(2t), t = sqrt((|z| + x)/2) for x >= 0
// (and the mirrored form for x < 0), so no cancellation occurs in either case.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace chert {

template <typename T>
struct cplx {
    T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T r, T i) { return cplx<T>{r, i}; }

template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

// a / b by the textbook formula a * conj(b) / |b|^2 (magnitudes here stay far
// from the float range limits: moduli ~1e7, velocities ~1e3).
template <typename T>
__device__ __forceinline__ cplx<T> operator/(cplx<T> a, cplx<T> b) {
    T d = T(1) / norm2(b);
    return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}

__device__ __forceinline__ float hyp(float x, float y) { return hypotf(x, y); }
__device__ __forceinline__ double hyp(double x, double y) { return hypot(x, y); }
__device__ __forceinline__ float sq(float x) { return sqrtf(x); }
__device__ __forceinline__ double sq(double x) { return sqrt(x); }

// Principal square root (Re >= 0).
template <typename T>
__device__ __forceinline__ cplx<T> csqrt(cplx<T> z) {
    T r = hyp(z.re, z.im);
    if (r == T(0)) return {T(0), T(0)};
    if (z.re >= T(0)) {
        T t = sq(T(0.5) * (r + z.re));
        return {t, z.im / (T(2) * t)};
    }
    T t = sq(T(0.5) * (r - z.re));
    return {fabs(z.im) / (T(2) * t), copysign(t, z.im)};
}

}  // namespace chert
