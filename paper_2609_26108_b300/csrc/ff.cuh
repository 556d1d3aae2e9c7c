// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
// Built from the error-free transformations of Knuth (two-sum) and Dekker
// (two-product, here with one fused multiply-add); the algorithms follow
// Hida, Li and Bailey's double-double library, transposed to float pairs.
// The cache build uses it for the root refinement and the ray quantities,
// which need more than float precision: on this part FP64 instructions issue
// at a small fraction of the float rate, while these run on the float pipes.
//
// The type lives in its own namespace so that its overloads of fabs, fmax,
// ... are found by argument-dependent lookup only, never in place of the
// float and double functions.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace chert {
namespace xf {

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit ff(int v) : hi(float(v)), lo(float(v - int(float(v)))) {}
    __host__ __device__ constexpr explicit ff(float v) : hi(v), lo(0.0f) {}
    __host__ __device__ constexpr explicit ff(double v)
        : hi(float(v)), lo(float(v) - float(v) == 0.0f ? float(v - double(float(v))) : 0.0f) {}
    __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return ff(s, (a - (s - bb)) + (b - bb));
}
// s + e = a + b exactly, given |a| >= |b|
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    const float s = a + b;
    return ff(s, b - (s - a));
}
// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    return ff(p, fmaf(a, b, -p));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }

// IEEE-style addition (accurate also under cancellation)
__device__ __forceinline__ ff operator+(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
// ff + float: the float joins with one two-sum
__device__ __forceinline__ ff operator+(ff a, float b) {
    ff s = two_sum(a.hi, b);
    s.lo += a.lo;
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff operator*(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff operator*(ff a, float b) {
    ff p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}

// Long division: three float quotients, each correcting the remainder of the
// previous ones.
__device__ __forceinline__ ff operator/(ff a, ff b) {
    const float q1 = a.hi / b.hi;
    ff r = a - b * q1;
    const float q2 = r.hi / b.hi;
    r = r - b * q2;
    const float q3 = r.hi / b.hi;
    const ff q = quick_two_sum(q1, q2);
    return q + ff(q3);
}

__device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(ff a, ff b) { return b < a; }
__device__ __forceinline__ bool operator<=(ff a, ff b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
__device__ __forceinline__ bool operator>=(ff a, ff b) { return b <= a; }
__device__ __forceinline__ bool operator==(ff a, ff b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(ff a, ff b) { return !(a == b); }

__device__ __forceinline__ ff fabs(ff a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ ff fmax(ff a, ff b) { return (a < b || a.hi != a.hi) ? b : a; }
__device__ __forceinline__ ff fmin(ff a, ff b) { return (b < a || a.hi != a.hi) ? b : a; }
__device__ __forceinline__ bool isfinite(ff a) { return ::isfinite(a.hi); }
__device__ __forceinline__ bool signbit(ff a) { return ::signbit(a.hi); }
__device__ __forceinline__ ff copysign(ff a, ff s) { return ::signbit(a.hi) == ::signbit(s.hi) ? a : -a; }

// Square root: one Newton correction of the float root, q + (a - q^2)/(2q).
__device__ __forceinline__ ff sq(ff a) {
    if (!(a.hi > 0.0f)) return ff(a.hi == 0.0f ? 0.0f : sqrtf(a.hi), 0.0f);
    const float q = sqrtf(a.hi);
    const ff p = two_prod(q, q);
    const float r = ((a.hi - p.hi) - p.lo + a.lo) / (2.0f * q);
    return quick_two_sum(q, r);
}
__device__ __forceinline__ ff hyp(ff x, ff y) { return sq(x * x + y * y); }

// cosh and sinh by their Maclaurin series in x^2 (Horner; coefficients 1/k!
// as compile-time float pairs), for the imaginary slowness angles of the scan
// (|x| <= 0.6: the first omitted term is below 1e-18); larger arguments,
// outside the scan range of any cache in use, go through double.
__device__ __forceinline__ ff ch_(ff x) {
    if (!(::fabsf(x.hi) <= 0.6f)) return ff(::cosh(double(x)));
    constexpr ff c16(1.0 / 20922789888000.0), c14(1.0 / 87178291200.0), c12(1.0 / 479001600.0),
        c10(1.0 / 3628800.0), c8(1.0 / 40320.0), c6(1.0 / 720.0), c4(1.0 / 24.0);
    const ff x2 = x * x;
    ff s = c16;
    s = s * x2 + c14;
    s = s * x2 + c12;
    s = s * x2 + c10;
    s = s * x2 + c8;
    s = s * x2 + c6;
    s = s * x2 + c4;
    s = s * x2 + ff(0.5f);
    return s * x2 + ff(1.0f);
}
__device__ __forceinline__ ff sh_(ff x) {
    if (!(::fabsf(x.hi) <= 0.6f)) return ff(::sinh(double(x)));
    constexpr ff c15(1.0 / 1307674368000.0), c13(1.0 / 6227020800.0), c11(1.0 / 39916800.0),
        c9(1.0 / 362880.0), c7(1.0 / 5040.0), c5(1.0 / 120.0), c3(1.0 / 6.0);
    const ff x2 = x * x;
    ff s = c15;
    s = s * x2 + c13;
    s = s * x2 + c11;
    s = s * x2 + c9;
    s = s * x2 + c7;
    s = s * x2 + c5;
    s = s * x2 + c3;
    s = s * x2 + ff(1.0f);
    return s * x;
}

__device__ __forceinline__ ff shfl(ff v, int src) {
    return ff(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}

}  // namespace xf
}  // namespace chert
