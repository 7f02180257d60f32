// Double-float arithmetic on the FP32 pipe.
//
// A dfloat is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// i.e. a 48-bit significand (relative rounding ~3.6e-15) with the exponent range
// of float.  Sums use Knuth's TwoSum and products Dekker's exact product via
// FMA (a*b = p + e, e = fma(a, b, -p)).  On GB300 an FP64 FMA issues at 1/64 of
// the FP32 rate, so FP64-class precision is cheaper this way for FMA-heavy code.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace sfhk {
// Own namespace so that these overloads are found by argument-dependent lookup
// only and do not hide the float/double math functions inside sfhk.
namespace dfns {

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __device__ __forceinline__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ dfloat(float x) : hi(x), lo(0.f) {}
    __device__ __forceinline__ dfloat(int x) : hi((float)x), lo(0.f) {}
    __device__ __forceinline__ dfloat(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly, |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e += t;
    fast_two_sum(s, e, s, e);
    e += f;
    fast_two_sum(s, e, s, e);
    return dfloat(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    fast_two_sum(p, e, s, t);
    return dfloat(s, t);
}
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
    // one correction of the float quotient
    const float q1 = a.hi / b.hi;
    const dfloat r = a - b * dfloat(q1);
    const float q2 = r.hi / b.hi;
    float s, t;
    fast_two_sum(q1, q2, s, t);
    return dfloat(s, t);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return b < a; }
__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return !(a == b); }
__device__ __forceinline__ bool isfinite(dfloat a) { return ::isfinite(a.hi); }
__device__ __forceinline__ dfloat fabs(dfloat a) { return a.hi < 0.f ? -a : a; }

// 1/sqrt(x): float estimate and one Newton step in double-float
__device__ __forceinline__ dfloat rsq(dfloat x) {
    const float y0 = rsqrtf(x.hi);
    const dfloat y(y0);
    const dfloat r = dfloat(1.0f) - x * (y * y);          // ~2^-23
    return y + y * (dfloat(0.5f) * r);
}
__device__ __forceinline__ dfloat sqrt(dfloat x) { return x.hi > 0.f ? x * rsq(x) : dfloat(0.f); }

// exp(x) = 2^k exp(r), r = x - k ln2 (double-float ln2), exp(r) by a Taylor
// series of r/8 (|r/8| <= 0.044, ten terms, truncation < 1e-19) squared three
// times; double-float coefficients 1/n.
__device__ __forceinline__ dfloat ex(dfloat x) {
    if (x.hi < -87.f) return dfloat(0.f);
    const float k = rintf(x.hi * 1.44269504f);
    const dfloat ln2(0.693147182f, -1.90465421e-09f);        // ln 2 = hi + lo
    dfloat r = x - dfloat(k) * ln2;
    r = r * dfloat(0.125f);
    dfloat t = dfloat(1.0f) + r * dfloat(1.0 / 10.0);
    t = dfloat(1.0f) + r * t * dfloat(1.0 / 9.0);
    t = dfloat(1.0f) + r * t * dfloat(0.125);
    t = dfloat(1.0f) + r * t * dfloat(1.0 / 7.0);
    t = dfloat(1.0f) + r * t * dfloat(1.0 / 6.0);
    t = dfloat(1.0f) + r * t * dfloat(0.2);
    t = dfloat(1.0f) + r * t * dfloat(0.25);
    t = dfloat(1.0f) + r * t * dfloat(1.0 / 3.0);
    t = dfloat(1.0f) + r * t * dfloat(0.5);
    t = dfloat(1.0f) + r * t;
    t = t * t;
    t = t * t;
    t = t * t;
    const float sc = __int_as_float((127 + (int)k) << 23);  // 2^k (|k| <= 126)
    return dfloat(t.hi * sc, t.lo * sc);
}

}  // namespace dfns
using dfns::dfloat;
}  // namespace sfhk
