// pic_dd.cuh -- float-float ("double-float") arithmetic for the mixed-precision
// particle push.  A value is hi + lo with two FP32 numbers, |lo| <= ulp(hi)/2,
// about 48 significant bits (relative resolution 2^-48 ~ 3.6e-15).  Sums use
// Knuth's TwoSum and products the FMA-based TwoProd (Dekker 1971; Shewchuk
// 1997; Hida, Li & Bailey's double-double with float limbs), so each operation
// costs a handful of FP32 instructions instead of one FP64 instruction issued
// at 1/64 of the FP32 rate on GB300.  Conversions between double and float run
// at FP32 speed; only the split of a double needs one FP64 subtraction.
#pragma once
#include <cuda_runtime.h>

struct dd {
    float h, l;
};

// ---- error-free transformations
__device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    const float e = (a - (s - v)) + (b - v);
    return dd{s, e};
}

__device__ __forceinline__ dd dd_quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return dd{s, b - (s - a)};
}

// ---- conversions
__device__ __forceinline__ dd dd_from(double x) {
    const float h = __double2float_rn(x);
    return dd{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dd_to(dd a) { return (double)a.h + (double)a.l; }
__host__ __device__ constexpr dd dd_const(double x) {
    return dd{static_cast<float>(x), static_cast<float>(x - static_cast<double>(static_cast<float>(x)))};
}

// ---- arithmetic
__device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return dd_quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ dd operator-(dd a) { return dd{-a.h, -a.l}; }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return dd_quick_two_sum(p, e);
}
// a * b + c
__device__ __forceinline__ dd fma(dd a, dd b, dd c) { return a * b + c; }

// 1/sqrt(x): FP32 estimate refined by one Newton step in float-float
__device__ __forceinline__ dd dd_rsqrt(dd x) {
    const float y0 = rsqrtf(x.h);
    const dd y{y0, 0.0f};
    const dd r = dd_const(1.0) - x * (y * y);  // residual ~ 2^-22
    return y + y * (dd{0.5f, 0.0f} * r);
}

// 1/x: FP32 estimate refined by one Newton step in float-float
__device__ __forceinline__ dd dd_rcp(dd x) {
    const float y0 = __frcp_rn(x.h);
    const dd y{y0, 0.0f};
    const dd r = dd_const(1.0) - x * y;
    return y + y * r;
}

// ---- one arithmetic interface for double and dd
template <class R>
struct Arith;

template <>
struct Arith<double> {
    __device__ static __forceinline__ double from(double x) { return x; }
    __device__ static __forceinline__ double to(double x) { return x; }
    __device__ static __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
    __device__ static __forceinline__ double two_over(double x) { return 2.0 / x; }
    __device__ static __forceinline__ double c(double x) { return x; }
};

template <>
struct Arith<dd> {
    __device__ static __forceinline__ dd from(double x) { return dd_from(x); }
    __device__ static __forceinline__ double to(dd x) { return dd_to(x); }
    __device__ static __forceinline__ dd rsqrt(dd x) { return dd_rsqrt(x); }
    __device__ static __forceinline__ dd rcp(dd x) { return dd_rcp(x); }
    __device__ static __forceinline__ dd two_over(dd x) { return dd_const(2.0) * dd_rcp(x); }
    __device__ static __forceinline__ dd c(double x) { return dd_const(x); }
};
