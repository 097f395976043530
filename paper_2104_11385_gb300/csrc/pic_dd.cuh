// pic_dd.cuh -- float-float ("double-float") arithmetic for the mixed-precision
// particle push.  A value is hi + lo with two FP32 numbers, |lo| <= ulp(hi)/2,
// about 48 significant bits (relative resolution 2^-48 ~ 3.6e-15).  Sums use
// Knuth's TwoSum and products the FMA-based TwoProd (Dekker 1971; Shewchuk
// 1997; Hida, Li & Bailey's double-double with float limbs), so each operation
// costs a handful of FP32 instructions instead of one FP64 instruction issued
// at 1/64 of the FP32 rate on GB300.  Conversions between double and float-
// float work on the bit patterns with integer instructions.
#pragma once
#include <cuda_runtime.h>

struct dd {
    float h, l;
};

// ---- error-free transformations
// Every FP32 step is an explicit round-to-nearest intrinsic: the compiler
// contracts a plain a * b + c into one FMA, which would let a sum see an
// unrounded product and break the exactness these transformations rely on.
__device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return dd{s, e};
}

__device__ __forceinline__ dd dd_quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// ---- conversions
// The FP64 routes of the conversions below are separate functions: inlined,
// the compiler predicates them and their FP64 instructions (which include the
// double <-> float conversions) then occupy the FP64 pipe on every call.
static __device__ __noinline__ dd dd_from_slow(double x) {
    const float h = __double2float_rn(x);
    return dd{h, __double2float_rn(x - (double)h)};
}
static __device__ __noinline__ double dd_to_slow(float h, float l) { return (double)h + (double)l; }

// double -> float-float by integer work on the IEEE-754 bits (every FP64
// instruction, conversions included, issues at the FP64 rate): hi is x rounded
// to 24 bits (ties away from zero on the magnitude), lo the remainder in units
// of 2^(e-52), at most 2^28 of them, rounded to 24 bits by one int->float
// conversion and scaled by adding to its exponent field.  |x - (hi + lo)| <=
// 2^-49 |x|.  Magnitudes outside [2^-74, 2^127) (where lo would leave the
// normal float range) take the two-conversion FP64 route; zero is exact.
__device__ __forceinline__ dd dd_from(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long u = b & 0x7FFFFFFFFFFFFFFFull;
    const int be = (int)(u >> 52);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    if (be >= 1023 - 74 && be <= 1023 + 126) {
        const unsigned long long hb = (u + (1ull << 28)) >> 29;  // exponent | 23-bit mantissa
        const float h = __uint_as_float(sgn | (unsigned)(hb - (896ull << 23)));
        // the bit patterns are linear in the value with slope 2^(e-52) up to
        // the binade above, so the pattern difference is the remainder
        const int d = (int)(long long)(u - (hb << 29));
        float l = 0.0f;
        if (d != 0)
            l = __uint_as_float((__float_as_uint(__int2float_rn(d)) + ((unsigned)(be - 1023 - 52) << 23)) ^ sgn);
        return dd{h, l};
    }
    if (u == 0ull) return dd{__uint_as_float(sgn), 0.0f};
    return dd_from_slow(x);
}

// float-float -> double by integer work, after one normalising TwoSum: hi
// widened exactly (exponent rebias, mantissa << 29), lo added in units of the
// double ulp of hi (truncated), with the pattern arithmetic of dd_from; a hi
// that is a power of two and a lo of the other sign land in the binade below,
// where the unit is half as large.  A hi or lo outside the normal float range
// takes the FP64 route.
__device__ __forceinline__ double dd_to(dd a) {
    a = dd_two_sum(a.h, a.l);
    const unsigned hb = __float_as_uint(a.h), lb = __float_as_uint(a.l);
    const int he = (int)((hb >> 23) & 0xFFu), le = (int)((lb >> 23) & 0xFFu);
    if (he >= 1 && he <= 254) {
        unsigned long long mag = ((unsigned long long)(hb & 0x7FFFFFFFu) + (896ull << 23)) << 29;
        if ((lb & 0x7FFFFFFFu) != 0u) {
            int sh = le - he + 29;
            if (le == 0 || sh > 5) return dd_to_slow(a.h, a.l);
            const unsigned long long ml = (unsigned long long)((lb & 0x7FFFFFu) | 0x800000u);
            const bool sub = ((hb ^ lb) & 0x80000000u) != 0u;
            if (sub && (hb & 0x7FFFFFu) == 0u) sh += 1;
            const unsigned long long dl = sh >= 0 ? (ml << sh) : (sh > -25 ? (ml >> (-sh)) : 0ull);
            mag = sub ? mag - dl : mag + dl;
        }
        return __longlong_as_double((long long)(mag | ((unsigned long long)(hb & 0x80000000u) << 32)));
    }
    return dd_to_slow(a.h, a.l);
}
__host__ __device__ constexpr dd dd_const(double x) {
    return dd{static_cast<float>(x), static_cast<float>(x - static_cast<double>(static_cast<float>(x)))};
}

// float-float -> double, branch-free after one normalising TwoSum: the form
// dd_to takes in the current deposit, where it runs dozens of times per
// particle.  Float subnormals flush to zero (|hi| below 2^-126
// gives 0, a subnormal lo is dropped: an absolute error below 2^-126).
__device__ __forceinline__ double dd_to_norm(dd a) {
    a = dd_two_sum(a.h, a.l);
    const unsigned hb = __float_as_uint(a.h), lb = __float_as_uint(a.l);
    const unsigned ha = hb & 0x7FFFFFFFu;
    unsigned long long mag = ((unsigned long long)ha + (896ull << 23)) << 29;
    const int sh0 = (int)((lb >> 23) & 0xFFu) - (int)(ha >> 23) + 29;
    const bool sub = ((hb ^ lb) & 0x80000000u) != 0u;
    const int sh = sh0 + ((sub && (ha & 0x7FFFFFu) == 0u) ? 1 : 0);
    const unsigned long long ml = (lb & 0x7F800000u) ? (unsigned long long)((lb & 0x7FFFFFu) | 0x800000u) : 0ull;
    const unsigned long long dl = sh >= 0 ? (ml << sh) : (ml >> min(-sh, 63));
    mag = sub ? mag - dl : mag + dl;
    mag = (ha >= 0x00800000u) ? mag : 0ull;
    return __longlong_as_double((long long)(mag | ((unsigned long long)(hb & 0x80000000u) << 32)));
}

// ---- arithmetic
// Chained operations leave the pair unnormalised (|lo| may reach a few
// ulp(hi)): TwoSum and TwoProd are exact for any operands, so the value stays
// hi + lo to about 2^-46 relative while each add saves 3 instructions and
// each product 3.  dd_norm (a TwoSum, exact whatever the magnitudes)
// restores |lo| <= ulp(hi)/2 where a conversion or an estimate needs it.
__device__ __forceinline__ dd dd_norm(dd a) { return dd_two_sum(a.h, a.l); }
__device__ __forceinline__ dd operator+(dd a, dd b) {
    const dd s = dd_two_sum(a.h, b.h);
    return dd{s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ dd operator-(dd a) { return dd{-a.h, -a.l}; }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return dd{p, e};
}
// a * b + c
__device__ __forceinline__ dd fma(dd a, dd b, dd c) { return a * b + c; }

// 1/sqrt(x): FP32 estimate refined by one Newton step in float-float
__device__ __forceinline__ dd dd_rsqrt(dd x) {
    x = dd_norm(x);
    const float y0 = rsqrtf(x.h);
    const dd y{y0, 0.0f};
    const dd r = dd_const(1.0) - x * (y * y);  // residual ~ 2^-22
    return y + y * (dd{0.5f, 0.0f} * r);
}

// 1/x: FP32 estimate refined by one Newton step in float-float
__device__ __forceinline__ dd dd_rcp(dd x) {
    x = dd_norm(x);
    const float y0 = __frcp_rn(x.h);
    const dd y{y0, 0.0f};
    const dd r = dd_const(1.0) - x * y;
    return y + y * r;
}

// ---- plain FP32 (the FP32 variant): conversions by integer work as well
static __device__ __noinline__ float f32_from_slow(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double f64_from_slow(float f) { return (double)f; }

// double -> float, rounded to 24 bits (ties away from zero on the magnitude)
// on the bit pattern; zero, and magnitudes outside [2^-100, 2^127), take the
// conversion instruction out of line
__device__ __forceinline__ float f32_from(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long u = b & 0x7FFFFFFFFFFFFFFFull;
    const int be = (int)(u >> 52);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    if (be >= 1023 - 100 && be <= 1023 + 126)
        return __uint_as_float(sgn | (unsigned)(((u + (1ull << 28)) >> 29) - (896ull << 23)));
    if (u == 0ull) return __uint_as_float(sgn);
    return f32_from_slow(x);
}

// float -> double, exact: exponent rebias and mantissa << 29 for normal floats
__device__ __forceinline__ double f64_from(float f) {
    const unsigned b = __float_as_uint(f), a = b & 0x7FFFFFFFu;
    const unsigned long long sg = (unsigned long long)(b & 0x80000000u) << 32;
    if (a >= 0x00800000u && a < 0x7F800000u)
        return __longlong_as_double((long long)(sg | (((unsigned long long)a + (896ull << 23)) << 29)));
    if (a == 0u) return __longlong_as_double((long long)sg);
    return f64_from_slow(f);
}

// ---- one arithmetic interface for double and dd
template <class R>
struct Arith;

template <>
struct Arith<double> {
    __device__ static __forceinline__ double from(double x) { return x; }
    __device__ static __forceinline__ double to(double x) { return x; }
    // 1/sqrt(x) for x >= 1 (1 + |u|^2): the hardware estimate refined by two
    // Newton-Raphson steps y <- y + y (1/2 - (x/2) y^2), each squaring the
    // relative error, to about 1 ulp
    __device__ static __forceinline__ double rsqrt(double x) {
        double y;
        asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
        const double hx = 0.5 * x;
        y = ::fma(y, ::fma(-hx * y, y, 0.5), y);
        y = ::fma(y, ::fma(-hx * y, y, 0.5), y);
        return y;
    }
    __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
    // 2/x for x >= 1: the hardware reciprocal estimate refined by two
    // Newton-Raphson steps (e = 1 - x y, y <- y + y e; each squares the
    // relative error), about 1 ulp, with fewer FP64 instructions than the
    // correctly rounded division
    __device__ static __forceinline__ double two_over(double x) {
        double y;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
        y = ::fma(y, ::fma(-x, y, 1.0), y);
        y = ::fma(y, ::fma(-x, y, 1.0), y);
        return 2.0 * y;
    }
    __device__ static __forceinline__ double c(double x) { return x; }
};

template <>
struct Arith<float> {
    __device__ static __forceinline__ float from(double x) { return f32_from(x); }
    __device__ static __forceinline__ double to(float x) { return f64_from(x); }
    __device__ static __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    __device__ static __forceinline__ float rcp(float x) { return __frcp_rn(x); }
    __device__ static __forceinline__ float two_over(float x) { return 2.0f * __frcp_rn(x); }
    __device__ static __forceinline__ float c(double x) { return static_cast<float>(x); }
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
