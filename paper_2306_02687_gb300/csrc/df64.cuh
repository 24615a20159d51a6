// df64.cuh -- double-float arithmetic on the float32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (about 48 significand bits).  GB300 executes float32 FMAs at ~73x the
// float64 rate, so the float64-accurate parts of the mixed form (micro
// kinematics, micro law, reduced residual, homogenized stress) run in this
// representation.  Building blocks are the error-free transformations of
// Knuth (TwoSum), Dekker (Fast2Sum) and the FMA-based exact product
// (TwoProd).  Every operation uses the *_rn intrinsics so that the compiler
// can neither contract nor reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace rverom {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

__device__ __forceinline__ df df_from(double x) {
    const float h = __double2float_rn(x);
    return df{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_div(df a, df b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

// Accumulator of a double-float dot product: hi carries the running sum of
// the leading products (TwoSum keeps its rounding error), lo collects the
// product errors, the cross terms and the TwoSum errors; normalize at the end.
struct dacc {
    float hi, lo;
};

__device__ __forceinline__ void dacc_fma(dacc &s, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const df t = two_sum(s.hi, p);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ df dacc_get(const dacc &s) { return fast_two_sum(s.hi, s.lo); }

// Natural logarithm of x > 0 to 3e-14 relative (2.4e-14 measured against
// float64 log over [0.5, 2]): x = 2^k m with
// m in [1/sqrt2, sqrt2), ln m = 2 atanh(t), t = (m - 1)/(m + 1), |t| < 0.172,
// 2 atanh(t) = 2t (1 + t^2/3 + t^4/5 + t^6/7 + t^8 R(t^2)); the first terms in
// double-float, the remainder R = 1/9 + t^2/11 + ... + t^8/17 in float32
// (its contribution is below 3e-5 relative, so float32 suffices).
__device__ __forceinline__ df df_log(df x) {
    int k;
    float m = frexpf(x.hi, &k);  // x.hi = m 2^k, m in [0.5, 1)
    if (m < 0.70710678f) {
        k -= 1;
    }
    const df xm = df{ldexpf(x.hi, -k), ldexpf(x.lo, -k)};
    const df num = df_add_f(xm, -1.0f);
    const df den = df_add_f(xm, 1.0f);
    const df t = df_div(num, den);
    const df t2 = df_mul(t, t);
    const float z = t2.hi;
    const float R = __fmaf_rn(z, __fmaf_rn(z, __fmaf_rn(z, __fmaf_rn(z, 1.0f / 17.0f, 1.0f / 15.0f), 1.0f / 13.0f),
                                          1.0f / 11.0f),
                              1.0f / 9.0f);
    const df c7 = df{0x1.24924ap-3f, -0x1.b6db6ep-28f};  // 1/7
    const df c5 = df{0x1.99999ap-3f, -0x1.99999ap-29f};  // 1/5
    const df c3 = df{0x1.555556p-2f, -0x1.555556p-27f};  // 1/3
    df S = df_add(c7, df_mul_f(t2, R));
    S = df_add(c5, df_mul(t2, S));
    S = df_add(c3, df_mul(t2, S));
    S = df_add_f(df_mul(t2, S), 1.0f);
    df l = df_mul(t, S);
    l = df{2.0f * l.hi, 2.0f * l.lo};
    if (k != 0) {
        const df ln2 = df{0x1.62e43p-1f, -0x1.05c61p-29f};  // ln 2
        l = df_add(l, df_mul_f(ln2, (float)k));
    }
    return l;
}

}  // namespace rverom
