// Double-float arithmetic: a value is hi + lo with two FP32 numbers (|lo| <= ulp(hi)/2),
// a 48-bit significand computed on the FP32 pipes. Error-free transforms after Dekker
// (1971) and Knuth (TAOCP vol. 2): TwoSum, FastTwoSum, and the FMA form of TwoProduct.
// The __f*_rn intrinsics keep the compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

struct __align__(8) df {
    float hi, lo;
};

// Conversion from FP64 (rounds to the nearest pair).
__host__ __device__ __forceinline__ df df_from_d(double x) {
    float h = (float)x;
    float l = (float)(x - (double)h);
    return df{h, l};
}

#if defined(__CUDACC__)
__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// a + b = s + e exactly (no precondition on |a|, |b|)
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// a + b = s + e exactly when |a| >= |b|
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// k + a for a small float constant k, in 4 instead of 10 operations. The high parts go
// through FastTwoSum with k as the leading operand, which is error-free when
// |k| >= |a.hi|; where |k| < |a.hi| the call sites' operands make k + a.hi itself
// representable (k an integer and |a.hi| >= 1, or Sterbenz: |a.hi| <= 2 |k|), and the
// error term then comes out exactly zero. Either way hi + e = k + a.hi exactly; only the
// final e + a.lo rounds. The pair is not renormalised (|lo| may reach ulp(hi)), which the
// products and sums downstream absorb (their error terms carry the low part).
__device__ __forceinline__ df df_add_exact_const(df a, float k) {
    const float s = __fadd_rn(k, a.hi);
    const float e = __fsub_rn(a.hi, __fsub_rn(s, k));
    return df{s, __fadd_rn(e, a.lo)};
}

__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

// a * b left as the pair {p, e} without the final FastTwoSum (|e| up to about 3 ulp(p) / 2
// instead of ulp(p) / 2), for products that feed further double-float products and sums:
// their error terms carry the larger low part, and the neglected lo * lo term grows from
// 2^-48 to about 2^-45 of the product.
__device__ __forceinline__ df df_mul_raw(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df{p, e};
}

__device__ __forceinline__ df df_mul_f_raw(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df{p, e};
}

// a * b + c (the sum renormalises, so the product need not)
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul_raw(a, b), c); }

__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_ge(df a, df b) { return !df_lt(a, b); }

__device__ __forceinline__ double df_to_d(df a) { return (double)a.hi + (double)a.lo; }

// Accumulator of double-float products sum_k w_k v_k: the high parts are added exactly
// (TwoSum), the low parts and the product errors in plain FP32; one renormalisation at
// the end. Same error bound as repeated df_fma, 12 instead of 18 FP32 operations a term.
struct dacc {
    float s, lo;
};

__device__ __forceinline__ dacc dacc_prod(df w, df v) {
    const float p = __fmul_rn(w.hi, v.hi);
    float e = __fmaf_rn(w.hi, v.hi, -p);
    e = __fmaf_rn(w.hi, v.lo, e);
    e = __fmaf_rn(w.lo, v.hi, e);
    return dacc{p, e};
}

__device__ __forceinline__ void dacc_add(dacc& a, df w, df v) {
    const dacc t = dacc_prod(w, v);
    const df s = two_sum(a.s, t.s);
    a.s = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ void dacc_add_df(dacc& a, df x) {
    const df s = two_sum(a.s, x.hi);
    a.s = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ df dacc_get(dacc a) { return fast_two_sum(a.s, a.lo); }

// The accumulated value as a pair without renormalising (|lo| a few ulps of s): exact as a
// sum, and fine as an operand of products and of df_add / dacc_add, whose error terms
// absorb the larger low part (error <= n 2^-48 relative for an n-term sum).
__device__ __forceinline__ df dacc_raw(dacc a) { return df{a.s, a.lo}; }
#endif
