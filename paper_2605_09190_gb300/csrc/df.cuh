// df.cuh -- double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (normalised), giving ~48 significant bits.  GB300's FP64 rate is a small
// fraction of its FP32 rate, so the pursuit keeps its state in this form.
// The building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (Fast2Sum) and the FMA-based exact product (TwoProd); every
// operation below uses explicitly rounded intrinsics so the compiler can
// neither contract nor reassociate them.
#pragma once
#include <cstdint>

struct df {
    float hi, lo;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly, valid when |a| >= |b| or a == 0 (Dekker).
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// p + e = a * b exactly (one FMA recovers the rounding error).
__device__ __forceinline__ df df_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// a * b for double-float operands; relative error ~2^-46.
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = df_two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p.hi, e);
}

// a + b with an absolute error ~2^-47 (|a| + |b|): the high words are added
// exactly, the low words in one rounding.  Cancellation of the high words is
// exact, so the error stays small relative to the operands, which is the
// bound the pursuit's certification uses.
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// c - u * w, the correlation update of one Gram entry, in one pass.
__device__ __forceinline__ df df_sub_mul(df c, df u, df w) {
    float p = __fmul_rn(u.hi, w.hi);
    float pe = __fmaf_rn(u.hi, w.hi, -p);
    pe = __fmaf_rn(u.hi, w.lo, pe);
    pe = __fmaf_rn(u.lo, w.hi, pe);
    df s = df_two_sum(c.hi, -p);
    float e = __fadd_rn(s.lo, __fsub_rn(c.lo, pe));
    return df_fast_two_sum(s.hi, e);
}

// Exact conversion of an integer with |v| < 2^48 to double-float.
__device__ __forceinline__ df df_from_i64(long long v) {
    float hi = __ll2float_rn(v);
    long long rem = v - (long long)hi;          // |rem| <= 2^23: exact in a float
    return df_fast_two_sum(hi, __ll2float_rn(rem));
}

// x + b for a float b, rounded once into a normalised pair.
__device__ __forceinline__ df df_add_float(df x, float b) {
    df s = df_two_sum(x.hi, b);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ df df_scale(df a, float pow2) {   // multiply by a power of two
    return {__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// a < b for normalised operands (lexicographic on (hi, lo)).
__device__ __forceinline__ bool df_lt(df a, df b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// Order-preserving 64-bit key of |a|: (bits(|hi|), monotone bits of
// sign(hi) * lo).  Comparing keys as unsigned integers compares |a|.
__device__ __forceinline__ unsigned long long df_abs_key(df a) {
    uint32_t h = __float_as_uint(a.hi);
    uint32_t ah = h & 0x7fffffffu;
    if (ah == 0u) return 0ull;
    uint32_t l = __float_as_uint(a.lo) ^ (h & 0x80000000u);   // sign(hi) * lo
    if ((l & 0x7fffffffu) == 0u) l = 0u;                       // -0 and +0 alike
    uint32_t ml = (l & 0x80000000u) ? ~l : (l | 0x80000000u);
    return ((unsigned long long)ah << 32) | ml;
}

// Inverse of df_abs_key given the sign of hi.
__device__ __forceinline__ df df_from_abs_key(unsigned long long key, bool negative) {
    uint32_t ah = (uint32_t)(key >> 32);
    if (ah == 0u) return {0.0f, 0.0f};
    uint32_t ml = (uint32_t)key;
    uint32_t l = (ml & 0x80000000u) ? (ml & 0x7fffffffu) : ~ml;
    float hi = __uint_as_float(ah);
    float slo = __uint_as_float(l);
    return negative ? df{-hi, -slo} : df{hi, slo};
}
