// mp_step.cuh -- per-step building blocks shared by the pursuit kernels
// (mp.cu, mp_cluster.cu): step records, top-2 summaries and their warp
// reductions, and the rank-1 correlation update of one atom family.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace aqmp {

struct StepRec {
    uint32_t j;
    float hi, lo;
};

constexpr uint32_t kNone = 0xffffffffu;

// Top-2 summary of a set of correlations.  P packs the largest |hi| (its
// float bits, high word) with (0xffff - index) << 1 | sign(hi) (low word), so
// the unsigned maximum of P picks the largest magnitude and, among equal
// magnitudes, the lowest index; k2 is the second largest |hi| bits (equal to
// the largest when two atoms share it) and lo1 the low word of the top.
struct Top2 {
    unsigned long long P;
    uint32_t k2;
    float lo1;
};

__device__ __forceinline__ Top2 top2_empty() { return Top2{0ull, 0u, 0.0f}; }

__device__ __forceinline__ unsigned long long top2_key(float hi, uint32_t j) {
    const uint32_t h = __float_as_uint(hi);
    return ((unsigned long long)(h & 0x7fffffffu) << 32) | (((0xffffu - j) << 1) | (h >> 31));
}

// Running top-2 kept on float magnitudes inside element loops (cheaper per
// element than the packed key); the top is tracked by its register slot, a
// compile-time constant in the unrolled loops (a thread's atom index grows
// with the slot), and converted to a Top2 once per thread.
struct Run2 {
    float v1, lo1, m2;     // signed top value, its low word, second largest |value|
    uint32_t s1;           // slot of the top (0xffff: none)
};

__device__ __forceinline__ Run2 run2_empty() { return Run2{0.0f, 0.0f, 0.0f, 0xffffu}; }

// Elements must be folded in ascending slot order (strict > keeps the
// lowest index among equal magnitudes).
__device__ __forceinline__ void run2_fold(Run2 &r, float hi, float lo, uint32_t slot) {
    const float ah = fabsf(hi), a1 = fabsf(r.v1);
    r.m2 = fmaxf(r.m2, fminf(a1, ah));
    const bool take = ah > a1;
    r.v1 = take ? hi : r.v1;
    r.lo1 = take ? lo : r.lo1;
    r.s1 = take ? slot : r.s1;
}

// Atom index of slot s for thread `lane` of a T-thread group: lane + T s.
template <int T>
__device__ __forceinline__ Top2 run2_top2(const Run2 &r, int lane) {
    const uint32_t h = __float_as_uint(r.v1);
    const uint32_t j1 = (uint32_t)lane + (uint32_t)T * r.s1;
    const unsigned long long P = r.v1 == 0.0f && r.s1 == 0xffffu
                                     ? 0ull
                                     : ((unsigned long long)(h & 0x7fffffffu) << 32) |
                                           (((0xffffu - j1) << 1) | (h >> 31));
    return Top2{P, __float_as_uint(r.m2), r.lo1};
}

// Fold one element into a running top-2.
__device__ __forceinline__ void top2_fold(Top2 &t, float hi, float lo, uint32_t j) {
    const unsigned long long Pe = top2_key(hi, j);
    t.k2 = max(t.k2, min((uint32_t)(t.P >> 32), (uint32_t)(Pe >> 32)));
    const bool take = Pe > t.P;
    t.P = take ? Pe : t.P;
    t.lo1 = take ? lo : t.lo1;
}

__device__ __forceinline__ Top2 top2_merge(const Top2 &a, const Top2 &b) {
    const bool aw = a.P > b.P;
    const uint32_t ka = (uint32_t)(a.P >> 32), kb = (uint32_t)(b.P >> 32);
    return Top2{aw ? a.P : b.P, max(max(a.k2, b.k2), min(ka, kb)), aw ? a.lo1 : b.lo1};
}

// The summary left when its top element is removed: the second key is the
// exact new largest magnitude (its index, sign and low word unknown: low
// word 0, which no atom's key has), and also bounds the new second key.
__device__ __forceinline__ Top2 stale_top2(const Top2 &t) {
    return Top2{(unsigned long long)t.k2 << 32, t.k2, 0.0f};
}

__device__ __forceinline__ uint32_t top2_index(const Top2 &t) { return 0xffffu - (((uint32_t)t.P & 0x1ffffu) >> 1); }
__device__ __forceinline__ bool top2_negative(const Top2 &t) { return ((uint32_t)t.P & 1u) != 0u; }
__device__ __forceinline__ float top2_amax(const Top2 &t) { return __uint_as_float((uint32_t)(t.P >> 32)); }

// Warp-wide top-2 from redux.sync maxima.  After the largest |hi| key, the
// lowest index among the lanes holding it and the second key are reduced
// side by side: when two lanes hold the largest key it is also the second
// (ballot count); otherwise the second is the largest of the other lanes'
// tops and the holder's own second.  Every lane gets the result.
__device__ __forceinline__ Top2 warp_top2(const Top2 &t) {
    const uint32_t hk = (uint32_t)(t.P >> 32);
    const uint32_t low = (uint32_t)t.P;
    const uint32_t mhk = __reduce_max_sync(0xffffffffu, hk);
    const bool holds = hk == mhk;
    const unsigned holders = __ballot_sync(0xffffffffu, holds);
    const uint32_t mlow = __reduce_max_sync(0xffffffffu, holds ? low : 0u);
    const uint32_t k2c = __reduce_max_sync(0xffffffffu, holds ? t.k2 : hk);
    const uint32_t mk2 = __popc(holders) > 1 ? mhk : k2c;
    const unsigned who = __ballot_sync(0xffffffffu, holds && low == mlow);
    const float lo1 = __shfl_sync(0xffffffffu, t.lo1, __ffs(who) - 1);
    return Top2{((unsigned long long)mhk << 32) | mlow, mk2, lo1};
}

__device__ __forceinline__ void warp_argmax64(unsigned long long &bk, uint32_t &bj) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, off);
        const uint32_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
        if (ok > bk || (ok == bk && oj < bj)) {
            bk = ok;
            bj = oj;
        }
    }
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Rank-1 update of the elements in slots [S0, S0 + G) (one atom family,
// whose in-family index is j - FOFF) and their new top-2, folded into one
// running top-2 (fewer instructions per step beat shorter dependency chains
// here: one accumulator measured 7% faster than four at b = 64).
template <int B, int T, int E, int G, int S0, int FOFF, bool DF>
__device__ __forceinline__ Top2 update_family(float (&ch)[E], float (&cl)[E], int lane, const df &u,
                                              const float2 *Vq) {
    // element (lane, s) is atom lane + T s, in-family column q = (lane / B) +
    // (T / B) s - FOFF / B (T and FOFF are multiples of B)
    const float2 *Vl = Vq + (unsigned)lane / (unsigned)B;
    Run2 acc = run2_empty();
#pragma unroll
    for (int s2 = 0; s2 < G; ++s2) {
        const int s = S0 + s2;
        const float2 w = Vl[(T / B) * s - FOFF / B];
        if (DF) {
            const df r = df_sub_mul(df{ch[s], cl[s]}, u, df{w.x, w.y});
            ch[s] = r.hi;
            cl[s] = r.lo;
        } else {
            ch[s] = __fmaf_rn(-u.hi, w.x, ch[s]);     // plain FP32 form: one FMA per entry
        }
        run2_fold(acc, ch[s], cl[s], (uint32_t)s);
    }
    return run2_top2<T>(acc, lane);
}

// Zero element j1 among slots [S0, S0 + G) (none if j1 is not one of them)
// and recompute their top-2.
template <int T, int E, int G, int S0>
__device__ __forceinline__ Top2 zero_and_rescan(float (&ch)[E], float (&cl)[E], int lane, uint32_t j1) {
    Run2 acc = run2_empty();
#pragma unroll
    for (int s2 = 0; s2 < G; ++s2) {
        const int s = S0 + s2;
        const int j = lane + T * s;
        if ((uint32_t)j == j1) { ch[s] = 0.0f; cl[s] = 0.0f; }
        run2_fold(acc, ch[s], cl[s], (uint32_t)s);
    }
    return run2_top2<T>(acc, lane);
}

// Zero slot S0 + s2 (0 <= s2 < G); the registers stay statically indexed.
template <int E, int G, int S0>
__device__ __forceinline__ void zero_slot(float (&ch)[E], float (&cl)[E], int s2) {
#pragma unroll
    for (int i = 0; i < G; ++i)
        if (i == s2) {
            ch[S0 + i] = 0.0f;
            cl[S0 + i] = 0.0f;
        }
}

}  // namespace aqmp
