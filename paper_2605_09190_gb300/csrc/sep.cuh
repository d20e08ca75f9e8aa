// sep.cuh -- the separable fixed-point dictionary of the exact correlation.
//
// Each 1-D basis row (DCT-II and Haar, Section 2.1 Eq. (1)-(2), Section 2.3)
// enters in fixed point, Bf = round(B 2^48), an integer below 2^47.5 in
// magnitude (|B| <= sqrt(2/b) <= 2^-0.5).  The 2-D atom (p, q) of a family is
// the outer product of rows p and q (Section 2.1; its pixel (i, m) sits at
// v = m b + i, Appendix A), so with this dictionary the correlation of a
// block y is the exact integer
//
//     T[p][q] = sum_m Bf[q][m] Z[p][m],    Z[p][m] = sum_i Bf[p][i] y[i][m],
//
// i.e. B Y B^T in integers, and c = T 2^-96 rounded once into a double-float.
// With centred pixels y~ = y - 128 the kernels form Z~ = Bf y~ and T~ = Bf^T Z~
// and add the exact centring term 128 R[p] R[q], R[p] = sum_i Bf[p][i].
// Magnitudes: |Z~| < 128 sqrt(b) 2^47.5 <= 2^59, |T| < 2^112 (b <= 128).
//
// Against the exact dictionary the fixed-point entry errs by at most
// 2^-49 (|B[p][i]| + |B[q][m]|) + 2^-97; the rounding into the double-float
// adds 2^-48 |c| at most.
#pragma once
#include <cstdint>

#include "df.cuh"

namespace aqmp {

constexpr int kSepFixBits = 48;                 // Bf = round(B 2^kSepFixBits)

// |a| rounded to the nearest float (ties to even) and the exact integer value
// of that float.
__device__ __forceinline__ float u128_round_float(unsigned __int128 a, unsigned __int128 &val) {
    const unsigned long long h = (unsigned long long)(a >> 64), l = (unsigned long long)a;
    if (h == 0ull && l < (1ull << 24)) {
        val = a;
        return (float)(unsigned)l;                                // exact
    }
    const int len = h ? 128 - __clzll((long long)h) : 64 - __clzll((long long)l);
    const int sh = len - 24;                                      // 1 <= sh <= 104
    unsigned long long m = (unsigned long long)(a >> sh);         // the top 24 bits
    const unsigned __int128 rem = a - ((unsigned __int128)m << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;           // m <= 2^24: exact in a float
    val = (unsigned __int128)m << sh;
    return __fmul_rn((float)m, __int_as_float((127 + sh) << 23)); // m 2^sh, exact
}

// T 2^-96 as the double-float (RN(T), RN(T - RN(T))) scaled by 2^-96: a
// function of T alone, ~2^-48 relative.
__device__ __forceinline__ df int128_to_df(__int128 T) {
    if (T == 0) return df{0.0f, 0.0f};
    const bool neg = T < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
    unsigned __int128 hv, lv;
    float hi = u128_round_float(a, hv);
    const bool rneg = a < hv;
    float lo = u128_round_float(rneg ? hv - a : a - hv, lv);
    if (rneg) lo = -lo;
    if (neg) {
        hi = -hi;
        lo = -lo;
    }
    const float s = __int_as_float((127 - 2 * kSepFixBits) << 23);   // 2^-96
    return df{__fmul_rn(hi, s), __fmul_rn(lo, s)};
}

}  // namespace aqmp
