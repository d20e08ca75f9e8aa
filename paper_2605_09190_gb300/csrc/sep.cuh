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

// Normalise a nonzero 128-bit magnitude (ahi:alo) so that bit 127 is set and
// round its top 24 bits to nearest, ties to even: m (<= 2^24), e the index of
// the leading bit, lz the normalising shift, and the signed remainder in
// normalised units, (rhi:rlo) = n - m 2^104 with |rhi| <= 2^39.
__device__ __forceinline__ void round24(unsigned long long ahi, unsigned long long alo, unsigned long long &m,
                                        int &e, int &lz, long long &rhi, unsigned long long &rlo) {
    lz = ahi ? __clzll((long long)ahi) : 64 + __clzll((long long)alo);
    unsigned long long nhi, nlo;
    if (lz == 0) {
        nhi = ahi;
        nlo = alo;
    } else if (lz < 64) {
        nhi = (ahi << lz) | (alo >> (64 - lz));
        nlo = alo << lz;
    } else {
        nhi = alo << (lz - 64);
        nlo = 0ull;
    }
    e = 127 - lz;
    m = nhi >> 40;
    const unsigned long long r = nhi & ((1ull << 40) - 1), half = 1ull << 39;
    if (r > half || (r == half && (nlo != 0ull || (m & 1ull)))) ++m;
    rhi = (long long)(nhi - (m << 40));      // exact modulo 2^64, and in range
    rlo = nlo;
}

// m 2^k as a float for 2^23 <= m <= 2^24 and a normal result.
__device__ __forceinline__ float pow2_float(unsigned long long m, int k) {
    return __int_as_float(((k + 23 + 127) << 23) + (int)(m - (1ull << 23)));
}

// T 2^-96 as the double-float (RN(T), RN(T - RN(T))) scaled by 2^-96, ties to
// even: a function of T alone, ~2^-48 relative.  |T| < 2^112.
__device__ __forceinline__ df int128_to_df(__int128 T) {
    if (T == 0) return df{0.0f, 0.0f};
    const bool neg = T < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
    const unsigned long long ahi = (unsigned long long)(a >> 64), alo = (unsigned long long)a;
    const int s96 = -2 * kSepFixBits;
    float hi, lo = 0.0f;
    if (ahi == 0ull && alo < (1ull << 24)) {
        hi = __fmul_rn((float)(unsigned)alo, __int_as_float((127 + s96) << 23));      // exact
    } else {
        unsigned long long m;
        int e, lz;
        long long rhi;
        unsigned long long rlo;
        round24(ahi, alo, m, e, lz, rhi, rlo);
        hi = pow2_float(m, e - 23 + s96);
        if (rhi != 0 || rlo != 0ull) {
            // |remainder| in normalised units, then rounded the same way and
            // scaled back by 2^-lz
            const bool rneg = rhi < 0;
            unsigned long long bhi = (unsigned long long)rhi, blo = rlo;
            if (rneg) {
                blo = ~rlo + 1ull;
                bhi = ~(unsigned long long)rhi + (blo == 0ull ? 1ull : 0ull);
            }
            unsigned long long m2;
            int e2, lz2;
            long long r2hi;
            unsigned long long r2lo;
            round24(bhi, blo, m2, e2, lz2, r2hi, r2lo);
            lo = pow2_float(m2, e2 - 23 - lz + s96);
            if (rneg) lo = -lo;
        }
    }
    return neg ? df{-hi, -lo} : df{hi, lo};
}

}  // namespace aqmp
