// corr_sep.cu -- (a2) initial correlation with the separable fixed-point
// dictionary (sep.cuh) on the integer SIMT pipes: exact, and the reference
// twin of the tensor-core kernel of corr_sep_tc.cu (same bits).
//
// Section 2.2 step (b) needs <r0, phi_j> for every atom j.  The DCT-II and
// Haar atoms are outer products of 1-D rows (Section 2.1), so the M = 2 b^2
// correlations of a block are B Y B^T for each family: two b x b x b products
// instead of the b^4 per family of a dense D^T y, and the rows' structure
// (the DCT-II rows' mirror symmetry, the Haar rows' two constant halves)
// cuts that further, as the kernel below describes.  In integers:
//   stage 1  Z~[p][m] = sum_i Bf[p][i] y~[i][m]   (48-bit x 8-bit -> int64)
//   stage 2  T~[p][q] = sum_m Bf[q][m] Z~[p][m]   (48-bit x 59-bit -> int128)
// Bf is held as 24-bit limbs (lo in [-2^23, 2^23), hi = (Bf - lo) / 2^24,
// |hi| < 2^23.5), and the stage-1 results (Z~+-, below, |Z~+-| < 2^60) as
// two 32-bit ones (zl in [-2^31, 2^31), zh = (z - zl) / 2^32, |zh| < 2^28),
// so every partial product is one 32 x 32 -> 64-bit multiply-add, at most
// 2^54.5 in magnitude, and each of the four limb sums over at most b/2 = 64
// terms stays below 2^61.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "haar_rows.cuh"
#include "sep.cuh"

namespace aqmp {

namespace {

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Leaves per CTA: enough for 4096 outputs per family and stage.
template <int B>
constexpr int sep_group() { return B >= 64 ? 1 : 4096 / (B * B); }

// Z~ split into balanced limbs: z = zl + zh 2^32.
struct Limbs2 {
    int32_t zl, zh;
};

__device__ __forceinline__ Limbs2 split2(long long z) {
    const int32_t zl = (int32_t)(uint32_t)(unsigned long long)z;    // z mod 2^32, in [-2^31, 2^31)
    return Limbs2{zl, (int32_t)((z - (long long)zl) >> 32)};
}

__device__ __forceinline__ long long mul_wide(int32_t a, int32_t b) { return (long long)a * (long long)b; }

}  // namespace

// Threads per CTA: at side 128 the leaf's shared memory (181 KB, most of it
// Z~+-) leaves room for one CTA per SM, so that CTA takes 768 threads to hide
// the latency of its loads; 256 elsewhere.
template <int B>
constexpr int sep_threads() { return B >= 128 ? 768 : 256; }

// Shared-memory layout of one CTA (G leaves): the centred pixels, their
// even and odd column halves, and the Z~ region, which the Haar pass reuses
// for its summed-area table.  A Haar-only launch (HO) keeps the pixels and
// the table alone.
template <int B, bool HO = false>
struct SepSmem {
    static constexpr int n = B * B, H = B / 2, G = sep_group<B>();
    static constexpr int RS = B + 1;                           // row stride of Z~+- and of the table
    static constexpr int YS = B + 4;                           // row stride of the pixels (bytes): the
                                                               // transposing stores hit distinct banks
    static constexpr size_t yt = 0;                            // int8  [G][i][YS]
    static constexpr size_t ys = (G * B * YS + 15) & ~15;      // int16 [G][parity][i < H][m]
    static constexpr size_t z = ys + (HO ? 0 : ((2 * G * n + 15) & ~15));   // Limbs2 [G][p][RS] / int [G][RS][RS]
    static constexpr size_t zbytes = HO ? ((sizeof(int) * G * RS * RS + 15) & ~15) : sizeof(Limbs2) * G * B * RS;
    static constexpr int E = 1 + ilog2(B);                     // Haar scale classes: row 0, scales 1 .. b/2
    static constexpr size_t hrow = z + zbytes;                 // int4 [B]: s, h, class, sign
    static constexpr size_t ptab = hrow + sizeof(int4) * B;    // ulonglong2 [E][E]: fL(c1) fL(c2), int128
    static constexpr size_t bytes = ptab + sizeof(ulonglong2) * E * E;
    static_assert(sizeof(int) * RS * RS <= sizeof(Limbs2) * B * RS, "table fits the Z~ region");
};

__device__ __forceinline__ long long bf_value(int2 w) { return (long long)w.y * (1ll << 24) + w.x; }

// P K for 0 <= P < 2^96 (as 64-bit halves lo, hi < 2^32) and |K| < 2^31:
// three 32 x 32 -> 64-bit products joined in int128.
__device__ __forceinline__ __int128 mul_u96_i32(const ulonglong2 &P, int K) {
    const unsigned k = (unsigned)(K < 0 ? -K : K);
    const unsigned long long a0 = (unsigned long long)(unsigned)P.x * k;
    const unsigned long long a1 = (unsigned long long)(unsigned)(P.x >> 32) * k;
    const unsigned long long a2 = (unsigned long long)(unsigned)P.y * k;
    const unsigned __int128 m = (unsigned __int128)a0 + ((unsigned __int128)a1 << 32) + ((unsigned __int128)a2 << 64);
    return K < 0 ? -(__int128)m : (__int128)m;
}

// One CTA handles G leaves at a time (grid-stride over the leaves).
//
// DCT-II family: row p of Bf equals (-1)^p times its mirror image, so with
// the column halves y+-[i][m] = y~[i][m] +- y~[b-1-i][m] (i < b/2) stage 1
// needs b/2 terms, and stage 1 stores Z~+-[p][m] = Z~[p][m] +- Z~[p][b-1-m]
// (m < b/2), of which stage 2 takes Z~+ for even q and Z~- for odd q, again
// over b/2 terms: half the multiply-adds of the plain products, the same
// exact integers.  |Z~+-| < 2^60, so zh < 2^28 and every limb sum over
// b/2 <= 64 terms stays below 2^61.
//
// Haar family: row p of Bf is constant on each of two dyadic halves
// (haar_halves), fL on the first and s_p fL on the second (s_p = +1 for row
// 0, -1 otherwise), and fL depends only on the row's scale.  So T~[p][q] =
// fL(p) fL(q) K with K = LL + s_q LR + s_p RL + s_p s_q RR, the sums of y~
// over the four half-by-half rectangles, read from the summed-area table of
// y~ (|entries| <= 2^21, |K| <= 2^21); the products fL(c1) fL(c2) of the
// 1 + log2 b scale classes are formed once per CTA in int128.
template <int B, bool HO>
__global__ void __launch_bounds__(sep_threads<B>())
corr_sep_simt_kernel(int nf, int fam0, int fmask, int Kpad, const int2 *__restrict__ Bs, const int2 *__restrict__ BsT,
                     const long long *__restrict__ Rs, const __nv_bfloat16 *__restrict__ Y,
                     const unsigned *count_dev, long long fixed_count, float2 *__restrict__ c0) {
    using L = SepSmem<B, HO>;
    constexpr int n = L::n, H = L::H, G = L::G, RS = L::RS, YS = L::YS;
    if (HO) fmask &= 2;                                       // the Haar family alone
    constexpr int PT = 4;                                     // p values per thread in DCT stage 2
    static_assert(B >= PT && B % PT == 0, "side");
    extern __shared__ __align__(16) unsigned char smem[];
    int8_t *yt = reinterpret_cast<int8_t *>(smem + L::yt);
    int16_t *ys = reinterpret_cast<int16_t *>(smem + L::ys);
    Limbs2 *Z = reinterpret_cast<Limbs2 *>(smem + L::z);
    int *S = reinterpret_cast<int *>(smem + L::z);

    constexpr int nt = sep_threads<B>(), nw = nt / 32, E = L::E;
    int4 *hrow = reinterpret_cast<int4 *>(smem + L::hrow);
    ulonglong2 *ptab = reinterpret_cast<ulonglong2 *>(smem + L::ptab);

    const long long count = count_dev ? (long long)*count_dev : fixed_count;
    const int M = nf * n;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if ((nf == 2 || fam0 == 1) && ((fmask >> 1) & 1)) {
        // the Haar rows' supports and classes, and the class products
        const int2 *Bh = Bs + (size_t)n;
        for (int r = tid; r < B; r += nt) {
            int sr, hr;
            haar_halves(r, B, sr, hr);
            const int cls = r == 0 ? 0 : 1 + (31 - __clz(B / (2 * hr)));
            hrow[r] = make_int4(sr, hr, cls, r == 0 ? 1 : -1);
        }
        for (int e = tid; e < E * E; e += nt) {
            const int c1 = e / E, c2 = e - c1 * E;
            const int r1 = c1 == 0 ? 0 : 1 << (c1 - 1), r2 = c2 == 0 ? 0 : 1 << (c2 - 1);   // first row of the class
            const unsigned __int128 P = (unsigned __int128)((__int128)bf_value(Bh[r1 * B]) * bf_value(Bh[r2 * B]));
            ptab[e] = make_ulonglong2((unsigned long long)P, (unsigned long long)(P >> 64));
        }
        __syncthreads();
    }
    for (long long base = (long long)blockIdx.x * G; base < count; base += (long long)gridDim.x * G) {
        const int live = (int)min((long long)G, count - base);
        // centred pixels, transposed so that the contractions read consecutive m
        for (int o = tid; o < G * n; o += nt) {
            const int g = o / n, v = o - g * n;
            const int m = v / B, i = v - m * B;
            int8_t y = 0;
            if (g < live) y = (int8_t)__bfloat162float(Y[(base + g) * Kpad + v]);
            yt[(g * B + i) * YS + m] = y;
        }
        __syncthreads();
        for (int f = 0; f < nf; ++f) {
            const int F = nf == 2 ? f : fam0;
            if (!((fmask >> F) & 1)) continue;                   // uniform
            const int2 *Bf = Bs + (size_t)F * n;
            const long long *R = Rs + F * B;
            float2 *out = c0 + (nf == 2 ? f * n : 0);
            if (F == 0) {
                if constexpr (!HO) {
                const int2 *BfT = BsT + (size_t)F * n;
                for (int o = tid; o < G * H * B; o += nt) {
                    const int g = o / (H * B), r = o - g * (H * B);
                    const int i = r / B, m = r - i * B;
                    const int a = yt[(g * B + i) * YS + m], c = yt[(g * B + B - 1 - i) * YS + m];
                    ys[(2 * g) * H * B + r] = (int16_t)(a + c);
                    ys[(2 * g + 1) * H * B + r] = (int16_t)(a - c);
                }
                __syncthreads();
                // stage 1: Z~[p][m] and Z~[p][b-1-m] together, m < b/2 across threads
                for (int o = tid; o < G * B * H; o += nt) {
                    const int g = o / (B * H), r = o - g * (B * H);
                    const int p = r / H, m = r - p * H;
                    const int16_t *yp = ys + (2 * g + (p & 1)) * H * B;
                    long long lo1 = 0, hi1 = 0, lo2 = 0, hi2 = 0;
#pragma unroll 8
                    for (int i = 0; i < H; ++i) {
                        const int2 w = Bf[p * B + i];
                        const int32_t a = yp[i * B + m], c = yp[i * B + B - 1 - m];
                        lo1 += mul_wide(w.x, a);
                        hi1 += mul_wide(w.y, a);
                        lo2 += mul_wide(w.x, c);
                        hi2 += mul_wide(w.y, c);
                    }
                    const long long z1 = hi1 * (1ll << 24) + lo1, z2 = hi2 * (1ll << 24) + lo2;
                    Limbs2 *zr = Z + (g * B + p) * RS;
                    zr[m] = split2(z1 + z2);
                    zr[H + 1 + m] = split2(z1 - z2);
                }
                __syncthreads();
                // stage 2: T~[g][p][q], q lane-fastest, PT consecutive p per thread
                for (int o = tid; o < G * n / PT; o += nt) {
                    const int g = o / (n / PT), r = o - g * (n / PT);
                    const int q = r % B, p0 = (r / B) * PT;
                    const Limbs2 *zr = Z + (g * B + p0) * RS + ((q & 1) ? H + 1 : 0);
                    long long a0[PT], a1[PT], a2[PT], a3[PT];
#pragma unroll
                    for (int k = 0; k < PT; ++k) a0[k] = a1[k] = a2[k] = a3[k] = 0;
#pragma unroll 4
                    for (int m = 0; m < H; ++m) {
                        const int2 w = BfT[m * B + q];                 // Bf[q][m]: (lo, hi)
#pragma unroll
                        for (int k = 0; k < PT; ++k) {
                            const Limbs2 z = zr[k * RS + m];
                            a0[k] += mul_wide(w.x, z.zl);              // weight 1
                            a1[k] += mul_wide(w.y, z.zl);              // 2^24
                            a2[k] += mul_wide(w.x, z.zh);              // 2^32
                            a3[k] += mul_wide(w.y, z.zh);              // 2^56
                        }
                    }
                    if (g < live) {
                        float v[2 * PT];
#pragma unroll
                        for (int k = 0; k < PT; ++k) {
                            __int128 T = (__int128)a3[k] * ((__int128)1 << 56) + (__int128)a2[k] * ((__int128)1 << 32) +
                                         (__int128)a1[k] * ((__int128)1 << 24) + (__int128)a0[k];
                            T += (__int128)(128ll * R[p0 + k]) * R[q];
                            const df c = int128_to_df(T);
                            v[2 * k] = c.hi;
                            v[2 * k + 1] = c.lo;
                        }
                        float4 *dst = reinterpret_cast<float4 *>(out + (base + g) * M + q * B + p0);
#pragma unroll
                        for (int k = 0; k < PT / 2; ++k)
                            dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    }
                }
                }
            } else {
                // summed-area table S[i][m] = sum of y~ over [0, i) x [0, m):
                // prefix sums along m (one warp per row), then along i (one
                // warp per column; stride RS = 1 mod 32 keeps it conflict-free)
                for (int o = tid; o < G * RS; o += nt) {
                    const int g = o / RS, e = o - g * RS;
                    S[g * RS * RS + e] = 0;                            // row 0
                    S[g * RS * RS + e * RS] = 0;                       // column 0
                }
                for (int row = warp; row < G * B; row += nw) {
                    const int g = row / B, i = row - g * B;
                    int carry = 0;
                    for (int c = 0; c < B; c += 32) {
                        int v = c + lane < B ? (int)yt[(g * B + i) * YS + c + lane] : 0;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const int u = __shfl_up_sync(0xffffffffu, v, d);
                            if (lane >= d) v += u;
                        }
                        if (c + lane < B) S[g * RS * RS + (i + 1) * RS + c + lane + 1] = carry + v;
                        carry += __shfl_sync(0xffffffffu, v, 31);
                    }
                }
                __syncthreads();
                for (int col = warp; col < G * B; col += nw) {
                    const int g = col / B, m = col - g * B + 1;
                    int carry = 0;
                    for (int c = 0; c < B; c += 32) {
                        int *at = S + g * RS * RS + (c + lane + 1) * RS + m;
                        int v = c + lane < B ? *at : 0;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const int u = __shfl_up_sync(0xffffffffu, v, d);
                            if (lane >= d) v += u;
                        }
                        if (c + lane < B) *at = carry + v;
                        carry += __shfl_sync(0xffffffffu, v, 31);
                    }
                }
                __syncthreads();
                // T~[g][p][q], p lane-fastest
                for (int o = tid; o < G * n; o += nt) {
                    const int g = o / n, r = o - g * n;
                    const int q = r / B, p = r - q * B;
                    const int4 hp = hrow[p], hq = hrow[q];
                    const int *Sg = S + g * RS * RS;
                    const int *r0 = Sg + hp.x * RS, *r1 = r0 + hp.y * RS, *r2 = r1 + hp.y * RS;
                    const int m0 = hq.x, m1 = hq.x + hq.y, m2 = hq.x + 2 * hq.y;
                    const int s00 = r0[m0], s01 = r0[m1], s02 = r0[m2];
                    const int s10 = r1[m0], s11 = r1[m1], s12 = r1[m2];
                    const int s20 = r2[m0], s21 = r2[m1], s22 = r2[m2];
                    const int LL = s11 - s01 - s10 + s00, LR = s12 - s02 - s11 + s01;
                    const int RL = s21 - s11 - s20 + s10, RR = s22 - s12 - s21 + s11;
                    const int K = (LL + hq.w * LR) + hp.w * (RL + hq.w * RR);
                    __int128 T = mul_u96_i32(ptab[hp.z * E + hq.z], K);
                    // rows r >= 1 sum to zero (halves of equal length and
                    // opposite values), so only (0, 0) has a centring term
                    if ((p | q) == 0) T += (__int128)(128ll * R[0]) * R[0];
                    if (g < live) {
                        const df c = int128_to_df(T);
                        out[(base + g) * M + q * B + p] = make_float2(c.hi, c.lo);
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int B, bool HO>
static cudaError_t launch_sep_simt_t(const CorrArgs &a, cudaStream_t st) {
    constexpr int G = sep_group<B>();
    const size_t smem = SepSmem<B, HO>::bytes;
    auto kern = corr_sep_simt_kernel<B, HO>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sep_threads<B>(), smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    long long need = ((long long)a.capacity + G - 1) / G;
    long long grid = (long long)sms * (per_sm < 1 ? 1 : per_sm);
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    const DictDev &d = *a.d;
    kern<<<(unsigned)grid, sep_threads<B>(), smem, st>>>(d.nf, d.fam0, a.fmask ? a.fmask : 3, d.Kpad, d.Bs, d.BsT,
                                                          d.Rs, a.Y, a.count,
                                                          a.fixed_count, a.c0);
    return cudaGetLastError();
}

cudaError_t launch_corr_sep_simt(const CorrArgs &a, cudaStream_t st) {
    // the Haar family alone gets its own instantiation: no DCT-II code or
    // shared memory, so more CTAs fit on an SM
    const DictDev &d = *a.d;
    const bool ho = a.fmask == 2 || (d.nf == 1 && d.fam0 == 1);
    switch (d.b) {
        case 4: return ho ? launch_sep_simt_t<4, true>(a, st) : launch_sep_simt_t<4, false>(a, st);
        case 8: return ho ? launch_sep_simt_t<8, true>(a, st) : launch_sep_simt_t<8, false>(a, st);
        case 16: return ho ? launch_sep_simt_t<16, true>(a, st) : launch_sep_simt_t<16, false>(a, st);
        case 32: return ho ? launch_sep_simt_t<32, true>(a, st) : launch_sep_simt_t<32, false>(a, st);
        case 64: return ho ? launch_sep_simt_t<64, true>(a, st) : launch_sep_simt_t<64, false>(a, st);
        case 128: return ho ? launch_sep_simt_t<128, true>(a, st) : launch_sep_simt_t<128, false>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace aqmp
