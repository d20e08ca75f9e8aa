// corr_sep_tc.cu -- (a2) the separable exact correlation (sep.cuh) on the
// 5th-generation tensor cores, side 64: the same exact integer T = B Y B^T
// per family as the SIMT twin (corr_sep.cu), rounded the same way, so both
// give identical bits.
//
// Digits.  Bf = sum_{s<6} d_s 2^(8s) with balanced digits |d_s| <= 128 (the
// top one <= 181), all exact BF16 values, as are the centred pixels.
//   Stage 1 (per leaf and family): Z~^T[m][p] = sum_i y~[i][m] Bf[p][i].
//     A = [d_2u rows p ; d_2u+1 rows p] (128 rows, K = i) from shared memory,
//     B = the leaf's pixels (rows m, K = i), one FP32 accumulator per digit
//     pair u: lane (s parity, p), column m.  |d y~| sums over 64 terms stay
//     below 2^24: exact.
//   Z~ (|Z~| < 2^59) is assembled exactly in int64 from the six digit sums
//   (the two parities meet through shared memory) and split into eight
//   balanced base-2^8 digits e_t, written into tensor memory as the A operand
//   of stage 2: tile v holds [e_2v rows p ; e_2v+1 rows p] (K = m).
//   Stage 2: T~[p][q] = sum_{t,s} 2^(8(t+s)) sum_m e_t[p][m] d_s[q][m].
//     A = tile v (tensor memory), B = d_s rows q (shared memory, 32 q per
//     pass), accumulated into column block 2v + s: lane half h of block c
//     then holds the digit diagonal t + s = c + h, the sum of at most three
//     digit products (one per tile v with 0 <= c - 2v < 6), each below
//     128 x 181 x 64 < 2^20.5 in magnitude: below 2^22, exact.
//   The epilogue reads each diagonal (an exact FP32 integer), joins
//   adjacent diagonals in one 32-bit multiply-add and those pairs in int64
//   groups, then in int128 (the base-2^8 Horner scheme), the two lane
//   halves meet through shared memory, and T = T~ + 128 R[p] R[q] is
//   rounded once into a double-float (int128_to_df).
//
// One CTA per SM (16 warps, all 512 TMEM columns: A tiles 0..127, stage-1
// accumulators 128..319, stage-2 accumulators 128..511), persistent over the
// leaves; thread 0 issues the TMA loads and the MMAs, all threads drain.
// Every wait is bounded by a timer; on expiry the kernel records
// AQMP_E_TIMEOUT, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "sep.cuh"
#include "tc_sep.cuh"

namespace aqmp {

namespace septc {

constexpr int kB = 64;                        // block side served here
constexpr int kThreads = 512;                 // 16 warps: 4 per TMEM lane quarter
constexpr int kTmemCols = 512;
constexpr int kColA = 0;                      // stage-2 A tiles: 4 x 32 columns
constexpr int kColD = 128;                    // accumulators
constexpr int kTileBd = 128 * 128;            // bytes: 128 rows x 128 B (two digits of one family)
constexpr int kTileY = 64 * 128;              // bytes: 64 rows (m) x 64 BF16 (i)
constexpr int kOffBd = 0;                     // 6 tiles: (family, digit pair)
constexpr int kOffY = kOffBd + 6 * kTileBd;   // 2 buffers
constexpr int kOffX = kOffY + 2 * kTileY;     // exchange: 64 KB
constexpr int kBytesX = 64 * 1024;
constexpr int kOffBar = kOffX + kBytesX;      // barriers: Bd, Y[2], MMA
constexpr int kOffMisc = kOffBar + 8 * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;

// Stage 1: M = 128, N = 64; stage 2: M = 128, N = 32; BF16 x BF16 -> F32.
constexpr uint32_t kIdesc1 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kIdesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);

}  // namespace septc

// Y map: the gathered leaves viewed as [capacity * 64 rows][64] BF16 (row m of
// leaf l at row 64 l + m, K = i); Bd map: [6 * 128 rows][64] BF16, tile (F, u)
// at row 128 (3 F + u).
__global__ void __launch_bounds__(septc::kThreads, 1)
corr_sep_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmBd, int nf,
                   int fam0, int fmask, const long long *__restrict__ Rs, const unsigned *count_dev,
                   long long fixed_count, float2 *__restrict__ c0, Counters *ctr) {
    using namespace septc;
    constexpr int n = kB * kB;
    const long long count = count_dev ? (long long)*count_dev : fixed_count;
    if ((long long)blockIdx.x >= count) return;                  // uniform
    const int M = nf * n;

    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const uint32_t sBd = base + kOffBd, sY = base + kOffY, sBar = base + kOffBar;
    const uint32_t barBd = sBar, barY0 = sBar + 8, barY1 = sBar + 16, barMma = sBar + 24;
    long long *X = reinterpret_cast<long long *>(gbase + kOffX);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(gbase + kOffMisc);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(barBd, 1);
        mbar_init(barY0, 1);
        mbar_init(barY1, 1);
        mbar_init(barMma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_holder)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;

    // the six digit tiles once, the first leaf's pixels
    if (threadIdx.x == 0) {
        mbar_expect_tx(barBd, 6 * kTileBd);
        for (int t = 0; t < 6; ++t) tma_load_2d(sBd + t * kTileBd, &tmBd, barBd, 0, 128 * t);
        mbar_expect_tx(barY0, kTileY);
        tma_load_2d(sY, &tmY, barY0, 0, (int)(64 * blockIdx.x));
    }
    bool ok = __syncthreads_and(mbar_wait(barBd, 0)) != 0;

    // TMEM lane quarter of this warp and the column group it drains
    const int quarter = warp & 3, cg = warp >> 2;
    const int row = quarter * 32 + lane;                          // TMEM lane = tile row
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int par = row >> 6, p = row & 63;
    uint32_t mma_phase = 0, y_phase[2] = {0u, 0u};
    int it = 0;
    for (long long leaf = blockIdx.x; ok && leaf < count; leaf += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t barY = buf ? barY1 : barY0;
        ok = __syncthreads_and(mbar_wait(barY, y_phase[buf])) != 0;
        y_phase[buf] ^= 1u;
        if (!ok) break;
        // prefetch the next leaf into the other buffer (its last reader
        // finished with the previous iteration's barriers)
        if (threadIdx.x == 0 && leaf + gridDim.x < count) {
            const uint32_t nb = buf ? barY0 : barY1;
            mbar_expect_tx(nb, kTileY);
            tma_load_2d(sY + (buf ^ 1) * kTileY, &tmY, nb, 0, (int)(64 * (leaf + gridDim.x)));
        }
        const uint32_t yaddr = sY + buf * kTileY;
        for (int f = 0; f < nf && ok; ++f) {
            const int F = nf == 2 ? f : fam0;
            if (!((fmask >> F) & 1)) continue;                   // uniform
            // ---- stage 1: Z~^T[m][p], one accumulator per digit pair u
            if (threadIdx.x == 0) {
                fence_after();
                for (int u = 0; u < 3; ++u) {
                    const unsigned long long ad = smem_desc(sBd + (3 * F + u) * kTileBd);
                    const unsigned long long bd = smem_desc(yaddr);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_ss(tmem + kColD + 64 * u, ad + 2ull * kk, bd + 2ull * kk, kIdesc1, kk > 0 ? 1u : 0u);
                }
                mma_commit(barMma);
            }
            ok = __syncthreads_and(mbar_wait(barMma, mma_phase)) != 0;
            mma_phase ^= 1u;
            if (!ok) break;
            fence_after();
            // ---- drain 1: this thread's parity sum Z_par[p][m] for its 16 m
            // (lane row = (parity, p), columns m = 16 cg + j); X is stored
            // m-major so that the lanes of a warp (consecutive p) hit
            // consecutive words
            {
                uint32_t r0[16], r1[16], r2[16];
                const uint32_t col = kColD + 16 * cg;
                tmem_ld16(lane_base + col, r0);
                tmem_ld16(lane_base + col + 64, r1);
                tmem_ld16(lane_base + col + 128, r2);
                wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long long z = (long long)small_int(r0[j]) + (long long)small_int(r1[j]) * 65536ll +
                                        (long long)small_int(r2[j]) * 4294967296ll;
                    X[(par * 64 + 16 * cg + j) * 64 + p] = z;
                }
            }
            __syncthreads();
            // both parities of Z~[p][m] -> eight balanced digits; this lane keeps
            // the digits of its own parity (tile v = t / 2, lane half = t mod 2).
            // With z' = Z~ + sum_{t<7} 128 2^(8t), digit t < 7 is byte t of z'
            // minus 128 and digit 7 is z' >> 56: no carry chain between digits.
            {
                uint32_t packed[4][8];
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2) {
                    int32_t dig[2][4];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int m = 16 * cg + 2 * j2 + e;
                        const long long zz = X[(0 * 64 + m) * 64 + p] + X[(1 * 64 + m) * 64 + p] * 256ll +
                                             0x80808080808080ll;
                        const uint32_t lo = (uint32_t)zz, hi = (uint32_t)((unsigned long long)zz >> 32);
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int t = 2 * v + par;
                            int32_t d;
                            if (t == 7) d = (int32_t)(zz >> 56);
                            else if (t < 4) d = (int32_t)((lo >> (8 * t)) & 255u) - 128;
                            else d = (int32_t)((hi >> (8 * (t - 4))) & 255u) - 128;
                            dig[e][v] = d;
                        }
                    }
#pragma unroll
                    for (int v = 0; v < 4; ++v) packed[v][j2] = bf16_bits(dig[0][v]) | (bf16_bits(dig[1][v]) << 16);
                }
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    // 8 packed columns (16 values of m)
                    asm volatile(
                        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                        ::"r"(lane_base + kColA + 32 * v + 8 * cg), "r"(packed[v][0]), "r"(packed[v][1]),
                          "r"(packed[v][2]), "r"(packed[v][3]), "r"(packed[v][4]), "r"(packed[v][5]),
                          "r"(packed[v][6]), "r"(packed[v][7])
                        : "memory");
                }
                wait_st();
            }
            fence_before();
            __syncthreads();
            // ---- stage 2, 32 values of q per pass
            for (int c = 0; c < 2 && ok; ++c) {
                if (threadIdx.x == 0) {
                    fence_after();
                    uint32_t written = 0u;
                    for (int v = 0; v < 4; ++v)
                        for (int s = 0; s < 6; ++s) {
                            const int cb = 2 * v + s;
                            const uint32_t btile = sBd + (3 * F + (s >> 1)) * kTileBd + (s & 1) * (64 * 128) +
                                                   c * (32 * 128);
                            const unsigned long long bd = smem_desc(btile);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t acc = ((written >> cb) & 1u) | (kk > 0 ? 1u : 0u);
                                mma_ts(tmem + kColD + 32 * cb, tmem + kColA + 32 * v + 8 * kk, bd + 2ull * kk,
                                       kIdesc2, acc);
                            }
                            written |= 1u << cb;
                        }
                    mma_commit(barMma);
                }
                // the row sums this lane's outputs need, fetched while the MMAs run
                const long long rowsum_p = Rs[F * kB + p];
                long long rowsum_q[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) rowsum_q[j] = Rs[F * kB + 32 * c + 8 * cg + 4 * par + j];
                ok = __syncthreads_and(mbar_wait(barMma, mma_phase)) != 0;
                mma_phase ^= 1u;
                if (!ok) break;
                fence_after();
                // ---- drain 2: lane (half hh, p), 8 values of q; block cb holds the
                // diagonal cb + hh.  Horner in base 2^8 over three groups of four
                // blocks (each exact in an int64: |D| < 2^22), the groups joined
                // in int128; then the lanes of the two halves add their sums.
                const int hh = par;
                long long grp[3][8];
#pragma unroll
                for (int g = 2; g >= 0; --g) {
                    uint32_t r[4][8];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t ta = lane_base + kColD + 32 * (4 * g + 3 - k) + 8 * cg;
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                            : "=r"(r[k][0]), "=r"(r[k][1]), "=r"(r[k][2]), "=r"(r[k][3]), "=r"(r[k][4]),
                              "=r"(r[k][5]), "=r"(r[k][6]), "=r"(r[k][7])
                            : "r"(ta));
                    }
                    wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        // r[k] holds block 4g + 3 - k: two adjacent diagonals meet in
                        // one 32-bit multiply-add on their biased bit patterns (the
                        // bias cancels modulo 2^32 and |pair| < 2^31), two pairs in
                        // one 64-bit multiply-add
                        const int32_t hi2 = pair8(r[0][j], r[1][j]);        // blocks 4g+3, 4g+2
                        const int32_t lo2 = pair8(r[2][j], r[3][j]);        // blocks 4g+1, 4g
                        grp[g][j] = (long long)hi2 * 65536ll + (long long)lo2;
                    }
                }
                fence_before();
                __syncthreads();                  // X is free (drain 1 done), D read
                __int128 *XT = reinterpret_cast<__int128 *>(X);
                // lanes of half hh finalise q = 8 cg + [4 hh, 4 hh + 4) of the pass;
                // they hand over the other four (stored j-major: consecutive p,
                // consecutive words)
                __int128 mine[4];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const __int128 sum = ((__int128)grp[2][j] * ((__int128)1 << 64) +
                                          (__int128)grp[1][j] * ((__int128)1 << 32) + (__int128)grp[0][j]) *
                                         (hh ? (__int128)256 : (__int128)1);
                    if ((j >> 2) != hh) XT[(size_t)((cg * 2 + hh) * 8 + j) * 64 + p] = sum;
                    else mine[j & 3] = sum;
                }
                __syncthreads();
                const long long rp128 = 128ll * rowsum_p;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if ((j >> 2) == hh) {
                        const __int128 other = XT[(size_t)((cg * 2 + 1 - hh) * 8 + j) * 64 + p];
                        const int q = 32 * c + 8 * cg + j;
                        const __int128 T = mine[j & 3] + other + (__int128)rp128 * rowsum_q[j & 3];
                        const df v = int128_to_df(T);
                        c0[leaf * M + (nf == 2 ? f * n : 0) + q * kB + p] = make_float2(v.hi, v.lo);
                    }
                }
                fence_before();
                __syncthreads();
            }
        }
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && !ok && ctr) raise_error(ctr, kDevErrTimeout, 12u);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

bool corr_sep_tc_available(int b, int) { return b == septc::kB; }

cudaError_t launch_corr_sep_tc(const CorrArgs &a, cudaStream_t st) {
    const DictDev &d = *a.d;
    if (d.b != septc::kB || !d.tmap_sepd || !a.tmap_Ysep) return cudaErrorInvalidValue;
    const long long rows = a.count ? (long long)a.capacity : a.fixed_count;
    if (rows <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)(rows < sms ? rows : sms);
    e = cudaFuncSetAttribute(corr_sep_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, septc::kSmemBytes);
    if (e != cudaSuccess) return e;
    corr_sep_tc_kernel<<<grid, septc::kThreads, septc::kSmemBytes, st>>>(
        *reinterpret_cast<const CUtensorMap *>(a.tmap_Ysep), *reinterpret_cast<const CUtensorMap *>(d.tmap_sepd),
        d.nf, d.fam0, a.fmask ? a.fmask : 3, d.Rs, a.count, a.fixed_count, a.c0, a.ctr);
    return cudaGetLastError();
}

}  // namespace aqmp
