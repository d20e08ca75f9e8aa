// corr_sepbf_tc.cu -- the initial correlation of the BF16 form with rescore,
// side 64: c0 ~ B Y B^T per family (Section 2.1: the 2-D atoms are outer
// products of 1-D rows; Section 2.2 step (b)) from BF16 tensor-core
// products with FP32 accumulation, and with it a bound e_j on its error for
// every atom, which the rescoring pursuit uses to know which atoms could be
// the argmax (mp.cu).
//
// Operands.  Pixels centred on the block's integer mean mu, y~ = y - mu
// (exact in BF16); each 1-D row split B = B_hi + B_lo + d (B_hi = bf16(B),
// B_lo = bf16(B - B_hi), |d| <= 2^-16 |B|) and its magnitude rounded up,
// |B|^ >= |B|.
//   Stage 1 (per family): [B_hi ; B_lo] Y~ gives (lane half h, row p) the
//     two parts of Z = B Y~; both halves add them in the same order,
//     Z~ = fl(P_hi + P_lo), and split it again: half 0 keeps bf16(Z~), half 1
//     bf16(Z~ - bf16(Z~)), as the stage-2 A operand in tensor memory.  For
//     the bound, [|B_0|^ ; |B_1|^] |Y~| gives Q_F, rounded up to BF16 after a
//     2^-18 relative margin.
//   Stage 2 (per family): [Z_hi ; Z_lo] B_hi^T and [Z_hi ; Z_lo] B_lo^T; the
//     four parts are summed in double-float.  Q^ |B_F|^T gives S_j >= the
//     atom's mass sum_{i,m} |B[p][i]| |y~[i][m]| |B[q][m]|.
//   Epilogue: c0_j = that sum + mu R[p] R[q] (double-float), and
//     e_j = 25 2^-19 S_j + 2^-40 mu |R[p] R[q]| + 2^-30 (the last term the
//     exact form's distance from the real correlation).
// Error budget (per atom, S its mass): the three splits 2^-16 S each; the
// FP32 accumulation, with each MMA of K = 16 taken to err by at most two
// units in the last place of the running magnitude (|D| + sum |a b|), 4
// MMAs per chain: 11.2 u S in stage 1 (products, the P_hi + P_lo sum) and
// 10.1 u S in stage 2 (u = 2^-24); in all 3 2^-16 S + 21.3 u S < 3.09 2^-16 S,
// below 25 2^-19 = 3.125 2^-16 with room for the double-float sums and the
// 2^-48 fixed-point dictionary of the exact form the rescore compares with.
//
// One CTA of 16 warps per SM (4 per TMEM lane quarter), persistent over the
// leaves, 448 TMEM columns: stage 1 at 0..191 (Q, then the two families'
// parts), the A operands at 192..287, stage 2 at 288..479 and, over the
// drained stage-1 columns, 0..191.  The dictionary tiles (48 KB) stay in
// shared memory; each leaf's pixels arrive by TMA into a double buffer.
// Thread 0 issues TMA and MMA, all warps drain.  Every wait is bounded by a
// timer; on expiry the kernel records AQMP_E_TIMEOUT, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "df.cuh"
#include "kernels.h"
#include "tc_sep.cuh"

namespace aqmp {

namespace sepbf {

constexpr int kB = 64;
constexpr int kThreads = 512;
constexpr int kTmemCols = 512;
// tensor-memory columns
constexpr int kColQ = 0, kColP0 = 64, kColP1 = 128;         // stage 1
constexpr int kColA0 = 192, kColA1 = 224, kColAQ = 256;     // stage-2 A operands (32 columns each)
constexpr int kColHi0 = 288, kColLo0 = 352, kColHi1 = 416;  // stage 2
constexpr int kColLo1 = 0, kColE0 = 64, kColE1 = 128;       // stage 2, over drained stage-1 columns
// shared memory
constexpr int kTile = 128 * 128;                            // 128 rows x 64 BF16
constexpr int kTileY = 64 * 128;                            // 64 rows (m) x 64 BF16 (i)
constexpr int kOffD = 0;                                    // [B_hi;B_lo] F=0, F=1, [|B_0|;|B_1|]
constexpr int kOffY = kOffD + 3 * kTile;                    // two buffers
constexpr int kOffA = kOffY + 2 * kTileY;                   // |y~|
constexpr int kOffX = kOffA + kTileY;                       // exchange: 2 x 64 x 64 floats
constexpr int kBytesX = 2 * 64 * 64 * 4;
constexpr int kOffBar = kOffX + kBytesX;
constexpr int kOffMisc = kOffBar + 8 * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;

constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);       // M = 128, N = 64, BF16 -> F32
constexpr float kRel = 25.0f * 0x1p-19f;
// the exact form's own distance from the real correlation (its 2^-48
// fixed-point rows: 2^-49 sum_v (|B[p][i]| + |B[q][m]|) y_v < 2^-31 for 8-bit
// pixels at side 64, and its double-float rounding < 2^-34)
constexpr float kFix = 0x1p-30f;

static_assert(kSmemBytes <= 232448, "shared memory above the per-block limit");

// BF16 bits of x rounded up (toward +inf); x >= 0 finite.
__device__ __forceinline__ uint32_t bf16_up_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u >> 16) + ((u & 0xffffu) != 0u ? 1u : 0u);
}

// BF16 bits of x rounded to nearest, ties to even.
__device__ __forceinline__ uint32_t bf16_rn_bits(float x) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float bf16_bits_to_float(uint32_t b) { return __uint_as_float(b << 16); }

}  // namespace sepbf

// Y map: the gathered leaves (centred on their means) as [capacity * 64 rows]
// [64] BF16, row m of leaf l at row 64 l + m (K = i); dictionary map:
// [384 rows][64] BF16 in boxes of 128 rows (the three tiles).
__global__ void __launch_bounds__(sepbf::kThreads, 1)
corr_sepbf_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmD, int nf,
                     int fam0, const float2 *__restrict__ Rbf, const uint8_t *__restrict__ mu,
                     const unsigned *count_dev, long long fixed_count, float2 *__restrict__ c0,
                     float *__restrict__ ebound, Counters *ctr) {
    using namespace septc;
    using namespace sepbf;
    constexpr int n = kB * kB;
    const long long count = count_dev ? (long long)*count_dev : fixed_count;
    if ((long long)blockIdx.x >= count) return;                  // uniform
    const int M = nf * n;

    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const uint32_t sD = base + kOffD, sY = base + kOffY, sA = base + kOffA, sBar = base + kOffBar;
    const uint32_t barD = sBar, barY0 = sBar + 8, barY1 = sBar + 16, barMma = sBar + 24;
    float *X = reinterpret_cast<float *>(gbase + kOffX);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(gbase + kOffMisc);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(barD, 1);
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

    if (threadIdx.x == 0) {
        mbar_expect_tx(barD, 3 * kTile);
        for (int t = 0; t < 3; ++t) tma_load_2d(sD + t * kTile, &tmD, barD, 0, 128 * t);
        mbar_expect_tx(barY0, kTileY);
        tma_load_2d(sY, &tmY, barY0, 0, (int)(64 * blockIdx.x));
    }
    bool ok = __syncthreads_and(mbar_wait(barD, 0)) != 0;

    const int quarter = warp & 3, cg = warp >> 2;
    const int row = quarter * 32 + lane;                          // TMEM lane = (half, p)
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int hl = row >> 6, p = row & 63;
    uint32_t mma_phase = 0, y_phase[2] = {0u, 0u};
    int it = 0;
    for (long long leaf = blockIdx.x; ok && leaf < count; leaf += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t barY = buf ? barY1 : barY0;
        ok = __syncthreads_and(mbar_wait(barY, y_phase[buf])) != 0;
        y_phase[buf] ^= 1u;
        if (!ok) break;
        if (threadIdx.x == 0 && leaf + gridDim.x < count) {
            const uint32_t nb = buf ? barY0 : barY1;
            mbar_expect_tx(nb, kTileY);
            tma_load_2d(sY + (buf ^ 1) * kTileY, &tmY, nb, 0, (int)(64 * (leaf + gridDim.x)));
        }
        const uint32_t yaddr = sY + buf * kTileY;
        // |y~|: the sign bits cleared in place of the same (swizzled) layout
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(gbase + kOffY + buf * kTileY);
            uint32_t *dst = reinterpret_cast<uint32_t *>(gbase + kOffA);
            for (int i = threadIdx.x; i < kTileY / 4; i += kThreads) dst[i] = src[i] & 0x7fff7fffu;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- stage 1: Q = [|B_0|^;|B_1|^] |y~|, P_f = [B_hi;B_lo] y~
        if (threadIdx.x == 0) {
            fence_after();
            const unsigned long long aq = smem_desc(sD + 2 * kTile), bq = smem_desc(sA), by = smem_desc(yaddr);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_ss(tmem + kColQ, aq + 2ull * kk, bq + 2ull * kk, kIdesc, kk ? 1u : 0u);
            for (int f = 0; f < nf; ++f) {
                const int F = nf == 2 ? f : fam0;
                const unsigned long long ap = smem_desc(sD + F * kTile);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_ss(tmem + (f ? kColP1 : kColP0), ap + 2ull * kk, by + 2ull * kk, kIdesc, kk ? 1u : 0u);
            }
            mma_commit(barMma);
        }
        ok = __syncthreads_and(mbar_wait(barMma, mma_phase)) != 0;
        mma_phase ^= 1u;
        if (!ok) break;
        fence_after();
        // ---- drain 1.  Q (lanes (F, p)) -> Q^ as the A operand of the bound
        {
            uint32_t r[16], pk[8];
            tmem_ld16(lane_base + kColQ + 16 * cg, r);
            wait_ld();
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                const uint32_t lo = bf16_up_bits(__fmul_ru(__uint_as_float(r[2 * j2]), 1.0f + 0x1p-18f));
                const uint32_t hi = bf16_up_bits(__fmul_ru(__uint_as_float(r[2 * j2 + 1]), 1.0f + 0x1p-18f));
                pk[j2] = lo | (hi << 16);
            }
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                         ::"r"(lane_base + kColAQ + 8 * cg), "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3]),
                           "r"(pk[4]), "r"(pk[5]), "r"(pk[6]), "r"(pk[7])
                         : "memory");
        }
        // P_f (lanes (h, p)): both halves form Z~ = fl(P_hi + P_lo) through
        // the exchange (m-major: the lanes of a warp hit consecutive words)
        for (int f = 0; f < nf; ++f) {
            uint32_t r[16];
            tmem_ld16(lane_base + (f ? kColP1 : kColP0) + 16 * cg, r);
            wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) X[(hl * 64 + 16 * cg + j) * 64 + p] = __uint_as_float(r[j]);
            __syncthreads();
            uint32_t pk[8];
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                uint32_t h2[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = 2 * j2 + e;
                    const float z = __fadd_rn(__uint_as_float(r[j]), X[((1 - hl) * 64 + 16 * cg + j) * 64 + p]);
                    const uint32_t zh = bf16_rn_bits(z);
                    h2[e] = hl == 0 ? zh : bf16_rn_bits(__fsub_rn(z, bf16_bits_to_float(zh)));
                }
                pk[j2] = h2[0] | (h2[1] << 16);
            }
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                         ::"r"(lane_base + (f ? kColA1 : kColA0) + 8 * cg), "r"(pk[0]), "r"(pk[1]), "r"(pk[2]),
                           "r"(pk[3]), "r"(pk[4]), "r"(pk[5]), "r"(pk[6]), "r"(pk[7])
                         : "memory");
            __syncthreads();
        }
        wait_st();
        fence_before();
        __syncthreads();
        // ---- stage 2
        if (threadIdx.x == 0) {
            fence_after();
            for (int f = 0; f < nf; ++f) {
                const int F = nf == 2 ? f : fam0;
                const uint32_t a2 = tmem + (f ? kColA1 : kColA0);
                const unsigned long long bh = smem_desc(sD + F * kTile), bl = smem_desc(sD + F * kTile + 64 * 128),
                                         be = smem_desc(sD + 2 * kTile + F * 64 * 128);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t acc = kk ? 1u : 0u;
                    mma_ts(tmem + (f ? kColHi1 : kColHi0), a2 + 8 * kk, bh + 2ull * kk, kIdesc, acc);
                    mma_ts(tmem + (f ? kColLo1 : kColLo0), a2 + 8 * kk, bl + 2ull * kk, kIdesc, acc);
                    mma_ts(tmem + (f ? kColE1 : kColE0), tmem + kColAQ + 8 * kk, be + 2ull * kk, kIdesc, acc);
                }
            }
            mma_commit(barMma);
        }
        const float muf = (float)mu[leaf];
        ok = __syncthreads_and(mbar_wait(barMma, mma_phase)) != 0;
        mma_phase ^= 1u;
        if (!ok) break;
        fence_after();
        // ---- drain 2: the (h, p) parts of T in double-float, the lo half
        // handed to the hi half; the bound from the lanes of family F
        float2 *X2 = reinterpret_cast<float2 *>(X);
        for (int f = 0; f < nf; ++f) {
            const int F = nf == 2 ? f : fam0;
            uint32_t rh[16], rl[16];
            tmem_ld16(lane_base + (f ? kColHi1 : kColHi0) + 16 * cg, rh);
            tmem_ld16(lane_base + (f ? kColLo1 : kColLo0) + 16 * cg, rl);
            wait_ld();
            df s[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) s[j] = df_two_sum(__uint_as_float(rh[j]), __uint_as_float(rl[j]));
            if (hl == 1) {
#pragma unroll
                for (int j = 0; j < 16; ++j) X2[(16 * cg + j) * 64 + p] = make_float2(s[j].hi, s[j].lo);
            }
            const size_t obase = (size_t)leaf * M + (nf == 2 ? (size_t)f * n : 0);
            const float2 rp = Rbf[F * kB + p];
            if (hl == F) {
                uint32_t re[16];
                tmem_ld16(lane_base + (f ? kColE1 : kColE0) + 16 * cg, re);
                wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int q = 16 * cg + j;
                    const float rq = Rbf[F * kB + q].x;
                    const float e = __fadd_ru(__fadd_ru(__fmul_ru(kRel, __uint_as_float(re[j])),
                                                        __fmul_ru(0x1p-40f, __fmul_ru(muf, fabsf(rp.x * rq) * 1.001f))),
                                              kFix);
                    ebound[obase + (size_t)q * kB + p] = e;
                }
            }
            __syncthreads();
            if (hl == 0) {
                const df mrp = df_mul(df{rp.x, rp.y}, df{muf, 0.0f});
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int q = 16 * cg + j;
                    const float2 o = X2[q * 64 + p];
                    const float2 rq = Rbf[F * kB + q];
                    df v = df_add(s[j], df{o.x, o.y});
                    v = df_add(v, df_mul(mrp, df{rq.x, rq.y}));
                    c0[obase + (size_t)q * kB + p] = make_float2(v.hi, v.lo);
                }
            }
            __syncthreads();
        }
        fence_before();
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && !ok && ctr) raise_error(ctr, kDevErrTimeout, 14u);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

bool corr_sepbf_available(int b) { return b == sepbf::kB; }

cudaError_t launch_corr_sepbf(const CorrArgs &a, cudaStream_t st) {
    const DictDev &d = *a.d;
    if (d.b != sepbf::kB || !d.tmap_sepbf || !a.tmap_Ysep || !a.mu || !a.ebound) return cudaErrorInvalidValue;
    const long long rows = a.count ? (long long)a.capacity : a.fixed_count;
    if (rows <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)(rows < sms ? rows : sms);
    e = cudaFuncSetAttribute(corr_sepbf_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sepbf::kSmemBytes);
    if (e != cudaSuccess) return e;
    corr_sepbf_tc_kernel<<<grid, sepbf::kThreads, sepbf::kSmemBytes, st>>>(
        *reinterpret_cast<const CUtensorMap *>(a.tmap_Ysep), *reinterpret_cast<const CUtensorMap *>(d.tmap_sepbf),
        d.nf, d.fam0, d.Rbf, a.mu, a.count, a.fixed_count, a.c0, a.ebound, a.ctr);
    return cudaGetLastError();
}

}  // namespace aqmp
