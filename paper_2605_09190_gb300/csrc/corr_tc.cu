// corr_tc.cu -- (a2) initial correlation c0 = D^T y for a batch of same-size
// leaves on the 5th-generation tensor cores (tcgen05.mma, TMEM accumulators,
// TMA loads), exact.
//
// D_fix = round(D 2^48) = sum_s d_s 64^(7-s) with balanced digits |d_s| <= 32;
// with y' = y - 128,
//     sum_v D_fix[j][v] y[v] = sum_s 64^(7-s) P_s[j] + 128 S_j,
//     P_s[j] = sum_v d_s[j][v] y'[v].
// Each P_s is one BF16 GEMM: digits and centred pixels are exact BF16
// values, products are at most 2^12 and |P_s| <= 2^24 for K <= 4096, so the
// FP32 accumulator in TMEM is exact.  The epilogue recombines the eight
// exact integers and rounds once to a double-float (fixed_to_df), which
// matches the SIMT kernel bit for bit.
//
// Above K = 4096 (side 128) the contraction runs as consecutive launches
// over K chunks of at most 4096: each chunk's eight accumulators are exact,
// the chunk's exact integer T_c = sum_s 64^(7-s) P_s (|T_c| < 2^62 for a
// unit-norm atom) is added into the output slot held as an int64, and the
// last chunk converts the total once -- the same value, rounded the same
// way, as a single pass.
//
// Tile: 128 atoms (TMEM lanes) x 64 leaves x the K range, eight accumulators
// of 64 columns each (the full 512-column TMEM).  One thread issues TMA loads, one
// issues MMAs, all four warps run the epilogue.  Every wait is bounded by a
// timer; on expiry the kernel records AQMP_E_TIMEOUT, releases its TMEM and
// returns.
#include <algorithm>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

// Largest K whose digit-plane sums stay exact in an FP32 accumulator
// (|P_s| <= 4096 * 2^5 * 2^7 = 2^24), and the roles of a launch over one K
// chunk.
constexpr int kCorrExactK = 4096;
enum { kCorrSingle = 0, kCorrFirst = 1, kCorrMiddle = 2, kCorrLast = 3 };

namespace tc {

constexpr int kM = 128;
constexpr int kN = 64;
constexpr int kK = 64;
constexpr int kStagesA = 8;
constexpr int kStagesB = 4;
constexpr int kTileA = kM * kK * 2;      // 16 KB
constexpr int kTileB = kN * kK * 2;      // 8 KB
constexpr int kTmemCols = 512;
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kStagesA * kTileA;
constexpr int kOffBar = kOffB + kStagesB * kTileB;
constexpr int kNumBars = 2 * kStagesA + 2 * kStagesB + 1;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;           // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity`; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned long long limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte
// swizzle, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ unsigned long long smem_desc(uint32_t addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3ffffu) >> 4);
    d |= (unsigned long long)1 << 16;                 // LBO (unused for this layout)
    d |= (unsigned long long)(1024 >> 4) << 32;       // SBO
    d |= (unsigned long long)1 << 46;                 // version
    d |= (unsigned long long)2 << 61;                 // 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);
// kind::f8f6f4 instruction descriptor: E4M3 x E4M3 (format code 0) -> F32.
constexpr uint32_t kIdesc8 = (1u << 4) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// One E4M3 MMA step of K = 32 (32 bytes of each 128-byte row, as K = 16
// of BF16, so the descriptors advance the same way).
__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc8), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc

// L = kLimbs: the exact form above.  L = 1: the reduced-precision form --
// one BF16 matrix bf16(D) against the centred pixels, FP32 accumulation,
// c0 = acc + 128 Sbf[j] (Sbf the row sums of bf16(D)), low word 0.
// FP8 (with L = 1): the FP8 form -- one E4M3 matrix e4m3(D s_j) against
// e4m3(y~ s_l), FP32 accumulation, c0 = acc / (s_j s_l) + 128 Sbf[j] with
// Sbf the dequantised row sums; a K block is 128 elements (one 128-byte row).
template <int L, bool FP8 = false>
__global__ void __launch_bounds__(tc::kThreads, 1)
corr_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
               int Mpad, int kb0, int KB, int mode, const long long *__restrict__ Sh,
               const long long *__restrict__ Sl, const float *__restrict__ Sbf, const unsigned *count_dev,
               long long fixed_count, float2 *__restrict__ c0, Counters *ctr,
               const float *__restrict__ inv_s_atom = nullptr, const float *__restrict__ inv_s_leaf = nullptr) {
    using namespace tc;
    constexpr int kKe = FP8 ? 2 * kK : kK;               // elements per 128-byte row
    const long long count = count_dev ? (long long)*count_dev : fixed_count;
    const long long leaf0 = (long long)blockIdx.x * kN;
    if (leaf0 >= count) return;                        // uniform: nothing to do
    const int m0 = blockIdx.y * kM;

    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const uint32_t sA = base + kOffA, sB = base + kOffB, sBar = base + kOffBar;
    auto fullA = [&](int i) { return sBar + 8u * i; };
    auto emptyA = [&](int i) { return sBar + 8u * (kStagesA + i); };
    auto fullB = [&](int i) { return sBar + 8u * (2 * kStagesA + i); };
    auto emptyB = [&](int i) { return sBar + 8u * (2 * kStagesA + kStagesB + i); };
    const uint32_t accBar = sBar + 8u * (2 * kStagesA + 2 * kStagesB);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(gbase + kOffMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStagesA; ++i) { mbar_init(fullA(i), 1); mbar_init(emptyA(i), 1); }
        for (int i = 0; i < kStagesB; ++i) { mbar_init(fullB(i), 1); mbar_init(emptyB(i), 1); }
        mbar_init(accBar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_holder)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int sa = 0, sb = 0;
        uint32_t pa = 0, pb = 0;
        for (int kb = 0; kb < KB && !*abort_flag; ++kb) {
            if (!mbar_wait(emptyB(sb), pb ^ 1u, abort_flag)) break;
            mbar_expect_tx(fullB(sb), kTileB);
            tma_load_2d(sB + sb * kTileB, &tmB, fullB(sb), (kb0 + kb) * kKe, (int)leaf0);
            if (++sb == kStagesB) { sb = 0; pb ^= 1u; }
            for (int s = 0; s < L; ++s) {
                if (!mbar_wait(emptyA(sa), pa ^ 1u, abort_flag)) break;
                mbar_expect_tx(fullA(sa), kTileA);
                tma_load_2d(sA + sa * kTileA, &tmA, fullA(sa), (kb0 + kb) * kKe, s * Mpad + m0);
                if (++sa == kStagesA) { sa = 0; pa ^= 1u; }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        int sa = 0, sb = 0;
        uint32_t pa = 0, pb = 0;
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            if (!(ok = mbar_wait(fullB(sb), pb, abort_flag))) break;
            for (int s = 0; s < L; ++s) {
                if (!(ok = mbar_wait(fullA(sa), pa, abort_flag))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned long long ad = smem_desc(sA + sa * kTileA);
                const unsigned long long bd = smem_desc(sB + sb * kTileB);
#pragma unroll
                for (int kk = 0; kk < kK / 16; ++kk) {
                    if (FP8)
                        mma_e4m3(tmem + (uint32_t)(s * kN), ad + 2ull * kk, bd + 2ull * kk,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                    else
                        mma_bf16(tmem + (uint32_t)(s * kN), ad + 2ull * kk, bd + 2ull * kk,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(emptyA(sa));
                if (++sa == kStagesA) { sa = 0; pa ^= 1u; }
            }
            if (!ok) break;
            mma_commit(emptyB(sb));
            if (++sb == kStagesB) { sb = 0; pb ^= 1u; }
        }
        mma_commit(accBar);                            // fires once every issued MMA is done
    }
    __syncwarp();

    // Epilogue: warp w reads TMEM lanes 32w..32w+31 (atoms m0 + 32w + lane).
    const bool acc_ok = mbar_wait(accBar, 0u, abort_flag) && !*abort_flag;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (acc_ok && L == 1) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const float centre = m < M ? 128.0f * Sbf[m] : 0.0f;
        const float inv_a = (FP8 && m < M) ? inv_s_atom[m] : 1.0f;
        for (int nb = 0; nb < kN; nb += 8) {
            float P[8];
            tmem_ld8(lane_addr + (uint32_t)nb, P);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const long long leaf = leaf0 + nb + i;
                    if (leaf < count) {
                        const float v = FP8 ? P[i] * inv_a * inv_s_leaf[leaf] : P[i];
                        c0[leaf * M + m] = make_float2(v + centre, 0.0f);
                    }
                }
            }
        }
    } else if (acc_ok) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const long long sh = m < M ? 128ll * Sh[m] : 0, sl = m < M ? 128ll * Sl[m] : 0;
        for (int nb = 0; nb < kN; nb += 8) {
            float P[kLimbs][8];
#pragma unroll
            for (int s = 0; s < kLimbs; ++s) tmem_ld8(lane_addr + (uint32_t)(s * kN + nb), P[s]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const long long leaf = leaf0 + nb + i;
                    if (leaf < count) {
                        long long top = 0, bot = 0;
#pragma unroll
                        for (int s = 0; s < 4; ++s) top = top * 64 + (long long)__float2int_rn(P[s][i]);
#pragma unroll
                        for (int s = 4; s < 8; ++s) bot = bot * 64 + (long long)__float2int_rn(P[s][i]);
                        long long *slot = reinterpret_cast<long long *>(c0 + leaf * M + m);
                        if (mode == kCorrSingle) {
                            const df v = fixed_to_df(top + sh, bot + sl);
                            c0[leaf * M + m] = make_float2(v.hi, v.lo);
                        } else {
                            long long T = top * (1ll << 24) + bot;      // this chunk, exact
                            if (mode != kCorrFirst) T += *slot;
                            if (mode == kCorrLast) {
                                const long long hi = T >> 24;           // floor; T = hi 2^24 + (T - hi 2^24)
                                const df v = fixed_to_df(hi + sh, (T - hi * (1ll << 24)) + sl);
                                c0[leaf * M + m] = make_float2(v.hi, v.lo);
                            } else {
                                *slot = T;
                            }
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag && ctr) raise_error(ctr, kDevErrTimeout, 10u);
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

bool corr_tc_available() { return true; }

cudaError_t launch_corr_tc_bf16(const CorrArgs &a, cudaStream_t st) {
    const DictDev &d = *a.d;
    if (!d.tmap_bf16 || !d.Sbf) return cudaErrorInvalidValue;
    const long long rows = a.count ? (long long)a.capacity : a.fixed_count;
    dim3 grid((unsigned)((rows + tc::kN - 1) / tc::kN), (unsigned)(d.Mpad / tc::kM));
    if (grid.x == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(corr_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::kSmemBytes);
    if (e != cudaSuccess) return e;
    const CUtensorMap *ma = reinterpret_cast<const CUtensorMap *>(d.tmap_bf16);
    const CUtensorMap *mb = reinterpret_cast<const CUtensorMap *>(a.tmap_Y);
    corr_tc_kernel<1><<<grid, tc::kThreads, tc::kSmemBytes, st>>>(*ma, *mb, d.M, d.Mpad, 0, d.Kpad / tc::kK,
                                                                  kCorrSingle, nullptr, nullptr, d.Sbf, a.count,
                                                                  a.fixed_count, a.c0, a.ctr);
    return cudaGetLastError();
}

cudaError_t launch_corr_tc_fp8(const CorrArgs &a, const float *inv_sl, cudaStream_t st) {
    const DictDev &d = *a.d;
    if (!d.tmap_fp8 || !d.S8 || !d.inv_s8 || !inv_sl) return cudaErrorInvalidValue;
    const long long rows = a.count ? (long long)a.capacity : a.fixed_count;
    dim3 grid((unsigned)((rows + tc::kN - 1) / tc::kN), (unsigned)(d.Mpad / tc::kM));
    if (grid.x == 0) return cudaSuccess;
    auto kern = corr_tc_kernel<1, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    if (e != cudaSuccess) return e;
    const CUtensorMap *ma = reinterpret_cast<const CUtensorMap *>(d.tmap_fp8);
    const CUtensorMap *mb = reinterpret_cast<const CUtensorMap *>(a.tmap_Y);
    kern<<<grid, tc::kThreads, tc::kSmemBytes, st>>>(*ma, *mb, d.M, d.Mpad, 0, kpad_fp8(d.n) / 128, kCorrSingle,
                                                     nullptr, nullptr, d.S8, a.count, a.fixed_count, a.c0, a.ctr,
                                                     d.inv_s8, inv_sl);
    return cudaGetLastError();
}

// Failure-path check: one thread waits, through the same bounded wait as the
// correlation kernel, on an mbarrier that nothing ever arrives on, and must
// give up after `limit_ns` and record AQMP_E_TIMEOUT in the error word.
__global__ void wait_selftest_kernel(Counters *ctr, unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    const uint32_t b = tc::smem_u32(&bar);
    tc::mbar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!tc::mbar_wait(b, 0u, &abort_flag, limit_ns)) raise_error(ctr, kDevErrTimeout, 99u);
}

cudaError_t launch_wait_selftest(Counters *ctr, unsigned long long limit_ns, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(ctr, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_corr_tc(const CorrArgs &a, cudaStream_t st) {
    const DictDev &d = *a.d;
    const long long rows = a.count ? (long long)a.capacity : a.fixed_count;
    dim3 grid((unsigned)((rows + tc::kN - 1) / tc::kN), (unsigned)(d.Mpad / tc::kM));
    if (grid.x == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(corr_tc_kernel<kLimbs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::kSmemBytes);
    if (e != cudaSuccess) return e;
    const CUtensorMap *ma = reinterpret_cast<const CUtensorMap *>(d.tmap_limbs);
    const CUtensorMap *mb = reinterpret_cast<const CUtensorMap *>(a.tmap_Y);
    // K chunks within the exactness bound of the FP32 accumulator
    const int kblocks = d.Kpad / tc::kK, chunk = kCorrExactK / tc::kK;
    const int chunks = (kblocks + chunk - 1) / chunk;
    for (int c = 0; c < chunks; ++c) {
        const int kb0 = c * chunk, kbs = std::min(chunk, kblocks - kb0);
        const int mode = chunks == 1 ? kCorrSingle : c == 0 ? kCorrFirst : c == chunks - 1 ? kCorrLast : kCorrMiddle;
        corr_tc_kernel<kLimbs><<<grid, tc::kThreads, tc::kSmemBytes, st>>>(
            *ma, *mb, d.M, d.Mpad, kb0, kbs, mode, d.Sh, d.Sl, nullptr, a.count, a.fixed_count, a.c0, a.ctr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace aqmp
