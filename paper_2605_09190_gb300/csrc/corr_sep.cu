// corr_sep.cu -- (a2) initial correlation with the separable fixed-point
// dictionary (sep.cuh) on the integer SIMT pipes: exact, and the reference
// twin of the tensor-core kernel of corr_sep_tc.cu (same bits).
//
// Section 2.2 step (b) needs <r0, phi_j> for every atom j.  The DCT-II and
// Haar atoms are outer products of 1-D rows (Section 2.1), so the M = 2 b^2
// correlations of a block are B Y B^T for each family: two b x b x b products
// (8 b^3 multiply-adds for both families) instead of the 4 b^4 of a dense
// D^T y.  In integers:
//   stage 1  Z~[p][m] = sum_i Bf[p][i] y~[i][m]   (48-bit x 8-bit -> int64)
//   stage 2  T~[p][q] = sum_m Bf[q][m] Z~[p][m]   (48-bit x 59-bit -> int128)
// Bf is held as 24-bit limbs (lo in [-2^23, 2^23), hi = (Bf - lo) / 2^24,
// |hi| < 2^23.5) and Z~ as two 32-bit ones (zl in [-2^31, 2^31), zh =
// (Z~ - zl) / 2^32, |zh| < 2^27), so every partial product is one 32 x 32 ->
// 64-bit multiply-add, at most 2^54.5 in magnitude, and each of the four
// limb sums over b <= 128 terms stays below 2^62.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "sep.cuh"

namespace aqmp {

namespace {

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

// Threads per CTA: at side 128 the leaf's Z~ (128 KB of limbs) leaves room
// for one CTA per SM, so that CTA takes 768 threads to hide the latency of
// its loads; 256 elsewhere.
template <int B>
constexpr int sep_threads() { return B >= 128 ? 768 : 256; }

// One CTA handles G leaves at a time (grid-stride over the leaves); for each
// family it runs stage 1 into shared memory (Z~ as limbs, row p, column m),
// then stage 2 with each thread owning one q and PT values of p.
template <int B>
__global__ void __launch_bounds__(sep_threads<B>())
corr_sep_simt_kernel(int nf, int fam0, int Kpad, const int2 *__restrict__ Bs, const int2 *__restrict__ BsT,
                     const long long *__restrict__ Rs, const __nv_bfloat16 *__restrict__ Y,
                     const unsigned *count_dev, long long fixed_count, float2 *__restrict__ c0) {
    constexpr int n = B * B;
    constexpr int G = sep_group<B>();
    constexpr int PT = B >= 4 ? 4 : B;                   // p values per thread in stage 2
    extern __shared__ __align__(16) unsigned char smem[];
    int8_t *yt = reinterpret_cast<int8_t *>(smem);                        // [G][i][m]
    Limbs2 *Z = reinterpret_cast<Limbs2 *>(smem + ((G * n + 15) & ~15)); // [G][p][m]

    const long long count = count_dev ? (long long)*count_dev : fixed_count;
    const int M = nf * n;
    const int tid = threadIdx.x;
    for (long long base = (long long)blockIdx.x * G; base < count; base += (long long)gridDim.x * G) {
        const int live = (int)min((long long)G, count - base);
        // centred pixels, transposed so that stage 1 reads consecutive m
        for (int o = tid; o < G * n; o += blockDim.x) {
            const int g = o / n, v = o - g * n;
            const int m = v / B, i = v - m * B;
            int8_t y = 0;
            if (g < live) y = (int8_t)__bfloat162float(Y[(base + g) * Kpad + v]);
            yt[g * n + i * B + m] = y;
        }
        __syncthreads();
        for (int f = 0; f < nf; ++f) {
            const int F = nf == 2 ? f : fam0;
            const int2 *Bf = Bs + (size_t)F * n;
            const int2 *BfT = BsT + (size_t)F * n;
            const long long *R = Rs + F * B;
            // stage 1: Z~[g][p][m], m fastest across threads
            for (int o = tid; o < G * n; o += blockDim.x) {
                const int g = o / n, r = o - g * n;
                const int p = r / B, m = r - p * B;
                long long lo = 0, hi = 0;
#pragma unroll 8
                for (int i = 0; i < B; ++i) {
                    const int2 w = Bf[p * B + i];
                    const int32_t y = yt[g * n + i * B + m];
                    lo += mul_wide(w.x, y);
                    hi += mul_wide(w.y, y);
                }
                Z[g * n + p * B + m] = split2(hi * (1ll << 24) + lo);   // |hi 2^24| < 2^63
            }
            __syncthreads();
            // stage 2: T~[g][p][q] for q = lane-fastest, PT values of p per thread
            for (int o = tid; o < G * n / PT; o += blockDim.x) {
                const int g = o / (n / PT), r = o - g * (n / PT);
                const int q = r % B, p0 = (r / B) * PT;
                long long a0[PT], a1[PT], a2[PT], a3[PT];
#pragma unroll
                for (int k = 0; k < PT; ++k) a0[k] = a1[k] = a2[k] = a3[k] = 0;
#pragma unroll 4
                for (int m = 0; m < B; ++m) {
                    const int2 w = BfT[m * B + q];                 // Bf[q][m]: (lo, hi)
#pragma unroll
                    for (int k = 0; k < PT; ++k) {
                        const Limbs2 z = Z[g * n + (p0 + k) * B + m];
                        a0[k] += mul_wide(w.x, z.zl);              // weight 1
                        a1[k] += mul_wide(w.y, z.zl);              // 2^24
                        a2[k] += mul_wide(w.x, z.zh);              // 2^32
                        a3[k] += mul_wide(w.y, z.zh);              // 2^56
                    }
                }
                if (g < live) {
#pragma unroll
                    for (int k = 0; k < PT; ++k) {
                        const int p = p0 + k;
                        __int128 T = (__int128)a3[k] * ((__int128)1 << 56) + (__int128)a2[k] * ((__int128)1 << 32) +
                                     (__int128)a1[k] * ((__int128)1 << 24) + (__int128)a0[k];
                        T += (__int128)(128ll * R[p]) * R[q];
                        const df c = int128_to_df(T);
                        c0[(base + g) * M + (nf == 2 ? f * n : 0) + q * B + p] = make_float2(c.hi, c.lo);
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int B>
static cudaError_t launch_sep_simt_t(const CorrArgs &a, cudaStream_t st) {
    constexpr int G = sep_group<B>();
    const size_t smem = (size_t)((G * B * B + 15) & ~15) + sizeof(Limbs2) * G * B * B;
    auto kern = corr_sep_simt_kernel<B>;
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
    kern<<<(unsigned)grid, sep_threads<B>(), smem, st>>>(d.nf, d.fam0, d.Kpad, d.Bs, d.BsT, d.Rs, a.Y, a.count,
                                                          a.fixed_count, a.c0);
    return cudaGetLastError();
}

cudaError_t launch_corr_sep_simt(const CorrArgs &a, cudaStream_t st) {
    switch (a.d->b) {
        case 4: return launch_sep_simt_t<4>(a, st);
        case 8: return launch_sep_simt_t<8>(a, st);
        case 16: return launch_sep_simt_t<16>(a, st);
        case 32: return launch_sep_simt_t<32>(a, st);
        case 64: return launch_sep_simt_t<64>(a, st);
        case 128: return launch_sep_simt_t<128>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace aqmp
