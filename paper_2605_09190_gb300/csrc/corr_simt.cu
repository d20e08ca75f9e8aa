// corr_simt.cu -- (a2) initial correlation c0 = D^T y on the integer SIMT
// pipes, exact.  Used to validate the tensor-core kernel bit for bit and
// selectable with AQMP_FLAG_SIMT_GEMM.
//
// With D_fix = round(D 2^48) = Dh 2^24 + Dl and the centred block y' = y - 128,
// T_j = sum_v D_fix[j][v] y[v] = (sum_v Dh y' + 128 Sh) 2^24 + (sum_v Dl y' + 128 Sl),
// every product fitting in 32 bits and every sum in 64; fixed_to_df rounds
// T_j 2^-48 once into a double-float.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

constexpr int kSimtAtoms = 64;   // atoms per CTA tile
constexpr int kSimtLeaves = 16;  // leaves per CTA tile
constexpr int kSimtK = 32;       // K chunk staged in shared memory

__global__ void __launch_bounds__(256)
corr_simt_kernel(int n, int M, int Kpad, const int32_t *__restrict__ Dh, const int32_t *__restrict__ Dl,
                 const long long *__restrict__ Sh, const long long *__restrict__ Sl,
                 const __nv_bfloat16 *__restrict__ Y, const unsigned *count_dev, long long fixed_count,
                 float2 *__restrict__ c0) {
    const long long count = count_dev ? (long long)*count_dev : fixed_count;
    const long long leaf0 = (long long)blockIdx.x * kSimtLeaves;
    if (leaf0 >= count) return;
    const int atom0 = blockIdx.y * kSimtAtoms;

    __shared__ int32_t sDh[kSimtAtoms][kSimtK + 1];
    __shared__ int32_t sDl[kSimtAtoms][kSimtK + 1];
    __shared__ int32_t sY[kSimtLeaves][kSimtK + 1];

    const int tid = threadIdx.x;
    const int a_local = tid & (kSimtAtoms - 1);          // one atom per thread
    const int l_base = (tid >> 6) * 4;                   // four leaves per thread
    long long acc_h[4] = {0, 0, 0, 0}, acc_l[4] = {0, 0, 0, 0};

    for (int k0 = 0; k0 < n; k0 += kSimtK) {
        for (int i = tid; i < kSimtAtoms * kSimtK; i += 256) {
            const int r = i / kSimtK, c = i - r * kSimtK;
            const int j = atom0 + r, v = k0 + c;
            const bool ok = j < M && v < n;
            sDh[r][c] = ok ? Dh[(size_t)j * n + v] : 0;
            sDl[r][c] = ok ? Dl[(size_t)j * n + v] : 0;
        }
        for (int i = tid; i < kSimtLeaves * kSimtK; i += 256) {
            const int r = i / kSimtK, c = i - r * kSimtK;
            const long long l = leaf0 + r;
            const int v = k0 + c;
            sY[r][c] = (l < count && v < n) ? (int32_t)__bfloat162float(Y[l * Kpad + v]) : 0;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < kSimtK; ++c) {
            const int32_t dh = sDh[a_local][c], dl = sDl[a_local][c];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t y = sY[l_base + q][c];
                acc_h[q] += (long long)(dh * y);         // |dh y| <= 2^30
                acc_l[q] += (long long)(dl * y);
            }
        }
        __syncthreads();
    }
    const int j = atom0 + a_local;
    if (j >= M) return;
    const long long sh = 128ll * Sh[j], sl = 128ll * Sl[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long l = leaf0 + l_base + q;
        if (l < count) {
            const df v = fixed_to_df(acc_h[q] + sh, acc_l[q] + sl);
            c0[l * M + j] = make_float2(v.hi, v.lo);
        }
    }
}

cudaError_t launch_corr_simt(const CorrArgs &a, cudaStream_t st) {
    const DictDev &d = *a.d;
    const long long rows = a.count ? (long long)a.capacity : a.fixed_count;
    dim3 grid((unsigned)((rows + kSimtLeaves - 1) / kSimtLeaves), (unsigned)((d.M + kSimtAtoms - 1) / kSimtAtoms));
    if (grid.x == 0) return cudaSuccess;
    corr_simt_kernel<<<grid, 256, 0, st>>>(d.n, d.M, d.Kpad, d.Dh, d.Dl, d.Sh, d.Sl, a.Y, a.count,
                                           a.fixed_count, a.c0);
    return cudaGetLastError();
}

}  // namespace aqmp
