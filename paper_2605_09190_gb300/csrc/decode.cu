// decode.cu -- Algorithm 3 (mp_decoder): for every leaf of one plane,
// y = D_N x, un-ravel, and place the block at its position.  Each pixel
// sums alpha_t B[p_t][i] B[q_t][m] over the leaf's atoms in FP32 (the stored
// coefficients are FP32); atoms listed twice simply add.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

// Leaves of `plane` in canonical order form one range (planes ascending).
__device__ __forceinline__ void plane_range(const LeafRec *leaves, unsigned long long n, uint32_t plane,
                                            unsigned long long &lo, unsigned long long &hi) {
    unsigned long long a = 0, b = n;
    while (a < b) {                                    // first leaf with plane >= `plane`
        const unsigned long long m = (a + b) >> 1;
        if (leaves[m].plane < plane) a = m + 1; else b = m;
    }
    lo = a;
    b = n;
    while (a < b) {                                    // first leaf with plane > `plane`
        const unsigned long long m = (a + b) >> 1;
        if (leaves[m].plane <= plane) a = m + 1; else b = m;
    }
    hi = a;
}

constexpr int kDecodeThreads = 128;
constexpr int kDecodeChunk = 256;                      // atoms staged per pass

struct DecodeStage {
    float al[kDecodeChunk];
    int p[kDecodeChunk], q[kDecodeChunk];
};

// One leaf of side B on the whole CTA: its atoms staged in shared memory as
// (alpha, offset of row p, offset of row q) into the FP32 basis of their
// family, so the per-pixel loop is two loads and two multiply-adds.  Side
// 128 runs over its pixels in four passes (32 accumulators per thread, as
// at side 64), re-staging the atoms for each.
template <int B>
__device__ __forceinline__ void decode_leaf(const DecodeArgs &a, const float *alpha, const LeafRec &L,
                                            DecodeStage &st) {
    constexpr int n = B * B;
    constexpr int PASSES = B > 64 ? (B / 64) * (B / 64) : 1;
    constexpr int NP = n / PASSES;                     // pixels per pass
    constexpr int PER = (NP + kDecodeThreads - 1) / kDecodeThreads;
    constexpr int LG = B == 4 ? 2 : B == 8 ? 3 : B == 16 ? 4 : B == 32 ? 5 : B == 64 ? 6 : 7;
    const float *basis = a.basis[LG];
#pragma unroll 1
    for (int pass = 0; pass < PASSES; ++pass) {
        float acc[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) acc[r] = 0.0f;
        for (int t0 = 0; t0 < L.n_atoms; t0 += kDecodeChunk) {
            const int cnt = min(kDecodeChunk, (int)L.n_atoms - t0);
            __syncthreads();
            for (int t = threadIdx.x; t < cnt; t += kDecodeThreads) {
                const AtomRec at = a.atoms[L.atom_off + t0 + t];
                int fam = (int)(at.j >= (uint32_t)n);
                const int f = (int)at.j - fam * n;
                if (a.nf == 1) fam = a.single_family;
                st.al[t] = alpha ? alpha[L.atom_off + t0 + t] : at.alpha;
                st.p[t] = fam * n + (f % B) * B;
                st.q[t] = fam * n + (f / B) * B;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int v = pass * NP + threadIdx.x + r * kDecodeThreads;
                if (threadIdx.x + r * kDecodeThreads < NP) {
                    const int m = v / B, i = v % B;
                    float s = acc[r];
                    for (int t = 0; t < cnt; ++t)
                        s = __fmaf_rn(st.al[t], __fmul_rn(basis[st.p[t] + i], basis[st.q[t] + m]), s);
                    acc[r] = s;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int v = pass * NP + threadIdx.x + r * kDecodeThreads;
            if (threadIdx.x + r * kDecodeThreads < NP)
                a.out[(long long)(L.y + v % B) * a.out_pitch + L.x + v / B] = acc[r];
        }
    }
    __syncthreads();
}

// One CTA per leaf of the plane.  `alpha` overrides the code's coefficients
// when not NULL (synthesis with caller coefficients).  BIG = false serves
// sides up to 64; BIG = true only side 128, in a launch of its own so that
// its register needs do not lower the occupancy of the common sizes.
template <bool BIG>
__global__ void __launch_bounds__(kDecodeThreads) decode_kernel(DecodeArgs a, const float *alpha) {
    __shared__ DecodeStage st;
    __shared__ unsigned long long s_range[2];
    if (threadIdx.x == 0) plane_range(a.leaves, a.n_leaves, a.plane, s_range[0], s_range[1]);
    __syncthreads();
    const unsigned long long lo = s_range[0], hi = s_range[1];
    for (unsigned long long li = lo + blockIdx.x; li < hi; li += gridDim.x) {
        const LeafRec L = a.leaves[li];
        if (BIG) {
            if (L.b == 128) decode_leaf<128>(a, alpha, L, st);
            continue;
        }
        switch (L.b) {
            case 4: decode_leaf<4>(a, alpha, L, st); break;
            case 8: decode_leaf<8>(a, alpha, L, st); break;
            case 16: decode_leaf<16>(a, alpha, L, st); break;
            case 32: decode_leaf<32>(a, alpha, L, st); break;
            case 64: decode_leaf<64>(a, alpha, L, st); break;
            default: break;
        }
    }
}

cudaError_t launch_decode_alpha(const DecodeArgs &a, const float *alpha, int num_sms, cudaStream_t st) {
    if (a.n_leaves == 0) return cudaSuccess;
    long long blocks = (long long)a.n_leaves;
    long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    decode_kernel<false><<<(unsigned)blocks, kDecodeThreads, 0, st>>>(a, alpha);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.basis[7] == nullptr) return e;      // no side-128 table: no side-128 leaves
    decode_kernel<true><<<(unsigned)blocks, kDecodeThreads, 0, st>>>(a, alpha);
    return cudaGetLastError();
}

cudaError_t launch_decode(const DecodeArgs &a, int num_sms, cudaStream_t st) {
    return launch_decode_alpha(a, nullptr, num_sms, st);
}

}  // namespace aqmp
