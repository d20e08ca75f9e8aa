// decode.cu -- Algorithm 3 (mp_decoder): for every leaf of one plane,
// y = D_N x, un-ravel, and place the block at its position.  Each pixel
// sums alpha_t B[p_t][i] B[q_t][m] over the leaf's atoms in FP32 (the stored
// coefficients are FP32); atoms listed twice simply add.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

__global__ void __launch_bounds__(128) decode_kernel(DecodeArgs a) {
    for (unsigned long long li = blockIdx.x; li < a.n_leaves; li += gridDim.x) {
        const LeafRec L = a.leaves[li];
        if (L.plane != a.plane) continue;
        const int b = L.b, n = b * b;
        int lg = 0;
        while ((1 << lg) < b) ++lg;
        const float *basis = a.basis[lg];
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const int m = v / b, i = v - m * b;
            float s = 0.0f;
            for (int t = 0; t < L.n_atoms; ++t) {
                const AtomRec at = a.atoms[L.atom_off + t];
                int fam = (int)(at.j >= (uint32_t)n);
                const int f = (int)at.j - fam * n;
                if (a.nf == 1) fam = a.single_family;
                const float *B = basis + fam * b * b;
                const int p = f % b, q = f / b;
                s = __fmaf_rn(at.alpha, __fmul_rn(B[p * b + i], B[q * b + m]), s);
            }
            a.out[(long long)(L.y + i) * a.out_pitch + L.x + m] = s;
        }
    }
}

cudaError_t launch_decode(const DecodeArgs &a, int num_sms, cudaStream_t st) {
    if (a.n_leaves == 0) return cudaSuccess;
    long long blocks = (long long)a.n_leaves;
    long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    decode_kernel<<<(unsigned)blocks, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace aqmp
