// tables.cu -- fixed-point dictionary tables built on the device from the
// FP64 1-D bases.
//
// Atom j of a family with 1-D matrix B is the 2-D atom (p, q) = (f mod b,
// f div b), f = j - family * b^2, and its entry at v = m b + i is
// B[p][i] B[q][m] (Section 2.1: outer products of 1-D rows; Appendix A:
// columns concatenated).  Each entry is put in fixed point,
// D_fix = round(D 2^48), and stored three ways: as 8 balanced base-64 BF16
// digits for the tensor cores, as a (Dh, Dl) pair for the SIMT kernel, and
// through its per-atom sum for the centring correction.
#include <algorithm>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

__device__ __forceinline__ long long fixed_entry(const double *basis, int b, int n, int nf, int fam0,
                                                 int j, int v) {
    const int fam = nf == 2 ? j / n : fam0;
    const int f = j - (nf == 2 ? (j / n) * n : 0);
    const int p = f % b, q = f / b;
    const int m = v / b, i = v - m * b;
    const double *B = basis + (size_t)fam * b * b;
    const double d = B[p * b + i] * B[q * b + m];
    return __double2ll_rn(d * 281474976710656.0);      // exact scaling by 2^48, then round
}

__global__ void fixed_tables_kernel(int b, int n, int M, int nf, int fam0, const double *basis,
                                    int Mpad, int Kpad, __nv_bfloat16 *limbs, int32_t *Dh,
                                    int32_t *Dl) {
    const long long total = (long long)M * n;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx / n), v = (int)(idx - (long long)j * n);
        const long long x = fixed_entry(basis, b, n, nf, fam0, j, v);
        const long long h = (x + (1ll << 23)) >> 24;
        Dh[idx] = (int32_t)h;
        Dl[idx] = (int32_t)(x - h * (1ll << 24));
        long long r = x;
#pragma unroll
        for (int s = kLimbs - 1; s >= 1; --s) {
            const long long dg = ((r + 32) & 63) - 32;          // balanced digit in [-32, 31]
            limbs[((size_t)s * Mpad + j) * Kpad + v] = __float2bfloat16_rn((float)dg);
            r = (r - dg) >> kDigitBits;
        }
        limbs[(size_t)j * Kpad + v] = __float2bfloat16_rn((float)r);   // top digit, |r| <= 32
    }
}

// One warp per atom: S_j = sum_v D_fix[j][v], split canonically.
__global__ void fixed_sums_kernel(int b, int n, int M, int nf, int fam0, const double *basis,
                                  long long *Sh, long long *Sl) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < M; j += warps) {
        long long s = 0;
        for (int v = lane; v < n; v += 32) s += fixed_entry(basis, b, n, nf, fam0, j, v);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            const long long h = (s + (1ll << 23)) >> 24;
            Sh[j] = h;
            Sl[j] = s - h * (1ll << 24);
        }
    }
}

__global__ void basis_to_float_kernel(const double *basis, float *out, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = (float)basis[i];
}

// Host entry used by the library: fam0 = family of a single-family
// dictionary (0 = DCT, 1 = Haar); ignored when nf == 2.
cudaError_t build_fixed_tables_fam(DictDev &d, const double *basis_dev, int fam0, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d.limbs, 0, sizeof(__nv_bfloat16) * (size_t)kLimbs * d.Mpad * d.Kpad, st);
    if (e != cudaSuccess) return e;
    const long long total = (long long)d.M * d.n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    fixed_tables_kernel<<<blocks, 256, 0, st>>>(d.b, d.n, d.M, d.nf, fam0, basis_dev, d.Mpad, d.Kpad,
                                                d.limbs, d.Dh, d.Dl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int sblocks = (d.M + 7) / 8;
    if (sblocks > 4096) sblocks = 4096;
    fixed_sums_kernel<<<sblocks, 256, 0, st>>>(d.b, d.n, d.M, d.nf, fam0, basis_dev, d.Sh, d.Sl);
    return cudaGetLastError();
}

// bf16(D[j][v]) rounded to nearest from the FP64 entry, zero padding to
// [Mpad][Kpad], and one warp per atom for the row sum of the BF16 values
// (summed in FP64, rounded once to FP32).
__global__ void bf16_table_kernel(int b, int n, int M, int nf, int fam0, const double *basis, int Mpad, int Kpad,
                                  __nv_bfloat16 *Dbf) {
    const long long total = (long long)Mpad * Kpad;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx / Kpad), v = (int)(idx - (long long)j * Kpad);
        double d = 0.0;
        if (j < M && v < n) {
            const int fam = nf == 2 ? j / n : fam0;
            const int f = j - (nf == 2 ? (j / n) * n : 0);
            const int p = f % b, q = f / b, m = v / b, i = v - m * b;
            const double *B = basis + (size_t)fam * b * b;
            d = B[p * b + i] * B[q * b + m];
        }
        Dbf[idx] = __double2bfloat16(d);
    }
}

__global__ void bf16_sums_kernel(int n, int M, int Kpad, const __nv_bfloat16 *Dbf, float *Sbf) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < M; j += warps) {
        double s = 0.0;
        for (int v = lane; v < n; v += 32) s += (double)__bfloat162float(Dbf[(size_t)j * Kpad + v]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) Sbf[j] = (float)s;
    }
}

cudaError_t build_bf16_tables(DictDev &d, const double *basis_dev, int fam0, cudaStream_t st) {
    const long long total = (long long)d.Mpad * d.Kpad;
    int blocks = (int)std::min<long long>((total + 255) / 256, 8192);
    bf16_table_kernel<<<blocks, 256, 0, st>>>(d.b, d.n, d.M, d.nf, fam0, basis_dev, d.Mpad, d.Kpad, d.Dbf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int sblocks = std::min((d.M + 7) / 8, 4096);
    bf16_sums_kernel<<<sblocks, 256, 0, st>>>(d.n, d.M, d.Kpad, d.Dbf, d.Sbf);
    return cudaGetLastError();
}

// FP8 form: one warp per atom finds max_v |D[j][v]|, picks the power of two
// s_j with max |D| s_j <= 448 (the largest finite E4M3 value), writes
// e4m3(D[j][v] s_j) (round to nearest, saturating) with zero padding to K8,
// and the row sum of the dequantised values (FP64, rounded once to FP32).
__global__ void fp8_table_kernel(int b, int n, int M, int nf, int fam0, const double *basis, int K8, uint8_t *D8,
                                 float *inv_s, float *S8) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < M; j += warps) {
        const int fam = nf == 2 ? j / n : fam0;
        const int f = j - (nf == 2 ? (j / n) * n : 0);
        const int p = f % b, q = f / b;
        const double *B = basis + (size_t)fam * b * b;
        double mx = 0.0;
        for (int v = lane; v < n; v += 32) mx = fmax(mx, fabs(B[p * b + v % b] * B[q * b + v / b]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        int ex = 0;
        if (mx > 0.0) ex = (int)floor(log2(448.0 / mx));
        const double s = ldexp(1.0, ex);
        double sum = 0.0;
        for (int v = lane; v < K8; v += 32) {
            __nv_fp8_storage_t q8 = 0;
            if (v < n) {
                const double d = B[p * b + v % b] * B[q * b + v / b];
                q8 = __nv_cvt_float_to_fp8((float)(d * s), __NV_SATFINITE, __NV_E4M3);
                __half_raw hr = __nv_cvt_fp8_to_halfraw(q8, __NV_E4M3);
                sum += (double)__half2float(__half(hr)) / s;
            }
            D8[(size_t)j * K8 + v] = q8;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0) {
            inv_s[j] = (float)(1.0 / s);
            S8[j] = (float)sum;
        }
    }
}

cudaError_t build_fp8_tables(DictDev &d, const double *basis_dev, int fam0, cudaStream_t st) {
    const int K8 = kpad_fp8(d.n);
    cudaError_t e = cudaMemsetAsync(d.D8, 0, (size_t)d.Mpad * K8, st);
    if (e != cudaSuccess) return e;
    const int blocks = std::min((d.M + 7) / 8, 8192);
    fp8_table_kernel<<<blocks, 256, 0, st>>>(d.b, d.n, d.M, d.nf, fam0, basis_dev, K8, d.D8, d.inv_s8, d.S8);
    return cudaGetLastError();
}

cudaError_t launch_basis_to_float(const double *basis_dev, float *out, int count, cudaStream_t st) {
    basis_to_float_kernel<<<(count + 255) / 256, 256, 0, st>>>(basis_dev, out, count);
    return cudaGetLastError();
}

}  // namespace aqmp
