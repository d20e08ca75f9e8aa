// diff.cu -- refinement of the coefficients on a fixed MP support: sparse
// synthesis (Algorithm 3) with caller coefficients and its adjoint, and the
// mean SSIM of Section 3 with its gradient with respect to the
// reconstruction, all on the device.
//
// Synthesis: recon[y+i][x+m] = sum_t alpha_t B[p_t][i] B[q_t][m] per leaf.
// Adjoint: d recon / d alpha_t is the atom itself, so
// grad alpha_t = <G_leaf, phi_t> = (B G B^T)[p_t][q_t] for the leaf's block G
// of the incoming gradient; the block transform is computed once per leaf
// and family (two b x b products) and gathered at the leaf's atoms.
//
// SSIM over the valid region with an 11 x 11 Gaussian window w = g g^T
// (sigma 1.5), K1 = 0.01, K2 = 0.03, L = 255.  Per window:
//   A1 = 2 mx my + C1, A2 = 2 (Exy - mx my) + C2,
//   B1 = mx^2 + my^2 + C1, B2 = (Exx - mx^2) + (Eyy - my^2) + C2,
//   f = A1 A2 / (B1 B2).
// With S = mean f over the N windows, for a pixel k of y:
//   dS/dy[k] = (1/N) sum_win w(k - win) (f_my + 2 y[k] f_Eyy + x[k] f_Exy),
//   f_my = f (2 mx / A1 - 2 mx / A2 - 2 my / B1 + 2 my / B2),
//   f_Exy = 2 f / A2,   f_Eyy = -f / B2,
// i.e. the per-window partials filtered back with the (symmetric, separable)
// window.  The window statistics and the back-filtered partials are
// accumulated in double-float; the per-window formula runs in FP64.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

namespace {

__constant__ double c_gauss[11];

__device__ __forceinline__ int ilog2_dev(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// One CTA per leaf: T_fam = B G B^T for the families present, then gather.
__global__ void synth_backward_kernel(const LeafRec *leaves, unsigned long long n_leaves, const AtomRec *atoms,
                                      uint32_t plane, const float *grad, long long pitch, float *grad_alpha,
                                      DecodeArgs bases) {
    extern __shared__ float sm[];
    for (unsigned long long li = blockIdx.x; li < n_leaves; li += gridDim.x) {
        const LeafRec L = leaves[li];
        if (L.plane != plane || L.n_atoms == 0) continue;
        const int b = L.b, n = b * b;
        const float *basis = bases.basis[ilog2_dev(b)];
        const int nfam = bases.nf;
        float *G = sm;               // b x b gradient block, G[i][m]
        float *U = G + n;            // B G (per family), U[p][m]
        float *Tc = U + n;           // one family's coefficients Tc[p][q]
        __syncthreads();
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const int i = v / b, m = v - i * b;
            G[v] = grad[(long long)(L.y + i) * pitch + L.x + m];
        }
        __syncthreads();
        for (int fam = 0; fam < nfam; ++fam) {
            const float *B = basis + (nfam == 1 ? bases.single_family : fam) * b * b;
            for (int v = threadIdx.x; v < n; v += blockDim.x) {          // U = B G
                const int p = v / b, m = v - p * b;
                float s = 0.0f;
                for (int i = 0; i < b; ++i) s = __fmaf_rn(B[p * b + i], G[i * b + m], s);
                U[v] = s;
            }
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x) {          // T = U B^T
                const int p = v / b, q = v - p * b;
                float s = 0.0f;
                for (int m = 0; m < b; ++m) s = __fmaf_rn(U[p * b + m], B[q * b + m], s);
                Tc[v] = s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < L.n_atoms; t += blockDim.x) {    // this family's atoms
                const uint32_t j = atoms[L.atom_off + t].j;
                const int fa = nfam == 2 ? (int)(j >= (uint32_t)n) : 0;
                if (fa != fam) continue;
                const int f = (int)j - (nfam == 2 ? fa * n : 0);
                grad_alpha[L.atom_off + t] = Tc[(f % b) * b + (f / b)];
            }
            __syncthreads();
        }
    }
}

// The 11-tap passes run in double-float on the FP32 pipes (GB300's FP64
// rate is a small fraction of its FP32 rate): each tap adds g v with the
// weight g as a (hi, lo) pair and v a pixel, an exact pixel product, or a
// stored pair, so the window sums keep ~2^-46 relative accuracy and
// E[x^2] - mu^2 is formed in FP64 from them without losing the variance.
// Intermediate planes hold (hi, lo) float pairs in the 8-byte slots.
__constant__ float2 c_gauss_df[11];

__device__ __forceinline__ df gw(int j) {
    const float2 g = c_gauss_df[j];
    return df{-g.x, -g.y};                          // negated: s - (-g) v = s + g v
}

__device__ __forceinline__ df df_of(double d) {
    const float hi = (float)d;
    return df{hi, (float)(d - (double)hi)};
}

// Horizontal 11-tap pass of the five products (x, y, x^2, y^2, x y) over the
// valid columns: H[k][row][a] for a < w - 10.
__global__ void ssim_hpass_kernel(const float *x, const float *y, int h, int w, long long pitch, float2 *H) {
    const int wo = w - 10;
    const long long plane = (long long)h * wo;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < plane;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / wo), a = (int)(idx - (long long)r * wo);
        df sx{0.0f, 0.0f}, sy = sx, sxx = sx, syy = sx, sxy = sx;
#pragma unroll
        for (int j = 0; j < 11; ++j) {
            const df g = gw(j);
            const float xv = x[(long long)r * pitch + a + j], yv = y[(long long)r * pitch + a + j];
            sx = df_sub_mul(sx, g, df{xv, 0.0f});
            sy = df_sub_mul(sy, g, df{yv, 0.0f});
            sxx = df_sub_mul(sxx, g, df_two_prod(xv, xv));
            syy = df_sub_mul(syy, g, df_two_prod(yv, yv));
            sxy = df_sub_mul(sxy, g, df_two_prod(xv, yv));
        }
        H[idx] = make_float2(sx.hi, sx.lo);
        H[plane + idx] = make_float2(sy.hi, sy.lo);
        H[2 * plane + idx] = make_float2(sxx.hi, sxx.lo);
        H[3 * plane + idx] = make_float2(syy.hi, syy.lo);
        H[4 * plane + idx] = make_float2(sxy.hi, sxy.lo);
    }
}

// Vertical pass, SSIM per window, its partials (scaled) and the mean.  The
// window formula runs in FP64 from the double-float sums, with one division.
__global__ void ssim_window_kernel(const float2 *H, int h, int w, double *P, double *sum, double gscale) {
    const int wo = w - 10, ho = h - 10;
    const long long hplane = (long long)h * wo, wins = (long long)ho * wo;
    const double C1 = (0.01 * 255.0) * (0.01 * 255.0), C2 = (0.03 * 255.0) * (0.03 * 255.0);
    double local = 0.0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < wins;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / wo), a = (int)(idx - (long long)r * wo);
        df m[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k] = df{0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 11; ++i) {
            const df g = gw(i);
            const long long o = (long long)(r + i) * wo + a;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float2 v = H[k * hplane + o];
                m[k] = df_sub_mul(m[k], g, df{v.x, v.y});
            }
        }
        const double mx = df_to_double(m[0]), my = df_to_double(m[1]);
        const double exx = df_to_double(m[2]), eyy = df_to_double(m[3]), exy = df_to_double(m[4]);
        const double A1 = 2 * mx * my + C1, A2 = 2 * (exy - mx * my) + C2;
        const double B1 = mx * mx + my * my + C1, B2 = (exx - mx * mx) + (eyy - my * my) + C2;
        const double A12 = A1 * A2, B12 = B1 * B2;
        const double r1 = 1.0 / (A12 * B12);                 // 1 / (A1 A2 B1 B2)
        const double f = A12 * A12 * r1;                      // A1 A2 / (B1 B2)
        local += f;
        if (P) {
            const double iA1 = A2 * B12 * r1, iA2 = A1 * B12 * r1, iB1 = A12 * B2 * r1, iB2 = A12 * B1 * r1;
            P[idx] = gscale * f * (2 * mx * iA1 - 2 * mx * iA2 - 2 * my * iB1 + 2 * my * iB2);   // f_my
            P[wins + idx] = gscale * (-f * iB2);                                              // f_Eyy
            P[2 * wins + idx] = gscale * (2 * f * iA2);                                       // f_Exy
        }
    }
    // block sum, one atomic per block
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) atomicAdd(sum, v / (double)wins);
    }
}

// Back through the vertical pass: V[k][row][a] = sum_i g[i] P[k][row - i][a]
// over the windows whose first row is row - i (full height, valid columns).
__global__ void ssim_vback_kernel(const double *P, int h, int w, float2 *V) {
    const int wo = w - 10, ho = h - 10;
    const long long wins = (long long)ho * wo, vplane = (long long)h * wo;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < vplane;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / wo), a = (int)(idx - (long long)r * wo);
        df s0{0.0f, 0.0f}, s1 = s0, s2 = s0;
#pragma unroll
        for (int i = 0; i < 11; ++i) {
            const int wr = r - i;
            if (wr < 0 || wr >= ho) continue;
            const df g = gw(i);
            const long long o = (long long)wr * wo + a;
            s0 = df_sub_mul(s0, g, df_of(P[o]));
            s1 = df_sub_mul(s1, g, df_of(P[wins + o]));
            s2 = df_sub_mul(s2, g, df_of(P[2 * wins + o]));
        }
        V[idx] = make_float2(s0.hi, s0.lo);
        V[vplane + idx] = make_float2(s1.hi, s1.lo);
        V[2 * vplane + idx] = make_float2(s2.hi, s2.lo);
    }
}

// Back through the horizontal pass and the products:
// grad_y[r][c] = G1 + 2 y G2 + x G3 with G_k[r][c] = sum_j g[j] V[k][r][c - j].
__global__ void ssim_hback_kernel(const float2 *V, const float *x, const float *y, int h, int w, long long pitch,
                                  float *grad) {
    const int wo = w - 10;
    const long long vplane = (long long)h * wo, npix = (long long)h * w;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < npix;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / w), c = (int)(idx - (long long)r * w);
        df g1{0.0f, 0.0f}, g2 = g1, g3 = g1;
#pragma unroll
        for (int j = 0; j < 11; ++j) {
            const int a = c - j;
            if (a < 0 || a >= wo) continue;
            const df g = gw(j);
            const long long o = (long long)r * wo + a;
            const float2 v1 = V[o], v2 = V[vplane + o], v3 = V[2 * vplane + o];
            g1 = df_sub_mul(g1, g, df{v1.x, v1.y});
            g2 = df_sub_mul(g2, g, df{v2.x, v2.y});
            g3 = df_sub_mul(g3, g, df{v3.x, v3.y});
        }
        const float xv = x[(long long)r * pitch + c], yv = y[(long long)r * pitch + c];
        // g1 + 2 y g2 + x g3
        df t = df_sub_mul(g1, df{-2.0f * yv, 0.0f}, g2);
        t = df_sub_mul(t, df{-xv, 0.0f}, g3);
        grad[(long long)r * pitch + c] = __fadd_rn(t.hi, t.lo);
    }
}

}  // namespace

cudaError_t upload_gauss11(cudaStream_t st) {
    double g[11], s = 0.0;
    for (int i = 0; i < 11; ++i) {
        const double r = i - 5.0;
        g[i] = exp(-(r * r) / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    for (int i = 0; i < 11; ++i) g[i] /= s;
    float2 gf[11];
    for (int i = 0; i < 11; ++i) {
        gf[i].x = (float)g[i];
        gf[i].y = (float)(g[i] - (double)gf[i].x);
    }
    cudaError_t e = cudaMemcpyToSymbolAsync(c_gauss, g, sizeof g, 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_gauss_df, gf, sizeof gf, 0, cudaMemcpyHostToDevice, st);
}

cudaError_t launch_synth_forward(const LeafRec *leaves, unsigned long long n_leaves, const AtomRec *atoms,
                                 const float *alpha, uint32_t plane, float *out, long long pitch,
                                 const DecodeArgs &bases, int num_sms, cudaStream_t st) {
    // the decoder with caller coefficients (decode.cu)
    DecodeArgs a = bases;
    a.leaves = leaves;
    a.n_leaves = n_leaves;
    a.atoms = atoms;
    a.plane = plane;
    a.out = out;
    a.out_pitch = pitch;
    return launch_decode_alpha(a, alpha, num_sms, st);
}

cudaError_t launch_synth_backward(const LeafRec *leaves, unsigned long long n_leaves, const AtomRec *atoms,
                                  uint32_t plane, const float *grad, long long pitch, float *grad_alpha,
                                  const DecodeArgs &bases, int max_side, int num_sms, cudaStream_t st) {
    if (n_leaves == 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)max_side * max_side * 3;   // G, U, Tc
    cudaError_t e = cudaFuncSetAttribute(synth_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    long long blocks = (long long)n_leaves;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    synth_backward_kernel<<<(unsigned)blocks, 256, smem, st>>>(leaves, n_leaves, atoms, plane, grad, pitch,
                                                                grad_alpha, bases);
    return cudaGetLastError();
}

cudaError_t launch_ssim(const float *x, const float *y, int h, int w, long long pitch, double *H, double *P,
                        double *V, double *sum, float *grad, double gscale, int num_sms, cudaStream_t st) {
    const unsigned grid = (unsigned)num_sms * 8;
    float2 *Hf = reinterpret_cast<float2 *>(H), *Vf = reinterpret_cast<float2 *>(V);   // (hi, lo) in 8-byte slots
    ssim_hpass_kernel<<<grid, 256, 0, st>>>(x, y, h, w, pitch, Hf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long wins = (long long)(h - 10) * (w - 10);
    const double scale = grad ? gscale / (double)wins : 0.0;
    ssim_window_kernel<<<grid, 256, 0, st>>>(Hf, h, w, grad ? P : nullptr, sum, scale);
    if ((e = cudaGetLastError()) != cudaSuccess || !grad) return e;
    ssim_vback_kernel<<<grid, 256, 0, st>>>(P, h, w, Vf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ssim_hback_kernel<<<grid, 256, 0, st>>>(Vf, x, y, h, w, pitch, grad);
    return cudaGetLastError();
}

}  // namespace aqmp
