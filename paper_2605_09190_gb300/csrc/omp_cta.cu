// omp_cta.cu -- Orthogonal Matching Pursuit per leaf (the solver the paper's
// authors ran, Section 2.2) at sides 32 and 64, with the quadtree split /
// emit of Algorithm 2.  The rules are those of omp.cu (sides 4..16): the
// residual energy ||y||^2 - x_S . c0_S tested before each step (Eq. (3),
// strict, with the MP kernel's equality band), the residual correlations
// c = c0 - G[:, S] x_S, argmax |c| with ties within 2^-32 ||y|| going to the
// lowest index, a new row of the Cholesky factor L of G_SS per selection
// (a pivot <= 2^-40 ends the pursuit), then the re-fit L L^T x_S = c0_S.
// Everything is FP64.
//
// One CTA of 256 threads owns one leaf; atom j = tid + 256 s is slot s of
// thread tid, so a thread's atoms of one family share p = tid mod b and step
// q by 256 / b.  The Gram matrix is the identity inside a family and
// kron(W, W) across (W = C H^T), so the cross-family part of G[:, S] x_S is
// W X_H W^T for the DCT atoms and W^T X_C W for the Haar atoms (X_F the
// family's coefficients as a b x b matrix).  While the other family's
// support is small each support atom is applied directly (one W factor per
// thread, one multiply-add per slot); past the crossover the two b x b x b
// products are formed through a shared b x b intermediate.
//
// The factor L (packed rows, up to k(k+1)/2 doubles) lives in a global slot
// per CTA.  Both triangular solves run in blocks of 32 rows: the part against
// the rows already solved is a matrix-vector product with coalesced reads of
// row segments (all warps), the 32 x 32 diagonal block one warp's chain of
// shuffles.  z = L^-1 c0_S grows by one entry per step; x_S = L^-T z is
// solved afresh.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

namespace {

constexpr double kTieRel = 0x1p-32;
constexpr double kBandRel = 0x1p-37;
constexpr double kPivotMin = 0x1p-40;
constexpr uint32_t kNoAtom = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxBudget = 1024;

__host__ __device__ __forceinline__ long long tri64(long long i) { return i * (i + 1) / 2; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Block-wide reductions: every thread returns the same value (the warps'
// partials are combined in warp order by every thread).
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w];
    return s;
}

__device__ __forceinline__ double block_max(double v, double *red) {
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = red[0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) m = fmax(m, red[w]);
    return m;
}

__device__ __forceinline__ uint32_t block_min_u32(uint32_t v, uint32_t *red) {
    v = __reduce_min_sync(0xffffffffu, v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t m = red[0];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) m = min(m, red[w]);
    return m;
}

// <phi_a, phi_b> from W (b x b, FP64): 1 on the diagonal, 0 elsewhere inside
// a family, W[p_d][p_h] W[q_d][q_h] between DCT atom d and Haar atom h (atom
// (p, q) has in-family index q b + p).
template <int B, int NF>
__device__ __forceinline__ double gram(const double *sW, uint32_t a, uint32_t b) {
    constexpr uint32_t n = B * B;
    const bool fa = a >= n, fb = b >= n;
    if (NF == 1 || fa == fb) return a == b ? 1.0 : 0.0;
    const uint32_t d = fa ? b : a, h = fa ? a - n : b - n;
    return sW[(d % B) * B + (h % B)] * sW[(d / B) * B + (h / B)];
}

// Shared-memory layout (doubles, then the support's atom indices).
template <int B, int NF>
struct OmpLayout {
    static constexpr int n = B * B;
    static constexpr int M = NF * n;
    static constexpr int E = M / kThreads;       // slots per thread
    static constexpr int EF = n / kThreads;      // slots per thread and family
    static constexpr int QS = kThreads / B;      // q step between a thread's slots
    static constexpr int W2 = NF == 2 ? 3 * B * B : 0;   // W, W^T, the b x b intermediate
    __host__ __device__ static constexpr size_t doubles(int k) { return (size_t)W2 + M + 32 * kWarps + 5 * (size_t)k; }
    __host__ __device__ static constexpr size_t bytes(int k) { return 8 * doubles(k) + 4 * (size_t)k + 64; }
    static_assert(n % kThreads == 0 && kThreads % B == 0, "layout needs 256 | b^2 and b | 256");
};

}  // namespace

template <int B, int NF>
__global__ void __launch_bounds__(kThreads, 1) omp_cta_kernel(MPArgs a) {
    using Ly = OmpLayout<B, NF>;
    constexpr int n = Ly::n, M = Ly::M, E = Ly::E, EF = Ly::EF, QS = Ly::QS;
    // direct application costs (1 + EF) per support atom and thread, the
    // separable one 2 EF B per direction
    constexpr int kCross = 2 * EF * B / (1 + EF);

    extern __shared__ __align__(16) unsigned char smem[];
    double *sW = reinterpret_cast<double *>(smem);     // W[pc][ph]
    double *sWT = sW + (NF == 2 ? B * B : 0);          // W^T[ph][pc]
    double *UV = sWT + (NF == 2 ? B * B : 0);          // b x b intermediate
    double *xd = reinterpret_cast<double *>(smem) + Ly::W2;   // x_S scattered over all M atoms
    double *red = xd + M;                              // 32 x warps reduction scratch
    const int k = a.lv.k;
    double *xs = red + 32 * kWarps;
    double *c0s = xs + k;
    double *zs = c0s + k;
    double *rdiag = zs + k;
    double *wv = rdiag + k;
    uint32_t *Sj = reinterpret_cast<uint32_t *>(wv + k);
    uint32_t *bc = Sj + k;                             // broadcast words

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (NF == 2)
        for (int i = tid; i < B * B; i += kThreads) {
            const double w = (double)a.W[i].x + (double)a.W[i].y;
            sW[i] = w;
            sWT[(i % B) * B + i / B] = w;
        }
    __syncthreads();

    const LevelArgs &lv = a.lv;
    const unsigned count = *lv.count;
    unsigned *work = &a.ctr->work_next[lv.level];
    double *Lslot = a.omp_L + (size_t)blockIdx.x * (size_t)tri64(k);
    const int p_own = tid % B, q_base = tid / B;

    for (;;) {
        if (tid == 0) bc[0] = atomicAdd(work, 1u);
        __syncthreads();
        const unsigned leaf = bc[0];
        __syncthreads();
        if (leaf >= count) break;

        const QueueEntry qe = lv.queue[leaf];
        const double tol = (double)a.planes[qe.plane].tol;
        const double eps2 = tol * tol * (double)n;
        const double E0 = (double)a.e0[leaf];
        const double Sy = sqrt(E0);
        const double tie_c = kTieRel * Sy, band_c = kBandRel * Sy;
        const double thr_e = eps2 - kTieRel * E0, band_e = kBandRel * E0;

        double c0r[E];
        const float2 *cp = a.c0 + (size_t)leaf * M;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const float2 v = cp[tid + kThreads * s];
            c0r[s] = (double)v.x + (double)v.y;
        }
        for (int i = tid; i < M; i += kThreads) xd[i] = 0.0;
        __syncthreads();
        int nS = 0, nC = 0, nH = 0;          // support size, and per family
        bool conv = false, tie = false;
        for (;;) {
            // (a6) accuracy test before every step, strict
            double acc = 0.0;
            for (int i = tid; i < nS; i += kThreads) acc += xs[i] * c0s[i];
            const double En = E0 - block_sum(acc, red);
            if (fabs(En - thr_e) < band_e) tie = true;
            if (En < thr_e) { conv = true; break; }
            if (nS == k) break;

            // residual correlations c = c0 - x (own family) - cross terms
            double cv[E];
#pragma unroll
            for (int s = 0; s < E; ++s) cv[s] = c0r[s] - xd[tid + kThreads * s];
            if (NF == 2) {
                const bool sepH = nC > kCross, sepC = nH > kCross;   // uniform
                if (!sepH || !sepC) {
                    for (int i = 0; i < nS; ++i) {
                        const uint32_t sa = Sj[i];
                        const double x = xs[i];
                        if (sa < (uint32_t)n) {
                            if (sepH) continue;
                            // DCT (ps, qs) -> Haar (p_own, q): W[ps][p_own] W[qs][q]
                            const uint32_t ps = sa % B, qs = sa / B;
                            const double ax = x * sW[ps * B + p_own];
#pragma unroll
                            for (int s = 0; s < EF; ++s) cv[EF + s] -= ax * sW[qs * B + q_base + QS * s];
                        } else {
                            if (sepC) continue;
                            // Haar (ps, qs) -> DCT (p_own, q): W[p_own][ps] W[q][qs]
                            const uint32_t ps = (sa - n) % B, qs = (sa - n) / B;
                            const double ax = x * sWT[ps * B + p_own];
#pragma unroll
                            for (int s = 0; s < EF; ++s) cv[s] -= ax * sW[(q_base + QS * s) * B + qs];
                        }
                    }
                }
                if (sepC) {
                    // DCT (p, q) -= (W X_H W^T)[p][q]: U[a][q] = sum_b X_H[a][b] W[q][b]
                    for (int e = tid; e < B * B; e += kThreads) {
                        const int aa = e / B, q = e % B;
                        double u = 0.0;
#pragma unroll 8
                        for (int bb = 0; bb < B; ++bb) u += xd[n + bb * B + aa] * sWT[bb * B + q];
                        UV[aa * B + q] = u;
                    }
                    __syncthreads();
#pragma unroll
                    for (int s = 0; s < EF; ++s) {
                        const int q = q_base + QS * s;
                        double t = 0.0;
#pragma unroll 8
                        for (int aa = 0; aa < B; ++aa) t += sWT[aa * B + p_own] * UV[aa * B + q];
                        cv[s] -= t;
                    }
                    __syncthreads();
                }
                if (sepH) {
                    // Haar (p, q) -= (W^T X_C W)[p][q]: V[pc][q] = sum_qc X_C[pc][qc] W[qc][q]
                    for (int e = tid; e < B * B; e += kThreads) {
                        const int pc = e / B, q = e % B;
                        double v = 0.0;
#pragma unroll 8
                        for (int qc = 0; qc < B; ++qc) v += xd[qc * B + pc] * sW[qc * B + q];
                        UV[pc * B + q] = v;
                    }
                    __syncthreads();
#pragma unroll
                    for (int s = 0; s < EF; ++s) {
                        const int q = q_base + QS * s;
                        double t = 0.0;
#pragma unroll 8
                        for (int pc = 0; pc < B; ++pc) t += sW[pc * B + p_own] * UV[pc * B + q];
                        cv[EF + s] -= t;
                    }
                    __syncthreads();
                }
            }
            double amax = 0.0;
#pragma unroll
            for (int s = 0; s < E; ++s) amax = fmax(amax, fabs(cv[s]));
            amax = block_max(amax, red);
            if (amax <= tie_c) break;                        // nothing left to remove
            const double edge = amax - tie_c;
            uint32_t jl = kNoAtom;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const uint32_t j = (uint32_t)(tid + kThreads * s);
                const double m = fabs(cv[s]);
                if (m >= edge && j < jl) jl = j;
                if (fabs(m - edge) < band_c) tie = true;
            }
            const uint32_t jb = block_min_u32(jl, reinterpret_cast<uint32_t *>(red));
            if ((jb % kThreads) == (uint32_t)tid) {
                double c0b = 0.0;
#pragma unroll
                for (int s = 0; s < E; ++s)
                    if ((uint32_t)s == jb / kThreads) c0b = c0r[s];
                red[32 * kWarps - 1] = c0b;
            }
            for (int i = tid; i < nS; i += kThreads) wv[i] = gram<B, NF>(sW, Sj[i], jb);
            __syncthreads();
            const double c0b = red[32 * kWarps - 1];

            // new Cholesky row: L w = G[S, jb], blocks of 32 rows
            for (int kb = 0; kb < nS; kb += 32) {
                const int ke = min(kb + 32, nS);
                if (kb > 0) {
                    // rows [kb, ke) against the solved w[0, kb)
                    for (int r = warp; r < ke - kb; r += kWarps) {
                        const double *Li = Lslot + tri64(kb + r);
                        double s = 0.0;
                        for (int c = lane; c < kb; c += 32) s += Li[c] * wv[c];
                        s = warp_sum(s);
                        if (lane == 0) wv[kb + r] -= s;
                    }
                    __syncthreads();
                }
                if (warp == 0) {
                    const int row = kb + lane;
                    double g = row < ke ? wv[row] : 0.0;
                    for (int c = kb; c < ke; ++c) {
                        double wc = lane == c - kb ? g * rdiag[c] : 0.0;
                        wc = __shfl_sync(0xffffffffu, wc, c - kb);
                        if (lane == c - kb) g = wc;
                        if (row > c && row < ke) g -= Lslot[tri64(row) + c] * wc;
                    }
                    if (row < ke) wv[row] = g;
                }
                __syncthreads();
            }
            double ww = 0.0;
            for (int i = tid; i < nS; i += kThreads) ww += wv[i] * wv[i];
            const double d = 1.0 - block_sum(ww, red);
            if (d > kPivotMin * 0x1p-4 && d < kPivotMin * 0x1p4) tie = true;
            if (d <= kPivotMin) break;                       // dependent on the support
            // append row nS; z grows by z_nS = (c0_jb - w . z) / L_nS,nS
            const double ld = sqrt(d), rd = 1.0 / ld;
            double wz = 0.0;
            for (int i = tid; i < nS; i += kThreads) {
                Lslot[tri64(nS) + i] = wv[i];
                wz += wv[i] * zs[i];
            }
            wz = block_sum(wz, red);
            if (tid == 0) {
                Lslot[tri64(nS) + nS] = ld;
                rdiag[nS] = rd;
                Sj[nS] = jb;
                c0s[nS] = c0b;
                zs[nS] = (c0b - wz) * rd;
            }
            if (jb < (uint32_t)n) ++nC; else ++nH;
            ++nS;
            __syncthreads();

            // re-fit: L^T x = z, blocks of 32 rows from the bottom
            for (int kb = ((nS - 1) / 32) * 32; kb >= 0; kb -= 32) {
                const int ke = min(kb + 32, nS);
                const int col = kb + lane;
                double s = 0.0;
                if (col < ke)
                    for (int r = ke + warp; r < nS; r += kWarps) s += Lslot[tri64(r) + col] * xs[r];
                red[warp * 32 + lane] = s;
                __syncthreads();
                if (warp == 0) {
                    double part = 0.0;
#pragma unroll
                    for (int w = 0; w < kWarps; ++w) part += red[w * 32 + lane];
                    double zp = col < ke ? zs[col] - part : 0.0;
                    for (int i = ke - 1; i >= kb; --i) {
                        double xi = lane == i - kb ? zp * rdiag[i] : 0.0;
                        xi = __shfl_sync(0xffffffffu, xi, i - kb);
                        if (lane == i - kb) zp = xi;
                        if (col < i) zp -= Lslot[tri64(i) + col] * xi;
                    }
                    if (col < ke) {
                        xs[col] = zp;
                        xd[Sj[col]] = zp;
                    }
                }
                __syncthreads();
            }
        }

        // (a7) emit or split, as the MP kernel
        const bool tie_any = __syncthreads_or(tie) != 0;
        if (tid == 0) {
            atomicAdd(&a.ctr->attempts[lv.level], 1ull);
            atomicAdd(&a.ctr->iterations[lv.level], (unsigned long long)nS);
            atomicMax(&a.ctr->max_steps[lv.level], (unsigned)nS);
        }
        const bool emit = conv || lv.is_last;
        if (emit) {
            if (tid == 0) {
                uint32_t off = kNoAtom, eslot = 0;
                const unsigned long long slot = atomicAdd(&a.ctr->n_leaves, 1ull);
                const unsigned long long o = atomicAdd(&a.ctr->n_atoms, (unsigned long long)nS);
                const uint8_t flags = (uint8_t)((tie_any ? 1u : 0u) | (qe.flags & 2u));
                if (slot >= a.leaf_cap || o + nS > a.atom_cap) {
                    raise_error(a.ctr, kDevErrQueueOverflow, 3u);
                } else {
                    LeafRec rec;
                    rec.plane = qe.plane;
                    rec.y = qe.y;
                    rec.x = qe.x;
                    rec.atom_off = (uint32_t)o;
                    rec.b = (uint16_t)B;
                    rec.n_atoms = (uint16_t)nS;
                    rec.converged = conv ? 1 : 0;
                    rec.flags = flags;
                    rec.reserved = 0;
                    a.leaves[slot] = rec;
                    off = (uint32_t)o;
                    eslot = (uint32_t)slot;
                    const unsigned long long cell = cell_of(a.cells, a.planes[qe.plane], qe.y, qe.x);
                    if (cell != ~0ull) a.cells.cell[cell] = (uint32_t)slot + 1u;
                    if (flags) atomicAdd(&a.ctr->near_tie_leaves, 1ull);
                }
                bc[1] = off;
                bc[2] = eslot;
            }
            __syncthreads();
            const uint32_t off = bc[1], eslot = bc[2];
            if (off != kNoAtom) {
                for (int i = tid; i < nS; i += kThreads) {
                    const double x = xs[i];
                    const float hi = (float)x;
                    a.atoms[off + i] = AtomRec{Sj[i], hi};
                    a.alpha_lo[off + i] = (float)(x - (double)hi);
                    a.atom_leaf[off + i] = eslot;
                }
            }
        } else if (tid == 0) {
            const unsigned slot = atomicAdd(lv.next_count, 4u);
            if (slot + 4u > lv.next_capacity) {
                raise_error(a.ctr, kDevErrQueueOverflow, 4u);
            } else {
                const uint32_t h = B / 2;
                const uint32_t fl = (qe.flags & 2u) | (tie_any ? 2u : 0u);
                lv.next_queue[slot + 0] = QueueEntry{qe.plane, qe.y, qe.x, fl};
                lv.next_queue[slot + 1] = QueueEntry{qe.plane, qe.y, qe.x + h, fl};
                lv.next_queue[slot + 2] = QueueEntry{qe.plane, qe.y + h, qe.x, fl};
                lv.next_queue[slot + 3] = QueueEntry{qe.plane, qe.y + h, qe.x + h, fl};
            }
        }
        __syncthreads();
    }
}

template <int B, int NF>
static cudaError_t launch_omp_cta_t(const MPArgs &a, cudaStream_t st) {
    const int k = a.lv.k;
    if (k < 1 || k > kMaxBudget || !a.omp_L || a.omp_slots < 1 ||
        a.omp_L_doubles < (unsigned long long)a.omp_slots * (unsigned long long)tri64(k))
        return cudaErrorInvalidValue;
    const size_t bytes = OmpLayout<B, NF>::bytes(k);
    auto kern = omp_cta_kernel<B, NF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    long long grid = a.omp_slots;
    if ((long long)a.lv.capacity < grid) grid = a.lv.capacity;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

int omp_cta_max_budget() { return kMaxBudget; }

unsigned long long omp_cta_workspace_doubles(int k, int slots) {
    return k < 1 ? 0ull : (unsigned long long)slots * (unsigned long long)tri64(k);
}

cudaError_t launch_omp_cta(const MPArgs &a, int nf, cudaStream_t st) {
    if (nf == 2) {
        switch (a.lv.b) {
            case 32: return launch_omp_cta_t<32, 2>(a, st);
            case 64: return launch_omp_cta_t<64, 2>(a, st);
        }
    } else {
        switch (a.lv.b) {
            case 32: return launch_omp_cta_t<32, 1>(a, st);
            case 64: return launch_omp_cta_t<64, 1>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace aqmp
