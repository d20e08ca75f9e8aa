// omp.cu -- Orthogonal Matching Pursuit per leaf (the solver the paper's
// authors ran, Section 2.2), for sides 4..16, with the quadtree split / emit
// of Algorithm 2 (sides 32 and 64: omp_cta.cu, the same rules).
//
// One warp owns one leaf.  Each step:
//   - residual energy ||r||^2 = ||y||^2 - x_S . c0_S (the residual is
//     orthogonal to span(D_S) after every re-fit), tested before the step
//     with the rule of Eq. (3) and the same equality band as the MP kernel;
//   - residual correlations c = c0 - G[:, S] x_S, the Gram entries generated
//     from W = C H^T (G is the identity inside a family and kron(W, W)
//     across the two);
//   - argmax |c| with the MP kernel's tie rule (values within 2^-32 ||y|| of
//     the largest are tied, lowest index wins) and certification band;
//   - the new row of the Cholesky factor L of G_SS (solve L w = G[S, j],
//     pivot 1 - |w|^2; a pivot <= 2^-40 ends the pursuit, the atom being
//     dependent on the support), then the re-fit L L^T x_S = c0_S.
// Everything is FP64.  L lives packed in shared memory; row i of every
// triangular solve belongs to lane i mod 32 and the solves run in axpy form
// (the owner finishes its row, shuffles the value, every lane updates its
// rows), so each step of their chains is one shuffle, not a reduction.  A
// leaf's budget k must be <= 64 (two rows per lane).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

namespace {

constexpr double kTieRel = 0x1p-32;
constexpr double kBandRel = 0x1p-37;
constexpr double kPivotMin = 0x1p-40;
constexpr uint32_t kNoAtom = 0xffffffffu;

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

__host__ __device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

// <phi_a, phi_b>: 1 on the diagonal, 0 elsewhere inside a family, and
// W[p_d][p_h] W[q_d][q_h] between DCT atom d = (p_d, q_d) and Haar atom
// h = (p_h, q_h) (atom (p, q) has in-family index q b + p).
template <int B, int NF>
__device__ __forceinline__ double gram(const double *sW, uint32_t a, uint32_t b) {
    constexpr uint32_t n = B * B;
    const bool fa = a >= n, fb = b >= n;
    if (NF == 1 || fa == fb) return a == b ? 1.0 : 0.0;
    const uint32_t d = fa ? b : a, h = fa ? a - n : b - n;
    return sW[(d % B) * B + (h % B)] * sW[(d / B) * B + (h / B)];
}

}  // namespace

template <int B, int NF>
__global__ void __launch_bounds__(256, 1) omp_kernel(MPArgs a) {
    constexpr int n = B * B;
    constexpr int M = NF * n;
    constexpr int E = (M + 31) / 32;
    // SLOTS: with two families and n a multiple of 32, element (lane, s) is
    // atom lane + 32 s, DCT for s < E/2, and its in-family (p, q) is
    // (lane mod B, lane / B + (32 / B) s, less B for the Haar slots)
    constexpr bool SLOTS = NF == 2 && (n % 32) == 0;

    extern __shared__ __align__(16) unsigned char smem[];
    double *sW = reinterpret_cast<double *>(smem);
    const int k = a.lv.k;
    const int per = tri(k) + 3 * k + M;                  // L, x_S, c0_S, 1 / L_ii, dense x (doubles)
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *base = sW + (NF == 2 ? B * B : 0);
    double *L = base + (size_t)warp * per;
    double *xs = L + tri(k);
    double *c0s = xs + k;
    double *rdiag = c0s + k;
    double *xd = rdiag + k;                              // x_S scattered over all M atoms
    uint32_t *Sj = reinterpret_cast<uint32_t *>(base + (size_t)warps * per) + (size_t)warp * k;

    if (NF == 2)
        for (int i = threadIdx.x; i < B * B; i += blockDim.x) sW[i] = (double)a.W[i].x + (double)a.W[i].y;
    __syncthreads();

    const LevelArgs &lv = a.lv;
    const unsigned count = *lv.count;
    unsigned *work = &a.ctr->work_next[lv.level];
    const uint32_t p_own = (uint32_t)lane % B, q_own = (uint32_t)lane / B;

    for (;;) {
        unsigned leaf = lane == 0 ? atomicAdd(work, 1u) : 0u;
        leaf = __shfl_sync(0xffffffffu, leaf, 0);
        if (leaf >= count) break;

        const QueueEntry qe = lv.queue[leaf];
        const double tol = (double)a.planes[qe.plane].tol;
        const double eps2 = tol * tol * (double)n;           // exact: tol has 24 bits, n a power of 2
        const double E0 = (double)a.e0[leaf];
        const double Sy = sqrt(E0);
        const double tie_c = kTieRel * Sy, band_c = kBandRel * Sy;
        const double thr_e = eps2 - kTieRel * E0, band_e = kBandRel * E0;

        double c0r[E];
        const float2 *cp = a.c0 + (size_t)leaf * M;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int j = lane + 32 * s;
            c0r[s] = j < M ? (double)cp[j].x + (double)cp[j].y : 0.0;
        }

        for (int i = lane; i < M; i += 32) xd[i] = 0.0;
        __syncwarp();
        int nS = 0;
        bool conv = false, tie = false;
        for (;;) {
            // (a6) accuracy test before every step, strict
            double acc = 0.0;
            for (int i = lane; i < nS; i += 32) acc += xs[i] * c0s[i];
            const double En = E0 - warp_sum(acc);
            if (fabs(En - thr_e) < band_e) tie = true;
            if (En < thr_e) { conv = true; break; }
            if (nS == k) break;

            // residual correlations c = c0 - G[:, S] x_S
            double cv[E];
#pragma unroll
            for (int s = 0; s < E; ++s) cv[s] = c0r[s];
            if (SLOTS) {
                // slots [0, E/2) hold DCT atoms, [E/2, E) Haar atoms, and a
                // lane's atoms share p = lane mod B: a support atom of one
                // family reaches the other family's slots through
                // W[p_d][p_h] (one factor per lane) times W[q_d][q_h]
                for (int i = 0; i < nS; ++i) {
                    const uint32_t sa = Sj[i];
                    const double x = xs[i];
                    if (sa < (uint32_t)n) {
                        const uint32_t ps = sa % B, qs = sa / B;
                        const double ax = x * sW[ps * B + p_own];
#pragma unroll
                        for (int s = E / 2; s < E; ++s) cv[s] -= ax * sW[qs * B + q_own + (32 / B) * s - B];
                    } else {
                        const uint32_t ps = (sa - n) % B, qs = (sa - n) / B;
                        const double ax = x * sW[p_own * B + ps];
#pragma unroll
                        for (int s = 0; s < E / 2; ++s) cv[s] -= ax * sW[(q_own + (32 / B) * s) * B + qs];
                    }
                }
            } else if (NF == 2) {
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const uint32_t j = lane + 32 * s;
                    if (j >= (uint32_t)M) continue;
                    for (int i = 0; i < nS; ++i)
                        if ((Sj[i] >= (uint32_t)n) != (j >= (uint32_t)n)) cv[s] -= gram<B, NF>(sW, j, Sj[i]) * xs[i];
                }
            }
            // the diagonal: each support atom's own coefficient, kept dense
#pragma unroll
            for (int s = 0; s < E; ++s)
                if (lane + 32 * s < M) cv[s] -= xd[lane + 32 * s];
            double amax = 0.0;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                if ((uint32_t)(lane + 32 * s) >= (uint32_t)M) cv[s] = 0.0;
                amax = fmax(amax, fabs(cv[s]));
            }
            amax = warp_max(amax);
            if (amax <= tie_c) break;                        // nothing left to remove
            const double edge = amax - tie_c;
            uint32_t jl = kNoAtom;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const uint32_t j = lane + 32 * s;
                if (j >= (uint32_t)M) continue;
                const double m = fabs(cv[s]);
                if (m >= edge && j < jl) jl = j;
                if (fabs(m - edge) < band_c) tie = true;
            }
            const uint32_t jb = __reduce_min_sync(0xffffffffu, jl);
            double c0b = 0.0;
#pragma unroll
            for (int s = 0; s < E; ++s)
                if ((uint32_t)(lane + 32 * s) == jb) c0b = c0r[s];
            c0b = __shfl_sync(0xffffffffu, c0b, (int)(jb & 31u));

            // new Cholesky row: L w = G[S, jb] (rows lane and lane + 32)
            double g0 = lane < nS ? gram<B, NF>(sW, Sj[lane], jb) : 0.0;
            double g1 = lane + 32 < nS ? gram<B, NF>(sW, Sj[lane + 32], jb) : 0.0;
            for (int i = 0; i < nS; ++i) {
                double wi = 0.0;
                if (lane == (i & 31)) wi = (i < 32 ? g0 : g1) * rdiag[i];
                wi = __shfl_sync(0xffffffffu, wi, i & 31);
                if (lane == (i & 31)) {
                    if (i < 32) g0 = wi; else g1 = wi;
                }
                if (lane > i && lane < nS) g0 -= L[tri(lane) + i] * wi;
                if (lane + 32 > i && lane + 32 < nS) g1 -= L[tri(lane + 32) + i] * wi;
            }
            // g0 / g1 now hold w for the lane's rows
            const double d = 1.0 - warp_sum((lane < nS ? g0 * g0 : 0.0) + (lane + 32 < nS ? g1 * g1 : 0.0));
            if (d > kPivotMin * 0x1p-4 && d < kPivotMin * 0x1p4) tie = true;
            if (d <= kPivotMin) break;                       // dependent on the support
            const int rb = tri(nS);
            if (lane < nS) L[rb + lane] = g0;
            if (lane + 32 < nS) L[rb + lane + 32] = g1;
            if (lane == 0) {
                const double ld = sqrt(d);
                L[rb + nS] = ld;
                rdiag[nS] = 1.0 / ld;
                Sj[nS] = jb;
                c0s[nS] = c0b;
            }
            ++nS;
            __syncwarp();

            // re-fit: L z = c0_S, then L^T x = z (rows lane and lane + 32)
            double z0 = lane < nS ? c0s[lane] : 0.0;
            double z1 = lane + 32 < nS ? c0s[lane + 32] : 0.0;
            for (int i = 0; i < nS; ++i) {
                double zi = 0.0;
                if (lane == (i & 31)) zi = (i < 32 ? z0 : z1) * rdiag[i];
                zi = __shfl_sync(0xffffffffu, zi, i & 31);
                if (lane == (i & 31)) {
                    if (i < 32) z0 = zi; else z1 = zi;
                }
                if (lane > i && lane < nS) z0 -= L[tri(lane) + i] * zi;
                if (lane + 32 > i && lane + 32 < nS) z1 -= L[tri(lane + 32) + i] * zi;
            }
            for (int i = nS - 1; i >= 0; --i) {
                double xi = 0.0;
                if (lane == (i & 31)) xi = (i < 32 ? z0 : z1) * rdiag[i];
                xi = __shfl_sync(0xffffffffu, xi, i & 31);
                if (lane == (i & 31)) {
                    if (i < 32) z0 = xi; else z1 = xi;
                }
                if (lane < i) z0 -= L[tri(i) + lane] * xi;
                if (lane + 32 < i) z1 -= L[tri(i) + lane + 32] * xi;
            }
            if (lane < nS) {
                xs[lane] = z0;
                xd[Sj[lane]] = z0;
            }
            if (lane + 32 < nS) {
                xs[lane + 32] = z1;
                xd[Sj[lane + 32]] = z1;
            }
            __syncwarp();
        }

        // (a7) emit or split, as the MP kernel
        const bool tie_any = __any_sync(0xffffffffu, tie) != 0;
        if (lane == 0) {
            atomicAdd(&a.ctr->attempts[lv.level], 1ull);
            atomicAdd(&a.ctr->iterations[lv.level], (unsigned long long)nS);
            atomicMax(&a.ctr->max_steps[lv.level], (unsigned)nS);
        }
        const bool emit = conv || lv.is_last;
        uint32_t off = kNoAtom, eslot = 0;
        if (emit) {
            if (lane == 0) {
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
            }
            off = __shfl_sync(0xffffffffu, off, 0);
            eslot = __shfl_sync(0xffffffffu, eslot, 0);
            if (off != kNoAtom) {
                for (int i = lane; i < nS; i += 32) {
                    const double x = xs[i];
                    const float hi = (float)x;
                    a.atoms[off + i] = AtomRec{Sj[i], hi};
                    a.alpha_lo[off + i] = (float)(x - (double)hi);
                    a.atom_leaf[off + i] = eslot;
                }
            }
        } else if (lane == 0) {
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
        __syncwarp();
    }
}

template <int B, int NF>
static cudaError_t launch_omp_t(const MPArgs &a, int num_sms, cudaStream_t st) {
    constexpr int warps = 8;
    const int k = a.lv.k;
    const size_t bytes = (NF == 2 ? sizeof(double) * B * B : 0) +
                         warps * (sizeof(double) * (size_t)(tri(k) + 3 * k + NF * B * B) + sizeof(uint32_t) * (size_t)k);
    auto kern = omp_kernel<B, NF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long need = ((long long)a.lv.capacity + warps - 1) / warps;
    long long grid = (long long)num_sms * per_sm;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 32 * warps, bytes, st>>>(a);
    return cudaGetLastError();
}

int omp_max_budget(int b) {
    if (b >= 4 && b <= 16) return 64;
    if (b == 32 || b == 64) return omp_cta_max_budget();
    return 0;
}

cudaError_t launch_omp(const MPArgs &a, int nf, int num_sms, cudaStream_t st) {
    if (a.lv.k > omp_max_budget(a.lv.b)) return cudaErrorInvalidValue;
    if (a.lv.b >= 32) return launch_omp_cta(a, nf, st);
    if (nf == 2) {
        switch (a.lv.b) {
            case 4: return launch_omp_t<4, 2>(a, num_sms, st);
            case 8: return launch_omp_t<8, 2>(a, num_sms, st);
            case 16: return launch_omp_t<16, 2>(a, num_sms, st);
        }
    } else {
        switch (a.lv.b) {
            case 4: return launch_omp_t<4, 1>(a, num_sms, st);
            case 8: return launch_omp_t<8, 1>(a, num_sms, st);
            case 16: return launch_omp_t<16, 1>(a, num_sms, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace aqmp
