// mp.cu -- persistent per-leaf Matching Pursuit (Section 2.2 steps (b)-(d),
// stop rule Eq. (3)) with the quadtree split / emit of Algorithm 2.
//
// One group of T threads owns one leaf for its whole pursuit.  The leaf's M
// correlations c_j = <r, phi_j> live in registers as double-float pairs, E/T
// of them per thread (element j = lane + T s).  Each step:
//   (a3) argmax |c_j|, ties to the lowest j: a 64-bit order-preserving key
//        per element, a shuffle reduction inside each warp and, for groups
//        wider than a warp, one pass through shared memory;
//   (a4) alpha = c_j*; c <- c - alpha G[:, j*].  The dictionary is the union
//        of two orthonormal separable bases (DCT-II and Haar), so its Gram
//        matrix is [[I, X], [X^T, I]] with X = kron(W, W), W = C H^T (b x b):
//        the own-family column is e_j* (c_j* <- 0) and the other family's
//        column is the outer product W[p*, :] (x) W[q*, :].  It is generated
//        from W in shared memory, so no Gram column is read from memory;
//   (a5) E <- E - alpha^2 (Pythagoras for unit-norm atoms): the residual
//        vector itself is never needed, only its energy;
//   (a6) converged iff E < eps^2 (strict), tested before every step; the
//        budget ends the pursuit after k steps.
// Then (a7) a converged leaf, or any leaf at the smallest side, is emitted
// with its steps; any other leaf pushes its four quadrants (TL, TR, BL, BR)
// onto the next level's queue.
//
// Equality in finite precision: correlations within 2^-32 ||y|| of the
// largest count as tied and the lowest index among them wins; an energy
// within 2^-32 ||y||^2 of eps^2 counts as equal to it (not converged).  The
// FP64 oracle applies the same rule, so exact mathematical ties resolve the
// same way on both sides whatever their rounding.
//
// Certification: the pursuit's state carries ~2^-46 relative error.  Any
// decision within 2^-37 (of ||y||, resp. ||y||^2) of one of those boundaries
// -- another atom (not identical to the chosen one, as the DCT DC and Haar
// scaling atoms are) near the tie edge, or the energy near the threshold --
// marks the leaf AQMP_LEAF_NEAR_TIE: it is then not certified to agree with
// an exact evaluation.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

struct StepRec {
    uint32_t j;
    float hi, lo;
};

// (key, index) max with the lowest index among equal keys.
__device__ __forceinline__ void keep_better(uint32_t &bk, uint32_t &bj, uint32_t ok, uint32_t oj) {
    if (ok > bk || (ok == bk && oj < bj)) {
        bk = ok;
        bj = oj;
    }
}

__device__ __forceinline__ void warp_argmax32(uint32_t &bk, uint32_t &bj) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const uint32_t ok = __shfl_xor_sync(0xffffffffu, bk, off);
        const uint32_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
        keep_better(bk, bj, ok, oj);
    }
}

__device__ __forceinline__ void warp_argmax64(unsigned long long &bk, uint32_t &bj) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, off);
        const uint32_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
        if (ok > bk || (ok == bk && oj < bj)) {
            bk = ok;
            bj = oj;
        }
    }
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// B: block side; T: threads per leaf (32 = one warp per leaf, several
// leaves per CTA; > 32 = one leaf per CTA); NF: atom families (2 = DCT+Haar,
// 1 = a single orthonormal family).
template <int B, int T, int NF>
__global__ void __launch_bounds__(T > 32 ? T : 256)
mp_kernel(MPArgs a) {
    constexpr int n = B * B;
    constexpr int M = NF * n;
    constexpr int E = (M + T - 1) / T;
    static_assert(T % B == 0, "thread count must be a multiple of the side");
    constexpr int NW = T / 32;               // warps per group (T > 32)
    constexpr uint32_t NONE = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *sW = reinterpret_cast<float2 *>(smem);             // W[p][p'] (hi, lo)
    float2 *sWT = sW + B * B;                                    // W^T
    unsigned char *after_tables = smem + (NF == 2 ? 2 * B * B * sizeof(float2) : 0);
    uint32_t *sPk = reinterpret_cast<uint32_t *>(after_tables);  // [2][NW] keys
    uint32_t *sPj = sPk + 2 * NW;                                 // [2][NW] indices
    uint32_t *sMisc = sPj + 2 * NW;                               // [8]
    unsigned long long *sRk = reinterpret_cast<unsigned long long *>(sMisc + 8);   // [NW] (8-aligned)
    uint32_t *sRj = reinterpret_cast<uint32_t *>(sRk + NW);      // [NW]
    StepRec *sSteps = reinterpret_cast<StepRec *>(sRj + NW);

    const LevelArgs &lv = a.lv;
    if (NF == 2) {
        for (int i = threadIdx.x; i < B * B; i += blockDim.x) {
            sW[i] = a.W[i];
            sWT[i] = a.WT[i];
        }
    }
    __syncthreads();

    const int lane = (T == 32) ? (threadIdx.x & 31) : threadIdx.x;
    const int group = (T == 32) ? (threadIdx.x >> 5) : 0;
    const int groups = (T == 32) ? (blockDim.x >> 5) : 1;
    StepRec *steps = sSteps + (size_t)group * lv.k;
    const int p_own = lane % B;
    const unsigned count = *lv.count;
    const int k = lv.k;

    for (unsigned leaf = blockIdx.x * groups + group; leaf < count; leaf += gridDim.x * groups) {
        const QueueEntry qe = lv.queue[leaf];
        const float tol = a.planes[qe.plane].tol;
        const df eps2 = df_scale(df_two_prod(tol, tol), (float)n);     // exact
        const uint32_t e0 = a.e0[leaf];
        df En = df_from_i64((long long)e0);
        // accuracy threshold eps^2 - 2^-32 ||y||^2 and its certification band
        const df thrE = df_sub(eps2, df_scale(df_from_i64((long long)e0), 0x1p-32f));
        const float bandE_f = ldexpf((float)e0, -37);
        const float S_f = sqrtf((float)e0);
        // window of |hi| below the largest within which the order or the tie
        // rule may depend on the low words: a few ulps plus the tie band
        const float pre = ldexpf(S_f, -32) * 1.05f + ldexpf(S_f, -37) * 1.05f;

        float ch[E], cl[E];
        const float2 *cp = a.c0 + (size_t)leaf * M;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int j = lane + T * s;
            if (j < M) {
                const float2 v = cp[j];
                ch[s] = v.x;
                cl[s] = v.y;
            } else {
                ch[s] = 0.0f;
                cl[s] = 0.0f;
            }
        }

        int t = 0;
        bool conv = false, tie = false;
        for (;;) {
            // (a6) accuracy test before every step, strict
            const bool below = df_lt(En, thrE);
            if (fabsf(En.hi - thrE.hi) <= bandE_f * 1.01f + 0x1p-20f * fabsf(thrE.hi)) {
                if (fabs(df_to_double(En) - df_to_double(thrE)) < ldexp((double)e0, -37)) tie = true;
            }
            if (below) { conv = true; break; }
            if (t == k) break;

            // (a3) argmax |c|.  Main pass on the high words (largest |hi|,
            // lowest index among equal); a second pass in full precision only
            // when another atom lies within `window` of it.
            uint32_t bk = 0u, bj = NONE;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const int j = lane + T * s;
                if (j < M) {
                    const uint32_t key = __float_as_uint(ch[s]) & 0x7fffffffu;
                    if (key > bk) { bk = key; bj = (uint32_t)j; }
                }
            }
            warp_argmax32(bk, bj);
            const int par = t & 1;
            if (T > 32) {
                if ((lane & 31) == 0) {
                    sPk[par * NW + (lane >> 5)] = bk;
                    sPj[par * NW + (lane >> 5)] = bj;
                }
                __syncthreads();
                const int l = lane & 31;
                bk = l < NW ? sPk[par * NW + l] : 0u;
                bj = l < NW ? sPj[par * NW + l] : NONE;
                warp_argmax32(bk, bj);
            }
            if (bk == 0u) break;                 // every correlation is exactly zero
            uint32_t j1 = bj;
            const float amax = __uint_as_float(bk);
            const float window = amax * 0x1p-20f + pre;
            // candidates: atoms other than j1 whose |hi| is within the window
            bool cand = false;
            float vh = 0.0f, vl = 0.0f;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const int j = lane + T * s;
                if (j < M) {
                    if ((uint32_t)j == j1) { vh = ch[s]; vl = cl[s]; }
                    else if (fabsf(ch[s]) >= amax - window) cand = true;
                }
            }
            bool any_cand;
            df alpha;
            if (T > 32) {
                if ((uint32_t)lane == j1 % (uint32_t)T) {
                    sMisc[2 * par] = __float_as_uint(vh);
                    sMisc[2 * par + 1] = __float_as_uint(vl);
                }
                any_cand = __syncthreads_or(cand) != 0;
                alpha = df{__uint_as_float(sMisc[2 * par]), __uint_as_float(sMisc[2 * par + 1])};
            } else {
                any_cand = __any_sync(0xffffffffu, cand);
                const int src = (int)(j1 & 31u);
                alpha = df{__shfl_sync(0xffffffffu, vh, src), __shfl_sync(0xffffffffu, vl, src)};
            }
            if (any_cand) {
                // Full precision among the candidates (j1 included): the true
                // largest magnitude, then the lowest index within 2^-32 ||y||
                // of it; any candidate within 2^-37 ||y|| of that edge is not
                // certified.
                const double tieC = ldexp((double)S_f, -32);
                const double bandC = ldexp((double)S_f, -37);
                unsigned long long mk = 0ull;
                uint32_t mj = NONE;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int j = lane + T * s;
                    if (j < M && fabsf(ch[s]) >= amax - window) {
                        const double m = fabs((double)ch[s] + (double)cl[s]);
                        const unsigned long long key = (unsigned long long)__double_as_longlong(m);
                        if (key > mk) { mk = key; mj = (uint32_t)j; }
                    }
                }
                warp_argmax64(mk, mj);
                if (T > 32) {
                    if ((lane & 31) == 0) {
                        sRk[lane >> 5] = mk;
                        sRj[lane >> 5] = mj;
                    }
                    __syncthreads();
                    const int l = lane & 31;
                    mk = l < NW ? sRk[l] : 0ull;
                    mj = l < NW ? sRj[l] : NONE;
                    warp_argmax64(mk, mj);
                }
                const double mmax = __longlong_as_double((long long)mk);
                const double edge = mmax - tieC;
                uint32_t lower = NONE;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int j = lane + T * s;
                    if (j < M && fabsf(ch[s]) >= amax - window) {
                        const double m = fabs((double)ch[s] + (double)cl[s]);
                        if (fabs(m - edge) < bandC) tie = true;
                        if (m >= edge && (uint32_t)j < lower) lower = (uint32_t)j;
                    }
                }
                float wh = 0.0f, wl = 0.0f;
                if (T > 32) {
                    if (lane == 0) sMisc[6] = NONE;
                    __syncthreads();
                    if (lower != NONE) atomicMin(&sMisc[6], lower);
                    __syncthreads();
                    lower = sMisc[6];
#pragma unroll
                    for (int s = 0; s < E; ++s)
                        if ((uint32_t)(lane + T * s) == lower) { wh = ch[s]; wl = cl[s]; }
                    if ((uint32_t)lane == lower % (uint32_t)T) {
                        sMisc[4] = __float_as_uint(wh);
                        sMisc[5] = __float_as_uint(wl);
                    }
                    __syncthreads();
                    wh = __uint_as_float(sMisc[4]);
                    wl = __uint_as_float(sMisc[5]);
                    __syncthreads();
                } else {
                    lower = warp_min(lower);
#pragma unroll
                    for (int s = 0; s < E; ++s)
                        if ((uint32_t)(lane + T * s) == lower) { wh = ch[s]; wl = cl[s]; }
                    wh = __shfl_sync(0xffffffffu, wh, (int)(lower & 31u));
                    wl = __shfl_sync(0xffffffffu, wl, (int)(lower & 31u));
                }
                j1 = lower;
                alpha = df{wh, wl};
            }
            if (lane == 0) steps[t] = StepRec{j1, alpha.hi, alpha.lo};

            // (a5) energy
            En = df_sub(En, df_mul(alpha, alpha));

            // (a4) correlation update through the Gram matrix
            const int fam1 = (int)(j1 >= (uint32_t)n);
            const int f1 = (int)j1 - fam1 * n;
            if (NF == 2) {
                const int p1 = f1 % B, q1 = f1 / B;
                const float2 *V = fam1 ? sWT : sW;
                const float2 vp = V[p1 * B + p_own];
                const df u = df_mul(alpha, df{vp.x, vp.y});
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int j = lane + T * s;
                    if (j < M) {
                        const int fam = (int)(j >= n);
                        if (fam != fam1) {
                            const int q = (j - fam * n) / B;
                            const float2 w = V[q1 * B + q];
                            const df r = df_sub_mul(df{ch[s], cl[s]}, u, df{w.x, w.y});
                            ch[s] = r.hi;
                            cl[s] = r.lo;
                        } else if (j == (int)j1) {
                            ch[s] = 0.0f;
                            cl[s] = 0.0f;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    if (lane + T * s == (int)j1) {
                        ch[s] = 0.0f;
                        cl[s] = 0.0f;
                    }
                }
            }
            ++t;
        }

        // group-wide outcome of the certification
        bool tie_any;
        if (T > 32) {
            tie_any = __syncthreads_or(tie) != 0;
        } else {
            tie_any = __any_sync(0xffffffffu, tie) != 0;
        }
        if (lane == 0) {
            atomicAdd(&a.ctr->attempts[lv.level], 1ull);
            atomicAdd(&a.ctr->iterations[lv.level], (unsigned long long)t);
        }
        const bool emit = conv || lv.is_last;
        uint32_t off = 0;
        if (emit) {
            if (lane == 0) {
                const unsigned long long slot = atomicAdd(&a.ctr->n_leaves, 1ull);
                const unsigned long long o = atomicAdd(&a.ctr->n_atoms, (unsigned long long)t);
                uint8_t flags = (uint8_t)((tie_any ? 1u : 0u) | (qe.flags & 2u));
                if (slot >= a.leaf_cap || o + t > a.atom_cap) {
                    raise_error(a.ctr, kDevErrQueueOverflow, 1u);
                    off = 0xffffffffu;
                } else {
                    LeafRec rec;
                    rec.plane = qe.plane;
                    rec.y = qe.y;
                    rec.x = qe.x;
                    rec.atom_off = (uint32_t)o;
                    rec.b = (uint16_t)B;
                    rec.n_atoms = (uint16_t)t;
                    rec.converged = conv ? 1 : 0;
                    rec.flags = flags;
                    rec.reserved = 0;
                    a.leaves[slot] = rec;
                    off = (uint32_t)o;
                    if (flags) atomicAdd(&a.ctr->near_tie_leaves, 1ull);
                }
            }
        } else if (lane == 0) {
            const unsigned slot = atomicAdd(lv.next_count, 4u);
            if (slot + 4u > lv.next_capacity) {
                raise_error(a.ctr, kDevErrQueueOverflow, 2u);
            } else {
                const uint32_t h = B / 2;
                const uint32_t fl = (qe.flags & 2u) | (tie_any ? 2u : 0u);
                lv.next_queue[slot + 0] = QueueEntry{qe.plane, qe.y, qe.x, fl};
                lv.next_queue[slot + 1] = QueueEntry{qe.plane, qe.y, qe.x + h, fl};
                lv.next_queue[slot + 2] = QueueEntry{qe.plane, qe.y + h, qe.x, fl};
                lv.next_queue[slot + 3] = QueueEntry{qe.plane, qe.y + h, qe.x + h, fl};
            }
        }
        if (emit) {
            if (T > 32) {
                if (lane == 0) sMisc[0] = off;
                __syncthreads();
                off = sMisc[0];
            } else {
                __syncwarp();
                off = __shfl_sync(0xffffffffu, off, 0);
            }
            if (off != 0xffffffffu) {
                for (int i = lane; i < t; i += T) {
                    const StepRec st = steps[i];
                    a.atoms[off + i] = AtomRec{st.j, st.hi};
                    a.alpha_lo[off + i] = st.lo;
                }
            }
        }
        if (T > 32) __syncthreads(); else __syncwarp();
    }
}

template <int B, int T, int NF>
static size_t mp_smem_bytes(int k, int groups) {
    constexpr int NW = T / 32;
    size_t bytes = (NF == 2 ? 2 * B * B * sizeof(float2) : 0);
    bytes += 4 * NW * sizeof(uint32_t) + 8 * sizeof(uint32_t);        // partials, misc
    bytes += NW * sizeof(unsigned long long) + NW * sizeof(uint32_t);  // wide partials
    bytes += (size_t)groups * k * sizeof(StepRec);
    return bytes;
}

template <int B, int T, int NF>
static cudaError_t launch_mp_t(const MPArgs &a, int num_sms, cudaStream_t st) {
    const int block = (T == 32) ? 256 : T;
    const int groups = (T == 32) ? block / 32 : 1;
    const size_t smem = mp_smem_bytes<B, T, NF>(a.lv.k, groups);
    auto kern = mp_kernel<B, T, NF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long need = ((long long)a.lv.capacity + groups - 1) / groups;
    long long grid = (long long)num_sms * per_sm;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mp(const MPArgs &a, int nf, int num_sms, cudaStream_t st) {
    const int b = a.lv.b;
    if (nf == 2) {
        switch (b) {
            case 4: return launch_mp_t<4, 32, 2>(a, num_sms, st);
            case 8: return launch_mp_t<8, 32, 2>(a, num_sms, st);
            case 16: return launch_mp_t<16, 32, 2>(a, num_sms, st);
            case 32: return launch_mp_t<32, 128, 2>(a, num_sms, st);
            case 64: return launch_mp_t<64, 512, 2>(a, num_sms, st);
        }
    } else {
        switch (b) {
            case 4: return launch_mp_t<4, 32, 1>(a, num_sms, st);
            case 8: return launch_mp_t<8, 32, 1>(a, num_sms, st);
            case 16: return launch_mp_t<16, 32, 1>(a, num_sms, st);
            case 32: return launch_mp_t<32, 128, 1>(a, num_sms, st);
            case 64: return launch_mp_t<64, 512, 1>(a, num_sms, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace aqmp
