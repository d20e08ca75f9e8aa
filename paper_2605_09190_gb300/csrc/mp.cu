// mp.cu -- persistent per-leaf Matching Pursuit (Section 2.2 steps (b)-(d),
// stop rule Eq. (3)) with the quadtree split / emit of Algorithm 2.
//
// One group of T threads owns one leaf for its whole pursuit.  The leaf's M
// correlations c_j = <r, phi_j> live in registers as double-float pairs, E of
// them per thread (element j = lane + T s).  Each step:
//   (a3) argmax |c_j|, lowest j among equals;
//   (a4) alpha = c_j*; c <- c - alpha G[:, j*].  The dictionary is the union
//        of two orthonormal separable bases (DCT-II and Haar), so its Gram
//        matrix is [[I, X], [X^T, I]] with X = kron(W, W), W = C H^T (b x b):
//        the own-family column is e_j* (c_j* <- 0) and the other family's
//        column is the outer product W[p*, :] (x) W[q*, :], generated from W
//        in shared memory -- no Gram column is read from memory;
//   (a5) E <- E - alpha^2 (Pythagoras for unit-norm atoms): the residual
//        vector itself is never needed, only its energy;
//   (a6) converged iff E < eps^2 (strict), tested before every step; the
//        budget ends the pursuit after k steps.
// Then (a7) a converged leaf, or any leaf at the smallest side, is emitted
// with its steps (and marked in the cell map that restores the depth-first
// order); any other leaf pushes its four quadrants (TL, TR, BL, BR) onto the
// next level's queue.  Leaves are handed out through a device
// counter, so a group that finishes a short pursuit takes the next leaf.
//
// Argmax cost.  Each thread keeps, per atom family, the top two |hi| keys of
// its elements (with the top's index, sign and low word).  A step changes one
// family (and zeroes one element of the other), so only that family's top-2
// is recomputed.  The group reduction carries (top key, index | sign, second
// key, low word): alpha arrives with the reduction, and whether any other
// atom lies within the decision window of the best is read off the second
// key, with no extra pass over the elements.
//
// Equality in finite precision: correlations within 2^-32 ||y|| of the
// largest count as tied and the lowest index among them wins; an energy
// within 2^-32 ||y||^2 of eps^2 counts as equal to it (not converged).  The
// FP64 oracle applies the same rule, so exact mathematical ties resolve the
// same way on both sides whatever their rounding.  When another atom is in
// the window, the step is decided in full precision over the candidates.
//
// Certification: the pursuit's state carries ~2^-46 relative error.  Any
// decision within 2^-37 (of ||y||, resp. ||y||^2) of one of those boundaries
// marks the leaf AQMP_LEAF_NEAR_TIE: it is then not certified to agree with
// an exact evaluation.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "mp_step.cuh"
#include "sep.cuh"
#include <cuda_fp16.h>


namespace aqmp {

// B: block side; T: threads per leaf (32 = one warp per leaf, several
// leaves per CTA; > 32 = one leaf per CTA); NF: atom families (2 = DCT+Haar,
// 1 = a single orthonormal family); DF: double-float state with certified
// decisions (true) or the plain FP32 form (false: FP32 correlations, energy
// and stop test, one FMA per Gram entry, no certification).

// MINB: resident CTAs per SM the compiler is asked to fit (registers per
// thread follow): 1 keeps the side-64 state in registers for the fastest
// single pursuit, 2 halves the registers so two leaves share an SM, which
// wins when leaves outnumber SMs.
// The BF16 form with rescore: the exact form's initial correlation of atoms
// list[0..cnt) (cnt <= 8) of one leaf, one warp per atom, each as the exact
// kernels compute it (sep.cuh): Z~[p][m] = sum_i Bf[p][i] y~[i][m] for
// m = lane and lane + 32 from the leaf's pixels (pixT[i b + m] = y - 128),
// T = sum_m Bf[q][m] Z~[p][m] + 128 R[p] R[q] in int128, rounded once;
// rv[w] receives that value minus the BF16 correlation's, as a double-float.
// Out of line: rounds are rare, and keeping their code out of the step keeps
// the step's code in the instruction cache.
template <int B, int NF>
__device__ __noinline__ void rescore_atoms(const MPArgs &a, unsigned leaf, const int8_t *pixT,
                                           const uint32_t *list, uint32_t cnt, float2 *rv, long long *rowbuf) {
    static_assert(B == 64, "two columns per lane");
    constexpr uint32_t n = B * B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((uint32_t)warp >= cnt) return;
    const uint32_t j = list[warp];
    const int F = NF == 2 ? (int)(j >= n) : a.fam0;
    const uint32_t f = j % n, p = f % B, q = f / B;
    const float2 approx = lane == 0 ? a.c0[(size_t)leaf * (NF * n) + j] : make_float2(0.0f, 0.0f);
    // row p of the fixed-point 1-D basis (its two 24-bit limbs) into this
    // warp's buffer, two entries a lane
    int2 *row = reinterpret_cast<int2 *>(rowbuf) + warp * B;
    {
        const int2 *rp = a.Bs + ((size_t)F * B + p) * B;
        row[lane] = rp[lane];
        row[lane + 32] = rp[lane + 32];
    }
    const int2 *rq = a.Bs + ((size_t)F * B + q) * B;
    const int2 w0 = rq[lane], w1 = rq[lane + 32];
    __syncwarp();
    // columns m = lane and lane + 32: the hi- and lo-limb sums as 32 x 32 ->
    // 64-bit multiply-adds (|limb y| < 2^31, 64 terms < 2^37), then
    // Z = 2^24 Zhi + Zlo (< 2^60)
    long long h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll 16
    for (int i = 0; i < B; ++i) {
        const int2 w = row[i];
        const int y0 = pixT[i * B + lane], y1 = pixT[i * B + lane + 32];
        h0 += (long long)w.y * y0;
        l0 += (long long)w.x * y0;
        h1 += (long long)w.y * y1;
        l1 += (long long)w.x * y1;
    }
    const long long z0 = h0 * 16777216ll + l0, z1 = h1 * 16777216ll + l1;
    __int128 acc = (__int128)((long long)w0.y * 16777216ll + (long long)w0.x) * z0 +
                   (__int128)((long long)w1.y * 16777216ll + (long long)w1.x) * z1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)acc, off);
        const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(acc >> 64), off);
        acc += (__int128)hi * ((__int128)1 << 64) + (__int128)lo;
    }
    if (lane == 0) {
        const __int128 T = acc + (__int128)(128ll * a.Rs[F * B + p]) * a.Rs[F * B + q];
        const df d = df_sub(int128_to_df(T), df{approx.x, approx.y});
        rv[warp] = make_float2(d.hi, d.lo);
    }
}

// RESC: the BF16 form with rescore (side 64, several warps per leaf, double-
// float state).  The leaf starts from the BF16 correlation c~0, within e_j
// of the exact form's c0 for every atom j; a shared bitmask records which
// atoms already carry their exact value.  Before a step is taken, every atom
// that could be the argmax -- an upper bound |c_j| + e_j (0 once exact) at
// or above the leader's lower bound less the full-precision window -- must
// be exact: its c0 recomputed from the pixels (rescore_atoms) and the
// difference added to its running correlation (the Gram updates applied so
// far are the same for both starts).  A round that has to rescore fills its
// 8 slots with further non-exact atoms above lambda times the leader (lambda
// adapted per leaf), the likely leaders of the next steps.  The step is then
// decided as in the exact form.  More than 8 atoms that must be rescored in
// one step hand the leaf, untouched, to the exact path.
template <int B, int T, int NF, bool DF, int MINB = (T > 32 ? 1 : 2), bool RESC = false>
__global__ void __launch_bounds__(T > 32 ? T : 256, MINB)
mp_kernel(MPArgs a) {
    constexpr int n = B * B;
    constexpr int M = NF * n;
    constexpr int E = (M + T - 1) / T;
    static_assert(T % B == 0, "thread count must be a multiple of the side");
    constexpr int NW = T / 32;               // warps per group (T > 32)
    static_assert(!RESC || (DF && T > 32 && NW >= 8 && E <= 32 && (M % T) == 0), "rescore layout");
    // SPLIT: the first E/2 elements of every thread are DCT atoms and the
    // rest Haar atoms, each family cached separately; otherwise one group.
    constexpr bool SPLIT = NF == 2 && (n % T) == 0 && (E % 2) == 0;
    constexpr int NG = SPLIT ? 2 : 1;
    constexpr int G = E / NG;
    constexpr bool FULL = (M % T) == 0;      // every (lane, s) is an atom
    // STALE: when the chosen atom was the top of its owner's summary, its
    // removal leaves that summary's second key as the exact new largest
    // magnitude; the owner keeps it with an unknown index (low word 0)
    // instead of rescanning its registers every step, and rescans only if
    // such a summary ever holds the group's largest key.  Equal keys put an
    // atom within the decision window, which is decided from the registers.
    // Measured on the 512x512 sweep: 9% faster at b = 32, 20% at b = 16; at
    // b = 64 the bookkeeping costs more than the rescan it saves (the
    // owner's rescan overlaps seven other warps' updates), so it is off there.
    constexpr bool STALE = SPLIT && DF && B < 64;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *sW = reinterpret_cast<float2 *>(smem);             // W[p][p'] (hi, lo)
    float2 *sWT = sW + B * B;                                    // W^T
    unsigned char *after_tables = smem + (NF == 2 ? 2 * B * B * sizeof(float2) : 0);
    uint4 *sPart = reinterpret_cast<uint4 *>(after_tables);      // [3][NW] top-2 partials
    uint32_t *sMisc = reinterpret_cast<uint32_t *>(sPart + 3 * NW);               // [12]
    unsigned long long *sRk = reinterpret_cast<unsigned long long *>(sMisc + 12); // [NW]
    uint32_t *sRj = reinterpret_cast<uint32_t *>(sRk + NW);      // [NW]
    StepRec *sSteps = reinterpret_cast<StepRec *>(sRj + NW);
    // RESC: the leaf's pixels (transposed), its bounds (FP16, rounded up),
    // the exact atoms (bitmask), the rescore's partial sums and a few words
    unsigned char *resc = reinterpret_cast<unsigned char *>(sSteps + (size_t)(T == 32 ? blockDim.x / 32 : 1) * a.lv.k);
    resc = reinterpret_cast<unsigned char *>(((uintptr_t)resc + 15) & ~(uintptr_t)15);
    int8_t *sPix = reinterpret_cast<int8_t *>(resc);
    __half *sE = reinterpret_cast<__half *>(resc + B * B);                 // [M]
    uint32_t *sEx = reinterpret_cast<uint32_t *>(sE + M);                  // [M / 32]
    unsigned long long *sP = reinterpret_cast<unsigned long long *>(sEx + (M + 31) / 32);   // [16]
    float2 *sRv = reinterpret_cast<float2 *>(sP + 16);                     // [8] one per rescored atom
    uint32_t *sRW = reinterpret_cast<uint32_t *>(sRv + 8);                 // [0..1] counts, [2..9] atoms
    float *sEm = reinterpret_cast<float *>(sRW + 16);                      // [NW]
    long long *sRow = reinterpret_cast<long long *>(resc + ((B * B + NF * B * B * 2 + (NF * B * B + 31) / 32 * 4 +
                                                              16 * 8 + 8 * 8 + 16 * 4 + NW * 4 + 15) & ~15));  // [8][B]
    const LevelArgs &lv = a.lv;
    __shared__ unsigned long long sCnt[3];              // per-CTA work counters (T == 32)
    __shared__ unsigned sMaxT;
    if (T == 32 && threadIdx.x < 3) sCnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) sMaxT = 0u;
    if (NF == 2) {
        for (int i = threadIdx.x; i < B * B; i += blockDim.x) {
            sW[i] = a.W[i];
            sWT[i] = a.WT[i];
        }
    }
    __syncthreads();

    const int lane = (T == 32) ? (threadIdx.x & 31) : threadIdx.x;
    const int group = (T == 32) ? (threadIdx.x >> 5) : 0;
    StepRec *steps = sSteps + (size_t)group * lv.k;
    const int p_own = lane % B;
    const unsigned count = *lv.count;
    const int k = lv.k;
    unsigned *work = a.work ? a.work : &a.ctr->work_next[lv.level];
    unsigned long long n_attempts = 0, n_steps = 0, n_windows = 0, n_resc = 0, n_rounds = 0;
    unsigned max_t = 0;

    for (;;) {
        // dynamic assignment: the next unclaimed leaf of this level
        unsigned leaf;
        if (T > 32) {
            if (lane == 0) sMisc[7] = atomicAdd(work, 1u);
            __syncthreads();
            leaf = sMisc[7];
            __syncthreads();
        } else {
            leaf = lane == 0 ? atomicAdd(work, 1u) : 0u;
            leaf = __shfl_sync(0xffffffffu, leaf, 0);
        }
        if (leaf >= count) break;

        const QueueEntry qe = lv.queue[leaf];
        const float tol = a.planes[qe.plane].tol;
        const df eps2 = df_scale(df_two_prod(tol, tol), (float)n);     // exact
        const uint32_t e0 = a.e0[leaf];
        df En = df_from_i64((long long)e0);
        // accuracy threshold eps^2 - 2^-32 ||y||^2 and its certification band
        const df thrE = df_sub(eps2, df_scale(df_from_i64((long long)e0), 0x1p-32f));
        const float bandE_f = ldexpf((float)e0, -37);
        const float eps2_f = __fmul_rn(__fmul_rn(tol, tol), (float)n);   // FP32 form's threshold
        const float S_f = sqrtf((float)e0);
        // window of |hi| below the largest within which the order or the tie
        // rule may depend on the low words: a few ulps plus the tie band
        const float pre = ldexpf(S_f, -32) * 1.05f + ldexpf(S_f, -37) * 1.05f;

        float ch[E], cl[E];
        Top2 top[NG];
        bool stale[NG];             // see STALE below
        const float2 *cp = a.c0 + (size_t)leaf * M;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            top[g] = top2_empty();
            stale[g] = false;
        }
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int j = lane + T * s;
            if (FULL || j < M) {
                const float2 v = cp[j];
                ch[s] = v.x;
                cl[s] = DF ? v.y : 0.0f;
                top2_fold(top[s / G], v.x, cl[s], (uint32_t)j);
            } else {
                ch[s] = 0.0f;
                cl[s] = 0.0f;
            }
        }

        float my_emax = 0.0f;               // RESC: largest bound of this thread's non-exact atoms
        uint32_t exm = 0u;                  // RESC: this thread's exact slots (the bitmask's own bits)
        float lam = 0.5f;                   // RESC: speculative threshold, relative to the leader
        float emax_all = 0.0f;              // RESC: largest bound of the leaf's non-exact atoms
        bool fallback = false;
        if constexpr (RESC) {
#pragma unroll
            for (int s2 = 0; s2 < E; ++s2) {
                const uint32_t j = (uint32_t)(lane + T * s2);
                const __half e = __float2half_ru(a.ebound[(size_t)leaf * M + j]);
                my_emax = fmaxf(my_emax, __half2float(e));       // the value the scans compare with
                sE[j] = e;
            }
            for (int w = lane; w < (M + 31) / 32; w += T) sEx[w] = 0u;
            if (lane < 2) sRW[lane] = 0u;
            {
                float v = my_emax;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
                if ((lane & 31) == 0) sEm[lane >> 5] = v;
            }
            const int centre = (int)a.mu[leaf] - 128;
            for (int v = lane; v < n; v += T)
                sPix[(v % B) * B + v / B] =
                    (int8_t)((int)__bfloat162float(a.Yc[(size_t)leaf * a.Kpad + v]) + centre);
            __syncthreads();
#pragma unroll
            for (int w = 0; w < NW; ++w) emax_all = fmaxf(emax_all, sEm[w]);
        }

        int t = 0, windows = 0;
        bool conv = false, tie = false;
        // With several warps per leaf, warp 0 alone keeps the residual energy
        // and takes the accuracy test; its verdict travels with the step's
        // argmax exchange (the test still decides before the step is used).
        const bool energy_warp = T == 32 || lane < 32;
        for (;;) {
            // (a6) accuracy test before every step, strict
            bool below = false;
            if (energy_warp) {
                below = DF ? df_lt(En, thrE) : (En.hi < eps2_f);
                if (DF && fabsf(En.hi - thrE.hi) <= bandE_f * 1.01f + 0x1p-20f * fabsf(thrE.hi)) {
                    if (fabs(df_to_double(En) - df_to_double(thrE)) < ldexp((double)e0, -37)) tie = true;
                }
            }
            if (T == 32) {
                if (below) { conv = true; break; }
                if (t == k) break;
            } else if (t == k) {
                if (lane == 0) sMisc[10] = below ? 1u : 0u;
                __syncthreads();
                conv = sMisc[10] != 0u;
                break;
            }

            // (a3) argmax |c| on the cached top-2 summaries
            bool stop = false;
            auto group_best = [&](int buf) {
                Top2 b = top[0];
#pragma unroll
                for (int g = 1; g < NG; ++g) b = top2_merge(b, top[g]);
                b = warp_top2(b);
                if (T > 32) {
                    if ((lane & 31) == 0)
                        sPart[buf * NW + (lane >> 5)] =
                            make_uint4((uint32_t)b.P, (uint32_t)(b.P >> 32), b.k2, __float_as_uint(b.lo1));
                    if (buf < 2 && lane == 0) sMisc[8 + buf] = below ? 1u : 0u;
                    __syncthreads();
                    if (buf < 2) stop = sMisc[8 + buf] != 0u;
                    const int l = lane & 31;
                    if (l < NW) {
                        const uint4 v = sPart[buf * NW + l];
                        b = Top2{((unsigned long long)v.y << 32) | v.x, v.z, __uint_as_float(v.w)};
                    } else {
                        b = top2_empty();
                    }
                    b = warp_top2(b);
                }
                return b;
            };
            Top2 best = group_best(t & 1);
            if (T > 32 && stop) { conv = true; break; }
            if (STALE && (best.P >> 32) != 0ull && (uint32_t)best.P == 0u) {
                // a summary left stale by the last step holds the largest
                // magnitude: its owners rescan and the group reduces again
                if (stale[0]) { top[0] = zero_and_rescan<T, E, G, 0>(ch, cl, lane, kNone); stale[0] = false; }
                if (stale[NG - 1]) {
                    top[NG - 1] = zero_and_rescan<T, E, G, G>(ch, cl, lane, kNone);
                    stale[NG - 1] = false;
                }
                best = group_best(2);
            }
            if ((best.P >> 32) == 0ull) break;   // every correlation is exactly zero
            if constexpr (RESC) {
                // certify the leader against the bounds: every atom whose
                // upper bound |c| + e reaches the leader's lower bound less the
                // full-precision window must be exact before the step is taken.
                // The per-step test is a branch-free mask over the thread's
                // slots against its largest bound; the exact bounds are read
                // only for the few slots it leaves
                uint32_t newly = 0u;
                for (;;) {
                    const uint32_t jb = top2_index(best);
                    const float amb = top2_amax(best);
                    const bool exb = (sEx[jb >> 5] >> (jb & 31)) & 1u;
                    const float eb = exb ? 0.0f : __half2float(sE[jb]);
                    const float L = __fsub_rd(__fsub_rd(amb, eb), __fadd_ru(__fmul_ru(amb, 0x1p-20f), pre));
                    // no atom can reach the leader: nothing to exchange
                    if (exb && __fadd_ru(__uint_as_float(best.k2), emax_all) < L) break;
                    float mine = top2_amax(top[0]);
#pragma unroll
                    for (int g = 1; g < NG; ++g) mine = fmaxf(mine, top2_amax(top[g]));
                    bool found = false;
                    if (__fadd_ru(mine, my_emax) >= L) {
                        const float thr = __fsub_rd(L, my_emax);
                        uint32_t cm = 0u;
#pragma unroll
                        for (int s2 = 0; s2 < E; ++s2) cm |= (fabsf(ch[s2]) >= thr ? 1u : 0u) << s2;
                        cm &= ~exm;
                        while (cm) {
                            const int s2 = __ffs(cm) - 1;
                            cm &= cm - 1u;
                            float m = 0.0f;
#pragma unroll
                            for (int s3 = 0; s3 < E; ++s3) m = s3 == s2 ? fabsf(ch[s3]) : m;
                            const uint32_t j = (uint32_t)(lane + T * s2);
                            if (__fadd_ru(m, __half2float(sE[j])) >= L) {
                                const uint32_t idx = atomicAdd(&sRW[0], 1u);
                                if (idx < 8u) sRW[2 + idx] = j;
                                found = true;
                            }
                        }
                    }
                    if (__syncthreads_or(found) == 0) break;          // nothing to rescore
                    const uint32_t cnt = min(sRW[0], 9u);
                    newly += cnt;
                    if (newly > 8u) { fallback = true; break; }
                    // fill the round with the likely next leaders: non-exact atoms
                    // above lam times the leader (not already listed), counted per
                    // warp (one shared atomic per warp), placed while there is room
                    uint32_t qmask = 0u;
                    if (mine >= lam * amb) {
                        const float thq = lam * amb;
#pragma unroll
                        for (int s2 = 0; s2 < E; ++s2) qmask |= (fabsf(ch[s2]) >= thq ? 1u : 0u) << s2;
                        qmask &= ~exm;
                        // drop the ones listed above (their owner is this thread)
                        for (uint32_t w = 0; w < cnt; ++w) {
                            const uint32_t j = sRW[2 + w];
                            if (j % (uint32_t)T == (uint32_t)lane) qmask &= ~(1u << (j / (uint32_t)T));
                        }
                    }
                    {
                        const uint32_t qc = (uint32_t)__popc(qmask);
                        uint32_t incl = qc;
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) {
                            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                            if ((lane & 31) >= off) incl += v;
                        }
                        const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
                        uint32_t wbase = 0u;
                        if ((lane & 31) == 31 && wtot) wbase = atomicAdd(&sRW[1], wtot);
                        wbase = __shfl_sync(0xffffffffu, wbase, 31);
                        uint32_t pos = cnt + wbase + incl - qc;
                        while (qmask && pos < 8u) {
                            const int s2 = __ffs(qmask) - 1;
                            qmask &= qmask - 1u;
                            sRW[2 + pos] = (uint32_t)(lane + T * s2);
                            ++pos;
                        }
                    }
                    __syncthreads();
                    const uint32_t spec = sRW[1];
                    const uint32_t tot = min(8u, cnt + spec);
                    rescore_atoms<B, NF>(a, leaf, sPix, sRW + 2, tot, sRv, sRow);
                    // steer toward 8..32 atoms above the threshold
                    lam = spec > 32u ? 0.5f * (1.0f + lam) : spec < 8u ? 0.5f * lam : lam;
                    __syncthreads();
                    if (lane == 0) {
                        sRW[0] = 0u;
                        sRW[1] = 0u;
                        n_resc += tot;
                        ++n_rounds;
                    }
                    // into the owners' registers: one predicated pass per atom
                    uint32_t touched = 0u;               // bit g: family g's summary to redo
                    bool redo_e = false;                 // the thread's largest bound left with it
                    for (uint32_t w = 0; w < tot; ++w) {
                        const uint32_t j = sRW[2 + w];
                        if (j % (uint32_t)T != (uint32_t)lane) continue;
                        const uint32_t sj = j / (uint32_t)T;
                        float vh = 0.0f, vl = 0.0f;
#pragma unroll
                        for (int s2 = 0; s2 < E; ++s2) {
                            vh = (uint32_t)s2 == sj ? ch[s2] : vh;
                            vl = (uint32_t)s2 == sj ? cl[s2] : vl;
                        }
                        const float2 d = sRv[w];
                        const df c = df_add(df{vh, vl}, df{d.x, d.y});
#pragma unroll
                        for (int s2 = 0; s2 < E; ++s2) {
                            ch[s2] = (uint32_t)s2 == sj ? c.hi : ch[s2];
                            cl[s2] = (uint32_t)s2 == sj ? c.lo : cl[s2];
                        }
                        exm |= 1u << sj;
                        atomicOr(&sEx[j >> 5], 1u << (j & 31));
                        touched |= 1u << (sj / (uint32_t)G);
                        redo_e |= __half2float(sE[j]) >= my_emax;
                    }
                    if (touched & 1u) top[0] = zero_and_rescan<T, E, G, 0>(ch, cl, lane, kNone);
                    if (NG > 1 && (touched & 2u)) top[NG - 1] = zero_and_rescan<T, E, G, G>(ch, cl, lane, kNone);
                    if (redo_e) {
                        my_emax = 0.0f;
                        for (int s2 = 0; s2 < E; ++s2)
                            if (!((exm >> s2) & 1u)) my_emax = fmaxf(my_emax, __half2float(sE[lane + T * s2]));
                    }
                    {
                        float v = my_emax;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
                        if ((lane & 31) == 0) sEm[lane >> 5] = v;
                    }
                    __syncthreads();
                    emax_all = sEm[0];
#pragma unroll
                    for (int w = 1; w < NW; ++w) emax_all = fmaxf(emax_all, sEm[w]);
                    best = group_best(2);
                }
                if (fallback || (best.P >> 32) == 0ull) break;
            }
            uint32_t j1 = top2_index(best);
            const float amax = top2_amax(best);
            df alpha = df{top2_negative(best) ? -amax : amax, best.lo1};
            const float window = amax * 0x1p-20f + pre;
            bool rare = false;
            if (DF && __uint_as_float(best.k2) >= amax - window) {
                rare = true;
                ++windows;
                // Another atom is within the window: decide in full precision
                // among the candidates -- the true largest magnitude, then the
                // lowest index within 2^-32 ||y|| of it; any candidate within
                // 2^-37 ||y|| of that edge is not certified.
                const double tieC = ldexp((double)S_f, -32);
                const double bandC = ldexp((double)S_f, -37);
                unsigned long long mk = 0ull;
                uint32_t mj = kNone;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int j = lane + T * s;
                    if ((FULL || j < M) && fabsf(ch[s]) >= amax - window) {
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
                    mj = l < NW ? sRj[l] : kNone;
                    warp_argmax64(mk, mj);
                }
                const double edge = __longlong_as_double((long long)mk) - tieC;
                uint32_t lower = kNone;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int j = lane + T * s;
                    if ((FULL || j < M) && fabsf(ch[s]) >= amax - window) {
                        const double m = fabs((double)ch[s] + (double)cl[s]);
                        if (fabs(m - edge) < bandC) tie = true;
                        if (m >= edge && (uint32_t)j < lower) lower = (uint32_t)j;
                    }
                }
                float wh = 0.0f, wl = 0.0f;
                if (T > 32) {
                    if (lane == 0) sMisc[6] = kNone;
                    __syncthreads();
                    if (lower != kNone) atomicMin(&sMisc[6], lower);
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
            if (energy_warp) {
                if (DF) En = df_sub(En, df_mul(alpha, alpha));
                else En = df{__fmaf_rn(-alpha.hi, alpha.hi, En.hi), 0.0f};
            }

            // (a4) correlation update through the Gram matrix
            const int fam1 = (int)(j1 >= (uint32_t)n);
            const bool owner = (uint32_t)lane == j1 % (uint32_t)T;
            if (NF == 2) {
                const int f1 = (int)j1 - fam1 * n;
                const int p1 = f1 % B, q1 = f1 / B;
                const float2 *V = fam1 ? sWT : sW;
                const float2 vp = V[p1 * B + p_own];
                const df u = DF ? df_mul(alpha, df{vp.x, vp.y}) : df{__fmul_rn(alpha.hi, vp.x), 0.0f};
                const float2 *Vq = V + q1 * B;
                if (SPLIT) {
                    // the other family: rank-1 update and its new top-2; the
                    // chosen atom's own family: only its owner changes
                    if (fam1) {
                        top[0] = update_family<B, T, E, G, 0, 0, DF>(ch, cl, lane, u, Vq);
                        stale[0] = false;
                        if (owner) {
                            if (STALE && !rare) {
                                zero_slot<E, G, G>(ch, cl, (int)(j1 / (uint32_t)T) - G);
                                top[NG - 1] = stale_top2(top[NG - 1]);
                                stale[NG - 1] = (top[NG - 1].P >> 32) != 0ull;
                            } else {
                                top[NG - 1] = zero_and_rescan<T, E, G, G>(ch, cl, lane, j1);
                                stale[NG - 1] = false;
                            }
                        }
                    } else {
                        top[NG - 1] = update_family<B, T, E, G, G, n, DF>(ch, cl, lane, u, Vq);
                        stale[NG - 1] = false;
                        if (owner) {
                            if (STALE && !rare) {
                                zero_slot<E, G, 0>(ch, cl, (int)(j1 / (uint32_t)T));
                                top[0] = stale_top2(top[0]);
                                stale[0] = (top[0].P >> 32) != 0ull;
                            } else {
                                top[0] = zero_and_rescan<T, E, G, 0>(ch, cl, lane, j1);
                                stale[0] = false;
                            }
                        }
                    }
                } else {
                    Top2 nt = top2_empty();
#pragma unroll
                    for (int s = 0; s < E; ++s) {
                        const int j = lane + T * s;
                        if (FULL || j < M) {
                            const int fam = (int)(j >= n);
                            if (fam != fam1) {
                                const int q = (j - fam * n) / B;
                                const float2 w = Vq[q];
                                if (DF) {
                                    const df r = df_sub_mul(df{ch[s], cl[s]}, u, df{w.x, w.y});
                                    ch[s] = r.hi;
                                    cl[s] = r.lo;
                                } else {
                                    ch[s] = __fmaf_rn(-u.hi, w.x, ch[s]);
                                }
                            } else if ((uint32_t)j == j1) {
                                ch[s] = 0.0f;
                                cl[s] = 0.0f;
                            }
                            top2_fold(nt, ch[s], cl[s], (uint32_t)j);
                        }
                    }
                    top[0] = nt;
                }
            } else if (owner) {
                Top2 nt = top2_empty();
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int j = lane + T * s;
                    if (FULL || j < M) {
                        if ((uint32_t)j == j1) { ch[s] = 0.0f; cl[s] = 0.0f; }
                        top2_fold(nt, ch[s], cl[s], (uint32_t)j);
                    }
                }
                top[0] = nt;
            }
            ++t;
        }
        if (RESC && fallback) {
            // more candidates than the rescore takes: the exact path redoes the leaf
            if (lane == 0) {
                const unsigned slot = atomicAdd(a.fb_count, 1u);
                if (slot < a.fb_capacity) a.fb_queue[slot] = qe;
                else raise_error(a.ctr, kDevErrQueueOverflow, 5u);
                atomicAdd(&a.ctr->fallbacks[lv.level], 1u);
            }
            __syncthreads();
            continue;
        }

        // group-wide outcome of the certification
        bool tie_any;
        if (T > 32) {
            tie_any = __syncthreads_or(tie) != 0;
        } else {
            tie_any = __any_sync(0xffffffffu, tie) != 0;
        }
        // work counters: kept by the group's lane 0, added once at exit
        n_attempts += 1;
        n_steps += (unsigned long long)t;
        n_windows += (unsigned long long)windows;
        max_t = max(max_t, (unsigned)t);
        const bool emit = conv || lv.is_last;
        uint32_t off = 0, eslot = 0;
        if (emit) {
            if (lane == 0) {
                const unsigned long long slot = atomicAdd(&a.ctr->n_leaves, 1ull);
                const unsigned long long o = atomicAdd(&a.ctr->n_atoms, (unsigned long long)t);
                uint8_t flags = (uint8_t)((tie_any ? 1u : 0u) | (qe.flags & 2u));
                if (slot >= a.leaf_cap || o + t > a.atom_cap) {
                    raise_error(a.ctr, kDevErrQueueOverflow, 1u);
                    off = kNone;
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
                    eslot = (uint32_t)slot;
                    const unsigned long long cell = cell_of(a.cells, a.planes[qe.plane], qe.y, qe.x);
                    if (cell != ~0ull) a.cells.cell[cell] = (uint32_t)slot + 1u;
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
                if (lane == 0) {
                    sMisc[0] = off;
                    sMisc[1] = eslot;
                }
                __syncthreads();
                off = sMisc[0];
                eslot = sMisc[1];
            } else {
                __syncwarp();
                off = __shfl_sync(0xffffffffu, off, 0);
                eslot = __shfl_sync(0xffffffffu, eslot, 0);
            }
            if (off != kNone) {
                for (int i = lane; i < t; i += T) {
                    const StepRec st = steps[i];
                    a.atoms[off + i] = AtomRec{st.j, st.hi};
                    a.alpha_lo[off + i] = st.lo;
                    a.atom_leaf[off + i] = eslot;
                }
            }
        }
        if (T > 32) __syncthreads(); else __syncwarp();
    }
    if (T == 32) {
        // one warp per leaf: the CTA's groups add their counters in shared
        // memory first, so the exit costs three global atomics per CTA, not
        // per warp (thousands of warps finish together at the small sides)
        if (lane == 0 && n_attempts) {
            atomicAdd(&sCnt[0], n_attempts);
            atomicAdd(&sCnt[1], n_steps);
            atomicAdd(&sCnt[2], n_windows);
            atomicMax(&sMaxT, max_t);
        }
        __syncthreads();
        if (threadIdx.x == 0 && sCnt[0]) {
            atomicAdd(&a.ctr->attempts[lv.level], sCnt[0]);
            atomicAdd(&a.ctr->iterations[lv.level], sCnt[1]);
            if (sCnt[2]) atomicAdd(&a.ctr->window_steps[lv.level], sCnt[2]);
            atomicMax(&a.ctr->max_steps[lv.level], sMaxT);
        }
    } else if (lane == 0 && n_attempts) {
        atomicAdd(&a.ctr->attempts[lv.level], n_attempts);
        atomicAdd(&a.ctr->iterations[lv.level], n_steps);
        if (n_windows) atomicAdd(&a.ctr->window_steps[lv.level], n_windows);
        atomicMax(&a.ctr->max_steps[lv.level], max_t);
    }
    if (RESC && lane == 0 && n_resc) {
        atomicAdd(&a.ctr->rescored[lv.level], n_resc);
        atomicAdd(&a.ctr->resc_rounds[lv.level], n_rounds);
    }
}

template <int B, int T, int NF>
static size_t mp_smem_bytes(int k, int groups) {
    constexpr int NW = T / 32;
    size_t bytes = (NF == 2 ? 2 * B * B * sizeof(float2) : 0);
    bytes += 3 * NW * sizeof(uint4) + 12 * sizeof(uint32_t);           // partials, misc
    bytes += NW * sizeof(unsigned long long) + NW * sizeof(uint32_t);  // full-precision partials
    bytes += (size_t)groups * k * sizeof(StepRec);
    return bytes;
}

template <int B, int T, int NF, bool DF, int MINB = (T > 32 ? 1 : 2), bool RESC = false>
static cudaError_t launch_mp_t(const MPArgs &a, int num_sms, cudaStream_t st) {
    const int block = (T == 32) ? 256 : T;
    const int groups = (T == 32) ? block / 32 : 1;
    const size_t smem = mp_smem_bytes<B, T, NF>(a.lv.k, groups) +
                        (RESC ? 16 + B * B + NF * B * B * 2 + (NF * B * B + 31) / 32 * 4 + 16 * 8 + 8 * sizeof(float2) +
                                    16 * sizeof(uint32_t) + (T / 32) * sizeof(float) + 16 + 8 * B * sizeof(long long)
                              : 0);
    if (RESC && (!a.ebound || !a.Yc || !a.mu || !a.Bs || !a.Rs || !a.fb_queue || !a.fb_count))
        return cudaErrorInvalidValue;
    auto kern = mp_kernel<B, T, NF, DF, MINB, RESC>;
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

// Rank-1 update of the other family's b^2 elements, starting at element O,
// of a thread that holds a whole leaf: element (p', q') takes u[p'] W[q*][q'].
template <int B, int M, int O, bool DF>
__device__ __forceinline__ void update_other(float (&ch)[M], float (&cl)[M], const df (&u)[B], const float2 *Wq) {
#pragma unroll
    for (int f = 0; f < B * B; ++f) {
        const float2 w = Wq[f / B];
        if (DF) {
            const df r = df_sub_mul(df{ch[O + f], cl[O + f]}, u[f % B], df{w.x, w.y});
            ch[O + f] = r.hi;
            cl[O + f] = r.lo;
        } else {
            ch[O + f] = __fmaf_rn(-u[f % B].hi, w.x, ch[O + f]);
        }
    }
}

// Whether the energy lies within 2^-37 ||y||^2 of the threshold in FP64; out
// of line, so that its FP64 work runs only when the FP32 pre-test asks.
__device__ __noinline__ bool energy_in_band(df En, df thrE, uint32_t e0) {
    return fabs(df_to_double(En) - df_to_double(thrE)) < ldexp((double)e0, -37);
}

// Side 4, one thread per leaf: a side-4 leaf has only 2 b^2 = 32 correlations,
// which fit one thread's registers, so the thread runs the whole pursuit
// with no shuffle, reduction or shared-memory exchange, and each warp runs
// 32 leaves side by side.  The arithmetic per element and the decision rules
// (top-2 summary, window, full-precision decision, certification band,
// energy test) are those of mp_kernel, element for element, so the two give
// the same result bit for bit.  Emission is aggregated per warp (one atomic
// for the warp's leaf slots, one for its atoms, one for its split children)
// and the work counters per CTA.
template <int NF, bool DF>
__global__ void __launch_bounds__(128) mp_thread_kernel(MPArgs a) {
    constexpr int B = 4, n = B * B, M = NF * n;
    __shared__ float2 sW[2 * B * B];                     // W then W^T
    __shared__ unsigned long long sCnt[3];
    __shared__ unsigned sMaxT;
    extern __shared__ __align__(16) unsigned char smem[];
    StepRec *steps = reinterpret_cast<StepRec *>(smem) + (size_t)threadIdx.x * a.lv.k;

    const LevelArgs &lv = a.lv;
    if (NF == 2)
        for (int i = threadIdx.x; i < 2 * B * B; i += blockDim.x) sW[i] = i < B * B ? a.W[i] : a.WT[i - B * B];
    if (threadIdx.x < 3) sCnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) sMaxT = 0u;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const unsigned count = *lv.count;
    const int k = lv.k;
    const unsigned stride = gridDim.x * blockDim.x;
    unsigned long long n_attempts = 0, n_steps = 0, n_windows = 0;
    unsigned max_t = 0;

    for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < count; base += stride) {
        const unsigned leaf = base + (unsigned)lane;
        const bool active = leaf < count;
        int t = 0;
        bool conv = false, tie = false;
        QueueEntry qe{0u, 0u, 0u, 0u};
        if (active) {
            qe = lv.queue[leaf];
            const float tol = a.planes[qe.plane].tol;
            const df eps2 = df_scale(df_two_prod(tol, tol), (float)n);
            const uint32_t e0 = a.e0[leaf];
            df En = df_from_i64((long long)e0);
            const df thrE = df_sub(eps2, df_scale(df_from_i64((long long)e0), 0x1p-32f));
            const float bandE_f = ldexpf((float)e0, -37);
            const float eps2_f = __fmul_rn(__fmul_rn(tol, tol), (float)n);
            const float S_f = sqrtf((float)e0);
            const float pre = ldexpf(S_f, -32) * 1.05f + ldexpf(S_f, -37) * 1.05f;

            float ch[M], cl[M];
            const float2 *cp = a.c0 + (size_t)leaf * M;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float2 v = cp[j];
                ch[j] = v.x;
                cl[j] = DF ? v.y : 0.0f;
            }
            int windows = 0;
            for (;;) {
                // (a6) accuracy test before every step, strict
                const bool below = DF ? df_lt(En, thrE) : (En.hi < eps2_f);
                if (DF && fabsf(En.hi - thrE.hi) <= bandE_f * 1.01f + 0x1p-20f * fabsf(thrE.hi)) {
                    if (energy_in_band(En, thrE, e0)) tie = true;
                }
                if (below) { conv = true; break; }
                if (t == k) break;

                // (a3) argmax: the top-2 summary of all elements
                Top2 best = top2_empty();
#pragma unroll
                for (int j = 0; j < M; ++j) top2_fold(best, ch[j], cl[j], (uint32_t)j);
                if ((best.P >> 32) == 0ull) break;   // every correlation is exactly zero
                uint32_t j1 = top2_index(best);
                const float amax = top2_amax(best);
                df alpha = df{top2_negative(best) ? -amax : amax, best.lo1};
                const float window = amax * 0x1p-20f + pre;
                uint32_t cand = 0u;                       // atoms in the window, by FP32 test
                if (DF && __uint_as_float(best.k2) >= amax - window) {
#pragma unroll
                    for (int j = 0; j < M; ++j)
                        if (fabsf(ch[j]) >= amax - window) cand |= 1u << j;
                }
                if (DF && NF == 2 && cand == (1u | (1u << n)) && __float_as_uint(ch[0]) == __float_as_uint(ch[n]) &&
                    __float_as_uint(cl[0]) == __float_as_uint(cl[n])) {
                    // the DCT DC atom and the identical Haar scaling atom, alone
                    // in the window with the same value: the full-precision rule
                    // below picks index 0 and flags nothing (the two are exactly
                    // tied, 2^5 tie bands from the certification band)
                    ++windows;
                    j1 = 0u;
                    alpha = df{ch[0], cl[0]};
                } else if (cand) {
                    ++windows;
                    const double tieC = ldexp((double)S_f, -32);
                    const double bandC = ldexp((double)S_f, -37);
                    unsigned long long mk = 0ull;
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        if (fabsf(ch[j]) >= amax - window) {
                            const double m = fabs((double)ch[j] + (double)cl[j]);
                            const unsigned long long key = (unsigned long long)__double_as_longlong(m);
                            if (key > mk) mk = key;
                        }
                    }
                    const double edge = __longlong_as_double((long long)mk) - tieC;
                    uint32_t lower = kNone;
                    float wh = 0.0f, wl = 0.0f;
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        if (fabsf(ch[j]) >= amax - window) {
                            const double m = fabs((double)ch[j] + (double)cl[j]);
                            if (fabs(m - edge) < bandC) tie = true;
                            if (m >= edge && (uint32_t)j < lower) {
                                lower = (uint32_t)j;
                                wh = ch[j];
                                wl = cl[j];
                            }
                        }
                    }
                    j1 = lower;
                    alpha = df{wh, wl};
                }
                steps[t] = StepRec{j1, alpha.hi, alpha.lo};

                // (a5) energy
                if (DF) En = df_sub(En, df_mul(alpha, alpha));
                else En = df{__fmaf_rn(-alpha.hi, alpha.hi, En.hi), 0.0f};

                // (a4) the other family through W, the chosen element zeroed
                if (NF == 2) {
                    const int fam1 = (int)(j1 >= (uint32_t)n);
                    const int f1 = (int)j1 - fam1 * n;
                    const int p1 = f1 % B, q1 = f1 / B;
                    const float2 *V = sW + fam1 * B * B;
                    df u[B];
#pragma unroll
                    for (int p = 0; p < B; ++p) {
                        const float2 vp = V[p1 * B + p];
                        u[p] = DF ? df_mul(alpha, df{vp.x, vp.y}) : df{__fmul_rn(alpha.hi, vp.x), 0.0f};
                    }
                    // element (p', q') of the other family takes u[p'] W[q1][q']
                    if (fam1) update_other<B, M, 0, DF>(ch, cl, u, V + q1 * B);
                    else update_other<B, M, n, DF>(ch, cl, u, V + q1 * B);
                }
#pragma unroll
                for (int j = 0; j < M; ++j)
                    if ((uint32_t)j == j1) { ch[j] = 0.0f; cl[j] = 0.0f; }
                ++t;
            }
            n_attempts += 1;
            n_steps += (unsigned long long)t;
            n_windows += (unsigned long long)windows;
            max_t = max(max_t, (unsigned)t);
        }

        // (a7) emission and splits, aggregated over the warp
        const bool emit = active && (conv || lv.is_last);
        const bool split = active && !emit;
        const unsigned below_mask = (1u << lane) - 1u;
        const unsigned emask = __ballot_sync(0xffffffffu, emit), smask = __ballot_sync(0xffffffffu, split);
        unsigned toff = emit ? (unsigned)t : 0u;               // exclusive prefix of the emitted steps
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, toff, off);
            if (lane >= off) toff += v;
        }
        const unsigned total_t = __shfl_sync(0xffffffffu, toff, 31);
        toff -= emit ? (unsigned)t : 0u;
        unsigned long long slot0 = 0ull, off0 = 0ull;
        unsigned q0 = 0u;
        bool ok = true;
        if (lane == 0) {
            if (emask) {
                slot0 = atomicAdd(&a.ctr->n_leaves, (unsigned long long)__popc(emask));
                off0 = atomicAdd(&a.ctr->n_atoms, (unsigned long long)total_t);
                if (slot0 + __popc(emask) > a.leaf_cap || off0 + total_t > a.atom_cap) {
                    raise_error(a.ctr, kDevErrQueueOverflow, 1u);
                    ok = false;
                }
            }
            if (smask) {
                q0 = atomicAdd(lv.next_count, 4u * (unsigned)__popc(smask));
                if (q0 + 4u * (unsigned)__popc(smask) > lv.next_capacity) raise_error(a.ctr, kDevErrQueueOverflow, 2u);
            }
        }
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        off0 = __shfl_sync(0xffffffffu, off0, 0);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (emit && ok) {
            const unsigned long long slot = slot0 + (unsigned long long)__popc(emask & below_mask);
            const unsigned long long o = off0 + toff;
            const uint8_t flags = (uint8_t)((tie ? 1u : 0u) | (qe.flags & 2u));
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
            const unsigned long long cell = cell_of(a.cells, a.planes[qe.plane], qe.y, qe.x);
            if (cell != ~0ull) a.cells.cell[cell] = (uint32_t)slot + 1u;
            if (flags) atomicAdd(&a.ctr->near_tie_leaves, 1ull);
            for (int i = 0; i < t; ++i) {
                const StepRec st = steps[i];
                a.atoms[o + i] = AtomRec{st.j, st.hi};
                a.alpha_lo[o + i] = st.lo;
                a.atom_leaf[o + i] = (uint32_t)slot;
            }
        }
        if (split) {
            const unsigned qs = q0 + 4u * (unsigned)__popc(smask & below_mask);
            if (qs + 4u <= lv.next_capacity) {
                const uint32_t h = B / 2;
                const uint32_t fl = (qe.flags & 2u) | (tie ? 2u : 0u);
                lv.next_queue[qs + 0] = QueueEntry{qe.plane, qe.y, qe.x, fl};
                lv.next_queue[qs + 1] = QueueEntry{qe.plane, qe.y, qe.x + h, fl};
                lv.next_queue[qs + 2] = QueueEntry{qe.plane, qe.y + h, qe.x, fl};
                lv.next_queue[qs + 3] = QueueEntry{qe.plane, qe.y + h, qe.x + h, fl};
            }
        }
    }
    // work counters: per CTA in shared memory, then three global atomics
    if (n_attempts) {
        atomicAdd(&sCnt[0], n_attempts);
        atomicAdd(&sCnt[1], n_steps);
        atomicAdd(&sCnt[2], n_windows);
        atomicMax(&sMaxT, max_t);
    }
    __syncthreads();
    if (threadIdx.x == 0 && sCnt[0]) {
        atomicAdd(&a.ctr->attempts[lv.level], sCnt[0]);
        atomicAdd(&a.ctr->iterations[lv.level], sCnt[1]);
        if (sCnt[2]) atomicAdd(&a.ctr->window_steps[lv.level], sCnt[2]);
        atomicMax(&a.ctr->max_steps[lv.level], sMaxT);
    }
}

template <int NF, bool DF>
static cudaError_t launch_mp_thread_t(const MPArgs &a, int num_sms, cudaStream_t st) {
    constexpr int block = 128;
    const size_t smem = (size_t)block * a.lv.k * sizeof(StepRec);
    auto kern = mp_thread_kernel<NF, DF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long need = ((long long)a.lv.capacity + block - 1) / block;
    long long grid = (long long)num_sms * per_sm;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

// Threads per leaf for the two largest sides (compile-time knobs; the other
// sides use one warp per leaf).
#ifndef AQMP_MP_T32
#define AQMP_MP_T32 128
#endif
#ifndef AQMP_MP_T64
#define AQMP_MP_T64 256
#endif

// Alternate launch shapes, chosen between by the host's autotuner: other
// threads per leaf at sides 16 and 32; two resident CTAs per SM at side 64.
#ifndef AQMP_MP_T16_ALT
#define AQMP_MP_T16_ALT 64
#endif
#ifndef AQMP_MP_T32_ALT
#define AQMP_MP_T32_ALT 64
#endif

template <bool DF>
static cudaError_t launch_mp_prec(const MPArgs &a, int nf, int variant, int num_sms, cudaStream_t st) {
    const int b = a.lv.b;
    if (b == 4 && a.lv.is_last)            // every side-4 leaf is emitted: one thread per leaf
        return nf == 2 ? launch_mp_thread_t<2, DF>(a, num_sms, st) : launch_mp_thread_t<1, DF>(a, num_sms, st);
    if (nf == 2) {
        switch (b) {
            case 4: return launch_mp_t<4, 32, 2, DF>(a, num_sms, st);
            case 8: return launch_mp_t<8, 32, 2, DF>(a, num_sms, st);
            case 16:
                return variant ? launch_mp_t<16, AQMP_MP_T16_ALT, 2, DF>(a, num_sms, st)
                               : launch_mp_t<16, 32, 2, DF>(a, num_sms, st);
            case 32:
                return variant ? launch_mp_t<32, AQMP_MP_T32_ALT, 2, DF>(a, num_sms, st)
                               : launch_mp_t<32, AQMP_MP_T32, 2, DF>(a, num_sms, st);
            case 64:
                if (DF && a.ebound)
                    return variant ? launch_mp_t<64, AQMP_MP_T64, 2, true, 2, true>(a, num_sms, st)
                                   : launch_mp_t<64, AQMP_MP_T64, 2, true, 1, true>(a, num_sms, st);
                return variant ? launch_mp_t<64, AQMP_MP_T64, 2, DF, 2>(a, num_sms, st)
                               : launch_mp_t<64, AQMP_MP_T64, 2, DF>(a, num_sms, st);
            case 128: return launch_mp_cluster(a, 2, DF, num_sms, st);
        }
    } else {
        switch (b) {
            case 4: return launch_mp_t<4, 32, 1, DF>(a, num_sms, st);
            case 8: return launch_mp_t<8, 32, 1, DF>(a, num_sms, st);
            case 16: return launch_mp_t<16, 32, 1, DF>(a, num_sms, st);
            case 32: return launch_mp_t<32, AQMP_MP_T32, 1, DF>(a, num_sms, st);
            case 64:
                if (DF && a.ebound) return launch_mp_t<64, AQMP_MP_T64, 1, true, 1, true>(a, num_sms, st);
                return launch_mp_t<64, AQMP_MP_T64, 1, DF>(a, num_sms, st);
            case 128: return launch_mp_cluster(a, 1, DF, num_sms, st);
        }
    }
    return cudaErrorInvalidValue;
}

bool mp_has_variant(int b, int nf) { return nf == 2 && (b == 16 || b == 32 || b == 64); }

cudaError_t launch_mp(const MPArgs &a, int nf, bool double_float, int variant, int num_sms, cudaStream_t st) {
    return double_float ? launch_mp_prec<true>(a, nf, variant, num_sms, st)
                        : launch_mp_prec<false>(a, nf, variant, num_sms, st);
}

}  // namespace aqmp
