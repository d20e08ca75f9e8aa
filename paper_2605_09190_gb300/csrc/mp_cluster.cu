// mp_cluster.cu -- the pursuit of side-128 leaves (Section 2.2 steps (b)-(d),
// stop rule Eq. (3), split / emit of Algorithm 2) on a thread-block cluster.
//
// A side-128 leaf has M = 2 b^2 = 32 768 correlations, 256 KB as double-float
// pairs: more than one SM holds next to its working registers.  A cluster of
// C CTAs owns the leaf (C = 4 for the DCT + Haar union, 2 for one family):
// with the virtual lane v = rank T + lane, thread `lane` of CTA `rank` keeps
// the 32 elements j = v + C T s in registers -- the single-CTA kernel's
// layout over C T threads, so every CTA holds a quarter (a half) of each
// family and each step's update is spread evenly over the cluster.
//
// A step chosen from one family updates the other through the rank-1 Gram
// column W[p*, p'] W[q*, q'] (W = C H^T, or its transpose).  An element's row
// p' is lane mod b, its column q' = 2 rank + lane div b + 8 s'; so a CTA reads
// only 32 of the b columns of each table -- kept as a local slice -- and one
// row entry W[p*, p'] per thread.  The full tables (2 x 128 KB) do not fit
// one CTA; their rows are sharded over the cluster (rows 32 r .. 32 r + 31 on
// rank r), and each thread loads its row entry from the owning peer through
// distributed shared memory.
//
// Each step every warp reduces its own top-2 summary (the same summaries,
// window rule and certification as the single-CTA kernel) and stores it into
// every CTA of the cluster through distributed shared memory -- a 16-byte
// slot per warp and CTA, written by st.async, which completes its bytes on
// the receiving CTA's mbarrier -- so after one wait every CTA merges the same
// values into the same choice.  The energy, the stop test and the choice then
// run identically on every CTA, and the cluster stays in lock step with no
// further exchange.  Each step updates the other family's elements on every
// CTA and zeroes the chosen element on its owner.  Rank 0 records the steps
// and emits or splits the leaf.
//
// Every exchange wait is bounded: on expiry the CTA records AQMP_E_TIMEOUT,
// stays resident for a grace period (so that peers, which poll the error
// word while they wait, stop writing into its shared memory) and returns.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "mp_step.cuh"

namespace aqmp {

namespace {

constexpr int kCT = 256;                                  // threads per CTA
constexpr unsigned long long kExchangeWaitNs = 2000000000ull;
constexpr unsigned long long kGraceNs = 50000000ull;

__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Asynchronous 16-byte store into a peer's shared memory that completes 16
// transaction bytes on the peer's mbarrier (no release fence is needed: the
// barrier's phase completes only once the bytes have landed).
__device__ __forceinline__ void st_async_peer(uint32_t addr, uint4 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint4 pack_top2(const Top2 &t) {
    return make_uint4((uint32_t)t.P, (uint32_t)(t.P >> 32), t.k2, __float_as_uint(t.lo1));
}

__device__ __forceinline__ Top2 unpack_top2(const uint4 &v) {
    return Top2{((unsigned long long)v.y << 32) | v.x, v.z, __uint_as_float(v.w)};
}

__device__ __forceinline__ float2 ld_peer_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

// Rank-1 update of the G elements in slots [S0, S0 + G) of one family and
// their new top-2: element (v, S0 + s2) takes u W[q*, q'] with q' the slot's
// column, read from the CTA's column slice at wcol[2 s2].
template <int VT, int E, int G, int S0, int TB, bool DF>
__device__ __forceinline__ Top2 update_cols(float (&ch)[E], float (&cl)[E], int v, const df &u,
                                            const float2 *wcol) {
    Run2 acc = run2_empty();
#pragma unroll
    for (int s2 = 0; s2 < G; ++s2) {
        const int s = S0 + s2;
        const float2 w = wcol[TB * s2];
        if (DF) {
            const df r = df_sub_mul(df{ch[s], cl[s]}, u, df{w.x, w.y});
            ch[s] = r.hi;
            cl[s] = r.lo;
        } else {
            ch[s] = __fmaf_rn(-u.hi, w.x, ch[s]);
        }
        run2_fold(acc, ch[s], cl[s], (uint32_t)s);
    }
    return run2_top2<VT>(acc, v);
}

// A low word that no summary carries (a NaN pattern): marks the stop
// verdict in warp 0's step summary.
constexpr uint32_t kStopWord = 0x7fffffffu;

// Bounded wait for phase `parity` of a local mbarrier fed by peers; false on
// timeout or when another CTA has recorded an error (checked while waiting).
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, volatile unsigned *err) {
    if (try_wait_cluster(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 1;; ++it) {
        if (try_wait_cluster(bar, parity)) return true;
        if ((it & 255u) == 0u && (*err != 0u || now_ns() - t0 > kExchangeWaitNs)) return false;
    }
}

// One exchange among the C CTAs of the cluster: lane r < C of warp 0 puts
// `v` (equal on those lanes) into slot [seq & 1][rank] of CTA r with an
// asynchronous store that completes 16 bytes on that slot's mbarrier there;
// thread 0 arms its own barrier for the C * 16 bytes of the phase and waits
// (bounded) for them.  All threads call it; the leading barrier keeps a slot
// from being rewritten (two exchanges later, by a peer that needs this
// CTA's next store first) while a thread still reads it.  Returns false on
// timeout or when another CTA has recorded an error (checked only while
// waiting); the verdict is CTA-uniform.
// LEAD = false skips that barrier where the caller has one between its last
// read of the previous exchange and this call.
template <int C, bool LEAD = true>
__device__ __forceinline__ bool cluster_exchange(uint4 *xs, unsigned long long *xbar, volatile uint32_t *verdict,
                                                 int &seq, uint32_t rank, const uint4 &v,
                                                 volatile unsigned *err, const uint4 *&out) {
    const int slot = seq & 1;
    const uint32_t parity = (uint32_t)(seq >> 1) & 1u;
    ++seq;
    if (LEAD) __syncthreads();
    const uint32_t bar = sh_addr(xbar + slot);
    if (threadIdx.x < C) {
        if (threadIdx.x == 0) arrive_expect_tx(bar, (uint32_t)(C * sizeof(uint4)));
        const uint32_t r = threadIdx.x;
        st_async_peer(peer_addr(sh_addr(xs + slot * C + rank), r), v, peer_addr(bar, r));
    }
    if (threadIdx.x == 0) *verdict = wait_phase(bar, parity, err) ? 1u : 0u;
    __syncthreads();
    out = xs + slot * C;
    return *verdict != 0u;
}

}  // namespace

// NF: atom families (2: DCT + Haar on four CTAs; 1: one orthonormal family
// on two); DF as in the single-CTA kernel (double-float state and certified
// decisions, or the plain FP32 form).
template <int B, int C, int NF, bool DF>
__global__ void __launch_bounds__(kCT, 1) mp_cluster_kernel(MPArgs a) {
    constexpr int T = kCT, n = B * B, M = NF * n, VT = C * T;
    constexpr int TB = T / B, VB = VT / B;     // a thread's columns: TB rank + lane / B + VB s
    constexpr int E = M / VT;                  // 32 elements per thread
    constexpr int NG = NF, G = E / NG;         // one top-2 per family
    constexpr int NW = T / 32;
    constexpr int RS = B / C;                  // table rows held per CTA (NF == 2)
    constexpr int CS = B * T / VT;             // columns of a CTA's slice (NF == 2: 32)
    static_assert(M % VT == 0 && T % B == 0 && G * VT == n, "layout");
    static_assert(NF == 1 || (CS % TB == 0 && RS * C == B), "slices");
    static_assert(C * NW <= 32, "one warp merges every warp's summary");

    extern __shared__ __align__(16) unsigned char smem[];
    // NF == 2: column slices colV[fam table][q1][32] and row shards rowV[fam table][32][b]
    float2 *sCol = reinterpret_cast<float2 *>(smem);                    // [2][B][CS]: W, W^T
    float2 *sRow = sCol + (NF == 2 ? 2 * B * CS : 0);                   // [2][RS][B]: W, W^T
    unsigned char *p = reinterpret_cast<unsigned char *>(sRow + (NF == 2 ? 2 * RS * B : 0));
    uint4 *sXs = reinterpret_cast<uint4 *>(p);                          // [2][C][NW] step exchange
    uint4 *sX = sXs + 2 * C * NW;                                       // [2][C] other exchanges
    unsigned long long *sXbar = reinterpret_cast<unsigned long long *>(sX + 2 * C);   // [2], then [2] step
    unsigned long long *sXsbar = sXbar + 2;
    uint32_t *sMisc = reinterpret_cast<uint32_t *>(sXbar + 4);          // [16]
    unsigned long long *sRk = reinterpret_cast<unsigned long long *>(sMisc + 16);     // [NW]
    uint32_t *sRj = reinterpret_cast<uint32_t *>(sRk + NW);             // [NW]
    StepRec *steps = reinterpret_cast<StepRec *>(sRj + NW);             // [k], rank 0

    const uint32_t rank = cluster_ctarank();
    const int lane = threadIdx.x;
    const int vl = (int)rank * T + lane;       // virtual lane: element s is atom vl + VT s
    const int p_own = lane % B;                // row p' of every element of this thread
    const int hb = lane / B;                   // column q' = 2 rank + hb + 8 s'
    const LevelArgs &lv = a.lv;
    volatile unsigned *err = &a.ctr->error;
    volatile uint32_t *verdict = sMisc + 12;

    if (NF == 2) {
        for (int i = threadIdx.x; i < 2 * B * CS; i += T) {
            const int tab = i / (B * CS), r = (i / CS) % B, lc = i % CS;
            const int q = VB * (lc / TB) + TB * (int)rank + (lc % TB);
            sCol[i] = (tab ? a.WT : a.W)[r * B + q];
        }
        for (int i = threadIdx.x; i < 2 * RS * B; i += T) {
            const int tab = i / (RS * B), r = (i / B) % RS, c = i % B;
            sRow[i] = (tab ? a.WT : a.W)[((int)rank * RS + r) * B + c];
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < 4; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_addr(sXbar + s)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // every peer's tables and barriers are in place before the first remote access
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");

    const unsigned count = *lv.count;
    const int k = lv.k;
    unsigned *work = &a.ctr->work_next[lv.level];
    unsigned long long n_attempts = 0, n_steps = 0, n_windows = 0;
    unsigned max_t = 0;
    int seq = 0, sseq = 0;
    bool aborted = false;
    const int warp = lane >> 5;
    const uint4 *xr;

    for (;;) {
        uint4 claim = make_uint4(0u, 0u, 0u, 0u);
        if (rank == 0 && threadIdx.x == 0) claim.x = atomicAdd(work, 1u);
        if (threadIdx.x < 32) claim.x = __shfl_sync(0xffffffffu, claim.x, 0);   // the sending lanes
        if (!cluster_exchange<C>(sX, sXbar, verdict, seq, rank, claim, err, xr)) { aborted = true; break; }
        const unsigned leaf = xr[0].x;
        if (leaf >= count) break;

        const QueueEntry qe = lv.queue[leaf];
        const float tol = a.planes[qe.plane].tol;
        const df eps2 = df_scale(df_two_prod(tol, tol), (float)n);
        const uint32_t e0 = a.e0[leaf];
        df En = df_from_i64((long long)e0);
        const df thrE = df_sub(eps2, df_scale(df_from_i64((long long)e0), 0x1p-32f));
        const float bandE_f = ldexpf((float)e0, -37);
        const float eps2_f = __fmul_rn(__fmul_rn(tol, tol), (float)n);
        const float S_f = sqrtf((float)e0);
        const float pre = ldexpf(S_f, -32) * 1.05f + ldexpf(S_f, -37) * 1.05f;

        float ch[E], cl[E];
        Top2 top[NG];
        const float2 *cp = a.c0 + (size_t)leaf * M;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            Run2 acc = run2_empty();
#pragma unroll
            for (int s2 = 0; s2 < G; ++s2) {
                const int s = g * G + s2;
                const float2 v = cp[vl + VT * s];
                ch[s] = v.x;
                cl[s] = DF ? v.y : 0.0f;
                run2_fold(acc, ch[s], cl[s], (uint32_t)s);
            }
            top[g] = run2_top2<VT>(acc, vl);
        }

        int t = 0, windows = 0;
        bool conv = false, tie = false;
        const bool energy_warp = lane < 32;
        for (;;) {
            // (a6) accuracy test before every step, strict (identical on every CTA)
            bool below = false;
            if (energy_warp) {
                below = DF ? df_lt(En, thrE) : (En.hi < eps2_f);
                if (DF && fabsf(En.hi - thrE.hi) <= bandE_f * 1.01f + 0x1p-20f * fabsf(thrE.hi)) {
                    if (fabs(df_to_double(En) - df_to_double(thrE)) < ldexp((double)e0, -37)) tie = true;
                }
            }
            if (t == k) {
                if (lane == 0) sMisc[10] = below ? 1u : 0u;
                __syncthreads();
                conv = sMisc[10] != 0u;
                break;
            }

            // (a3) argmax: every warp's top-2 goes to every CTA of the
            // cluster (lane r < C of each warp stores it into CTA r), so
            // after one wait each CTA holds all C NW summaries and every warp
            // reduces them alike; warp 0's entry carries the stop verdict.
            Top2 best;
            {
                Top2 wb = top[0];
#pragma unroll
                for (int g = 1; g < NG; ++g) wb = top2_merge(wb, top[g]);
                wb = warp_top2(wb);
                uint4 v = pack_top2(wb);
                if (warp == 0 && below) v.w = kStopWord;
                const int ss = sseq & 1;
                const uint32_t spar = (uint32_t)(sseq >> 1) & 1u;
                ++sseq;
                const uint32_t sbar = sh_addr(sXsbar + ss);
                if (lane == 0) arrive_expect_tx(sbar, (uint32_t)(C * NW * sizeof(uint4)));
                if ((lane & 31) < C) {
                    const uint32_t r = (uint32_t)(lane & 31);
                    st_async_peer(peer_addr(sh_addr(sXs + (ss * C + (int)rank) * NW + warp), r), v,
                                  peer_addr(sbar, r));
                }
                if (lane == 0) sMisc[13 + ss] = wait_phase(sbar, spar, err) ? 1u : 0u;
                __syncthreads();
                if (sMisc[13 + ss] == 0u) { aborted = true; break; }
                const uint4 *xe = sXs + ss * C * NW;
                if (xe[rank * NW].w == kStopWord) { conv = true; break; }
                best = (lane & 31) < C * NW ? unpack_top2(xe[lane & 31]) : top2_empty();
                best = warp_top2(best);
            }
            if ((best.P >> 32) == 0ull) break;   // every correlation is exactly zero
            uint32_t j1 = top2_index(best);
            const float amax = top2_amax(best);
            df alpha = df{top2_negative(best) ? -amax : amax, best.lo1};
            const float window = amax * 0x1p-20f + pre;
            if (DF && __uint_as_float(best.k2) >= amax - window) {
                // Another atom is within the window: decide in full precision
                // over the cluster's candidates (largest magnitude, then the
                // lowest index within 2^-32 ||y|| of it; candidates within
                // 2^-37 ||y|| of that edge are not certified).
                ++windows;
                const double tieC = ldexp((double)S_f, -32);
                const double bandC = ldexp((double)S_f, -37);
                unsigned long long mk = 0ull;
                uint32_t mj = kNone;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    if (fabsf(ch[s]) >= amax - window) {
                        const double m = fabs((double)ch[s] + (double)cl[s]);
                        const unsigned long long key = (unsigned long long)__double_as_longlong(m);
                        if (key > mk) { mk = key; mj = (uint32_t)(vl + VT * s); }
                    }
                }
                warp_argmax64(mk, mj);
                if ((lane & 31) == 0) {
                    sRk[lane >> 5] = mk;
                    sRj[lane >> 5] = mj;
                }
                __syncthreads();
                mk = (lane & 31) < NW ? sRk[lane & 31] : 0ull;
                mj = (lane & 31) < NW ? sRj[lane & 31] : kNone;
                warp_argmax64(mk, mj);
                if (!cluster_exchange<C>(sX, sXbar, verdict, seq, rank,
                                         make_uint4((uint32_t)mk, (uint32_t)(mk >> 32), mj, 0u), err, xr)) {
                    aborted = true;
                    break;
                }
                {
                    const uint4 e = (lane & 31) < C ? xr[lane & 31] : make_uint4(0u, 0u, kNone, 0u);
                    mk = ((unsigned long long)e.y << 32) | e.x;
                    mj = e.z;
                    warp_argmax64(mk, mj);
                }
                const double edge = __longlong_as_double((long long)mk) - tieC;
                uint32_t lower = kNone;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    if (fabsf(ch[s]) >= amax - window) {
                        const double m = fabs((double)ch[s] + (double)cl[s]);
                        const uint32_t j = (uint32_t)(vl + VT * s);
                        if (fabs(m - edge) < bandC) tie = true;
                        if (m >= edge && j < lower) lower = j;
                    }
                }
                if (lane == 0) sMisc[6] = kNone;
                __syncthreads();
                if (lower != kNone) atomicMin(&sMisc[6], lower);
                __syncthreads();
                if (!cluster_exchange<C>(sX, sXbar, verdict, seq, rank, make_uint4(sMisc[6], 0u, 0u, 0u), err,
                                         xr)) {
                    aborted = true;
                    break;
                }
                lower = kNone;
#pragma unroll
                for (int r = 0; r < C; ++r) lower = min(lower, xr[r].x);
                // the owner of `lower` publishes its value
                if (lane == 0) sMisc[3] = 0u;
                __syncthreads();
#pragma unroll
                for (int s = 0; s < E; ++s)
                    if ((uint32_t)(vl + VT * s) == lower) {
                        sMisc[3] = 1u;
                        sMisc[4] = __float_as_uint(ch[s]);
                        sMisc[5] = __float_as_uint(cl[s]);
                    }
                __syncthreads();
                if (!cluster_exchange<C>(sX, sXbar, verdict, seq, rank, make_uint4(sMisc[3], sMisc[4], sMisc[5], 0u),
                                         err, xr)) {
                    aborted = true;
                    break;
                }
                float wh = 0.0f, wl = 0.0f;
#pragma unroll
                for (int r = 0; r < C; ++r)
                    if (xr[r].x != 0u) {
                        wh = __uint_as_float(xr[r].y);
                        wl = __uint_as_float(xr[r].z);
                    }
                j1 = lower;
                alpha = df{wh, wl};
            }
            if (rank == 0 && lane == 0) steps[t] = StepRec{j1, alpha.hi, alpha.lo};

            // (a5) energy
            if (energy_warp) {
                if (DF) En = df_sub(En, df_mul(alpha, alpha));
                else En = df{__fmaf_rn(-alpha.hi, alpha.hi, En.hi), 0.0f};
            }

            // (a4) correlation update through the Gram matrix: the other
            // family on every CTA, the chosen element on its owner
            const bool owner = j1 % (uint32_t)VT == (uint32_t)vl;
            if (NF == 2) {
                const int fam1 = (int)(j1 >= (uint32_t)n);
                const int f1 = (int)j1 - fam1 * n;
                const int p1 = f1 % B, q1 = f1 / B;
                // the table of the chosen family's steps: W for a DCT atom, W^T for a Haar atom
                const int tab = fam1;
                const uint32_t raddr = sh_addr(sRow + (size_t)tab * RS * B + (p1 % RS) * B + p_own);
                const float2 vp = ld_peer_f2(peer_addr(raddr, (uint32_t)(p1 / RS)));
                const df u = DF ? df_mul(alpha, df{vp.x, vp.y}) : df{__fmul_rn(alpha.hi, vp.x), 0.0f};
                const float2 *wcol = sCol + (size_t)tab * B * CS + q1 * CS + hb;
                if (fam1) {
                    top[0] = update_cols<VT, E, G, 0, TB, DF>(ch, cl, vl, u, wcol);
                    if (owner) top[1] = zero_and_rescan<VT, E, G, G>(ch, cl, vl, j1);
                } else {
                    top[1] = update_cols<VT, E, G, G, TB, DF>(ch, cl, vl, u, wcol);
                    if (owner) top[0] = zero_and_rescan<VT, E, G, 0>(ch, cl, vl, j1);
                }
            } else if (owner) {
                top[0] = zero_and_rescan<VT, E, G, 0>(ch, cl, vl, j1);
            }
            ++t;
        }
        if (aborted) break;

        // cluster-wide outcome of the certification
        const bool tie_cta = __syncthreads_or(tie) != 0;
        if (!cluster_exchange<C>(sX, sXbar, verdict, seq, rank, make_uint4(tie_cta ? 1u : 0u, 0u, 0u, 0u), err,
                                 xr)) {
            aborted = true;
            break;
        }
        bool tie_any = false;
#pragma unroll
        for (int r = 0; r < C; ++r) tie_any = tie_any || xr[r].x != 0u;

        if (rank == 0) {
            n_attempts += 1;
            n_steps += (unsigned long long)t;
            max_t = max(max_t, (unsigned)t);
            n_windows += (unsigned long long)windows;
            const bool emit = conv || lv.is_last;
            if (emit) {
                if (lane == 0) {
                    uint32_t off = kNone, eslot = 0;
                    const unsigned long long slot = atomicAdd(&a.ctr->n_leaves, 1ull);
                    const unsigned long long o = atomicAdd(&a.ctr->n_atoms, (unsigned long long)t);
                    const uint8_t flags = (uint8_t)((tie_any ? 1u : 0u) | (qe.flags & 2u));
                    if (slot >= a.leaf_cap || o + t > a.atom_cap) {
                        raise_error(a.ctr, kDevErrQueueOverflow, 1u);
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
                    sMisc[0] = off;
                    sMisc[1] = eslot;
                }
                __syncthreads();
                const uint32_t off = sMisc[0], eslot = sMisc[1];
                if (off != kNone) {
                    for (int i = lane; i < t; i += T) {
                        const StepRec st = steps[i];
                        a.atoms[off + i] = AtomRec{st.j, st.hi};
                        a.alpha_lo[off + i] = st.lo;
                        a.atom_leaf[off + i] = eslot;
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
        }
    }
    if (rank == 0 && lane == 0 && n_attempts) {
        atomicAdd(&a.ctr->attempts[lv.level], n_attempts);
        atomicAdd(&a.ctr->iterations[lv.level], n_steps);
        if (n_windows) atomicAdd(&a.ctr->window_steps[lv.level], n_windows);
        atomicMax(&a.ctr->max_steps[lv.level], max_t);
    }
    if (aborted && threadIdx.x == 0) {
        raise_error(a.ctr, kDevErrTimeout, 11u);
        const unsigned long long t0 = now_ns();
        while (now_ns() - t0 < kGraceNs) {
        }
    }
}

template <int B, int C, int NF, bool DF>
static cudaError_t launch_cluster_t(const MPArgs &a, int num_sms, cudaStream_t st) {
    constexpr int NW = kCT / 32, CS = B * kCT / (C * kCT), RS = B / C;
    (void)num_sms;
    // NF == 2: column slices 2 x b x CS and row shards 2 x RS x b double-float pairs
    const size_t smem = (NF == 2 ? (size_t)2 * (B * CS + RS * B) * sizeof(float2) : 0) + 2 * C * NW * sizeof(uint4) +
                        2 * C * sizeof(uint4) + 4 * sizeof(unsigned long long) + 16 * sizeof(uint32_t) +
                        NW * (sizeof(unsigned long long) + sizeof(uint32_t)) + (size_t)a.lv.k * sizeof(StepRec);
    auto kern = mp_cluster_kernel<B, C, NF, DF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kCT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    long long need = (long long)a.lv.capacity;
    if (need > clusters) need = clusters;
    if (need < 1) need = 1;
    cfg.gridDim = dim3((unsigned)(need * C), 1, 1);
    return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_mp_cluster(const MPArgs &a, int nf, bool double_float, int num_sms, cudaStream_t st) {
    if (a.lv.b == 128) {
        if (nf == 2)
            return double_float ? launch_cluster_t<128, 4, 2, true>(a, num_sms, st)
                                : launch_cluster_t<128, 4, 2, false>(a, num_sms, st);
        return double_float ? launch_cluster_t<128, 2, 1, true>(a, num_sms, st)
                            : launch_cluster_t<128, 2, 1, false>(a, num_sms, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace aqmp
