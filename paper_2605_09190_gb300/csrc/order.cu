// order.cu -- the output list of Algorithm 2 in canonical order, on the device.
//
// The pursuit kernels emit leaves in the order their groups finish, and mark
// each emitted leaf (slot + 1) at its top-left min-block cell in a map laid
// out in the canonical order (planes, roots in raster order, Z-order inside
// the root = depth-first TL, TR, BL, BR).  Two launches then restore the
// encoder's list X without a sort:
//   phase 0: an exclusive scan of the cell map's occupancy ranks the leaves
//            (perm[rank] = slot);
//   phase 1: an exclusive scan of the ranked leaves' step counts gives the
//            new atom offsets; the leaf records are written in rank order;
//   phase 2: every atom moves to its leaf's new offset, one thread per atom
//            (the pursuit kernels record each atom's leaf), so that a few
//            long leaves do not serialise the copy.
// Each phase is a single-pass scan: tiles are claimed in launch order from a
// counter, publish their aggregate, and look back over their predecessors
// (decoupled look-back).  A tile only waits on tiles claimed before it, whose
// blocks are already running; every wait is bounded and reports
// AQMP_E_TIMEOUT through the counters if it ever runs out.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

constexpr int kOrderThreads = 256;
constexpr int kCellItems = 16;                               // cells per thread in phase 0
constexpr int kCellTile = kOrderThreads * kCellItems;
constexpr int kLeafTile = kOrderThreads;                     // ranks per tile in phase 1
constexpr unsigned long long kFlagAgg = 1ull << 62;          // tile aggregate published
constexpr unsigned long long kFlagIncl = 2ull << 62;         // inclusive prefix published
constexpr unsigned long long kFlagMask = 3ull << 62;

__device__ __forceinline__ unsigned long long order_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of x over the block; `total` receives the block's sum.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t x, uint32_t *s, uint32_t &total) {
    constexpr int NW = kOrderThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < NW ? s[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < NW) s[lane] = wi - w;
        if (lane == NW - 1) s[NW] = wi;
    }
    __syncthreads();
    const uint32_t r = s[warp] + incl - x;
    total = s[NW];
    return r;
}

// Publish this tile's aggregate, sum the predecessors' and publish the
// inclusive prefix; returns the exclusive prefix.  Called by warp 0, which
// inspects 32 predecessors per round: the nearest one holding an inclusive
// prefix ends the walk (before tile 0 counts as an inclusive 0).
__device__ uint32_t look_back(unsigned long long *status, unsigned long long tile, uint32_t agg, const OrderArgs &a,
                              unsigned site) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release(&status[0], kFlagIncl | agg);
        return 0u;
    }
    if (lane == 0) st_release(&status[tile], kFlagAgg | agg);
    uint32_t excl = 0;
    long long end = (long long)tile;               // this round covers [end - 32, end)
    const unsigned long long t0 = order_clock();
    for (;;) {
        const long long j = end - 1 - lane;
        const unsigned long long s = j >= 0 ? ld_acquire(&status[j]) : kFlagIncl;
        const unsigned long long f = s & kFlagMask;
        const unsigned incl = __ballot_sync(0xffffffffu, f == kFlagIncl);
        const int stop = incl ? __ffs(incl) - 1 : 31;                   // lanes [0, stop] are needed
        const unsigned need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
        if (__ballot_sync(0xffffffffu, f == 0ull) & need) {
            if (__any_sync(0xffffffffu, order_clock() - t0 > a.limit_ns)) {
                if (lane == 0) raise_error(a.ctr, kDevErrTimeout, site);
                break;
            }
            __nanosleep(32);
            continue;
        }
        excl += __reduce_add_sync(0xffffffffu, lane <= stop ? (uint32_t)s : 0u);
        if (incl) break;
        end -= 32;
    }
    if (lane == 0) st_release(&status[tile], kFlagIncl | (uint32_t)(excl + agg));
    return excl;
}

__device__ __forceinline__ unsigned long long cell_tiles(const OrderArgs &a) {
    return (a.cells.n_cells + kCellTile - 1) / kCellTile;
}

// Phase 0: rank = number of occupied cells before the leaf's cell.
__global__ void __launch_bounds__(kOrderThreads) order_rank_kernel(OrderArgs a) {
    __shared__ uint32_t s[kOrderThreads / 32 + 1];
    __shared__ unsigned long long s_tile;
    __shared__ uint32_t s_prefix;
    unsigned long long *counter = a.status;
    unsigned long long *status = a.status + 2;
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1ull);
    __syncthreads();
    const unsigned long long tile = s_tile;
    const unsigned long long n = a.cells.n_cells;
    const unsigned long long i0 = tile * kCellTile + (unsigned long long)threadIdx.x * kCellItems;
    uint32_t v[kCellItems];
    if (i0 + kCellItems <= n) {
        const uint4 *q = reinterpret_cast<const uint4 *>(a.cells.cell + i0);
#pragma unroll
        for (int k = 0; k < kCellItems / 4; ++k) {
            const uint4 t = q[k];
            v[4 * k + 0] = t.x;
            v[4 * k + 1] = t.y;
            v[4 * k + 2] = t.z;
            v[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kCellItems; ++k) v[k] = i0 + k < n ? a.cells.cell[i0 + k] : 0u;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kCellItems; ++k) cnt += v[k] != 0u;
    uint32_t total;
    const uint32_t local = block_exclusive(cnt, s, total);
    if (threadIdx.x < 32) {
        const uint32_t p = look_back(status, tile, total, a, 20u);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
    unsigned long long r = (unsigned long long)s_prefix + local;
#pragma unroll
    for (int k = 0; k < kCellItems; ++k) {
        if (v[k] != 0u) {
            if (r < a.leaf_cap) a.perm[r] = v[k] - 1u;
            ++r;
        }
    }
}

// Phase 1: new atom offsets (a scan of the ranked step counts) and the
// leaf records in canonical order.
__global__ void __launch_bounds__(kOrderThreads) order_offsets_kernel(OrderArgs a) {
    __shared__ uint32_t s[kOrderThreads / 32 + 1];
    __shared__ unsigned long long s_tile;
    __shared__ uint32_t s_prefix;
    unsigned long long *counter = a.status + 1;
    unsigned long long *status = a.status + 2 + cell_tiles(a);
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1ull);
    __syncthreads();
    const unsigned long long tile = s_tile;
    unsigned long long n = *a.n_leaves;
    if (n > a.leaf_cap) n = a.leaf_cap;
    const unsigned long long t0 = tile * kLeafTile;
    if (t0 >= n) return;        // every later tile starts further on: none waits on this one
    const unsigned long long r = t0 + threadIdx.x;
    LeafRec rec{};
    uint32_t x = 0, i = 0;
    bool ok = false;
    if (r < n) {
        i = a.perm[r];
        if (i < n) {
            rec = a.leaves_in[i];
            ok = (unsigned long long)rec.atom_off + rec.n_atoms <= a.atom_cap;
            x = ok ? rec.n_atoms : 0u;
        }
    }
    uint32_t total;
    const uint32_t local = block_exclusive(x, s, total);
    if (threadIdx.x < 32) {
        const uint32_t p = look_back(status, tile, total, a, 21u);
        if (threadIdx.x == 0) s_prefix = p;
    }
    __syncthreads();
    const unsigned long long dst = (unsigned long long)s_prefix + local;
    if (ok && dst + x <= a.atom_cap) {
        a.new_off[i] = (uint32_t)dst;
        rec.atom_off = (uint32_t)dst;
        a.out->leaves[r] = rec;
    }
}

// Phase 2: every emitted atom to its leaf's new offset (one thread per atom).
__global__ void __launch_bounds__(kOrderThreads) order_copy_kernel(OrderArgs a) {
    unsigned long long n = *a.n_atoms;
    if (n > a.atom_cap) n = a.atom_cap;
    unsigned long long nl = *a.n_leaves;
    if (nl > a.leaf_cap) nl = a.leaf_cap;
    AtomRec *atoms_out = a.out->atoms;
    float *lo_out = a.out->lo;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t slot = a.atom_leaf[k];
        if (slot >= nl) continue;
        const unsigned long long src0 = a.leaves_in[slot].atom_off;
        if (k < src0) continue;
        const unsigned long long to = (unsigned long long)a.new_off[slot] + (k - src0);
        if (to < a.atom_cap) {
            atoms_out[to] = a.atoms_in[k];
            lo_out[to] = a.lo_in[k];
        }
    }
}

unsigned long long order_status_words(unsigned long long n_cells, unsigned long long leaf_cap) {
    return 2 + (n_cells + kCellTile - 1) / kCellTile + (leaf_cap + kLeafTile - 1) / kLeafTile;
}

cudaError_t launch_order_phase(const OrderArgs &a, int phase, int num_sms, cudaStream_t st) {
    if (phase == 2) {
        unsigned long long blocks = (a.atom_cap + kOrderThreads - 1) / kOrderThreads;
        const unsigned long long most = (unsigned long long)num_sms * 8;
        if (blocks > most) blocks = most;
        if (blocks < 1) blocks = 1;
        order_copy_kernel<<<(unsigned)blocks, kOrderThreads, 0, st>>>(a);
        return cudaGetLastError();
    }
    const unsigned long long tiles = phase == 0 ? (a.cells.n_cells + kCellTile - 1) / kCellTile
                                                : (a.leaf_cap + kLeafTile - 1) / kLeafTile;
    if (tiles == 0) return cudaSuccess;
    if (tiles > 0x7fffffffull) return cudaErrorInvalidValue;
    if (phase == 0) order_rank_kernel<<<(unsigned)tiles, kOrderThreads, 0, st>>>(a);
    else order_offsets_kernel<<<(unsigned)tiles, kOrderThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace aqmp
