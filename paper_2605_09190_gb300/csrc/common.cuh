// common.cuh -- records and constants shared by the AQMP kernels and host code.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "df.cuh"

namespace aqmp {

// The dictionary enters the correlation kernels in fixed point:
// D_fix = round(D * 2^48), an integer of at most 47 bits (|D| <= 1/2 for
// blocks of side >= 4), written as 8 balanced base-64 digits in [-32, 32].
// Every digit and every centred pixel (y - 128, in [-128, 127]) is an exact
// BF16 value, each product is at most 2^12 and a sum over K <= 4096 terms
// stays within 2^24, so an FP32 tensor-core accumulator holds it exactly.
constexpr int kFixBits = 48;
constexpr int kLimbs = 8;
constexpr int kDigitBits = 6;
constexpr int kMaxLevels = 8;          // block sides 4 .. 512 at most
constexpr int kKBlock = 64;            // K padding unit (one 128-byte BF16 row)
constexpr int kMaxSide = 128;          // largest block side this build serves

// One quadtree node waiting for its pursuit.
struct QueueEntry {
    uint32_t plane, y, x, flags;       // flags: AQMP_LEAF_NEAR_TIE_PARENT
};

// Device copy of an input plane.
struct PlaneDesc {
    const uint8_t *pix;
    long long pitch;
    int h, w;
    float tol;                         // RMSE tolerance (float, as given)
    unsigned root_off;                 // first root's slot in the level-0 queue
    unsigned roots_x;                  // roots per row
    unsigned pad;
};

// Output records (layouts match aqmp_leaf / aqmp_atom of the C ABI).
struct LeafRec {
    uint32_t plane, y, x, atom_off;
    uint16_t b, n_atoms;
    uint8_t converged, flags;
    uint16_t reserved;
};
struct AtomRec {
    uint32_t j;
    float alpha;
};

// Device counters, zeroed at the start of every encode.
struct Counters {
    unsigned long long n_leaves;
    unsigned long long n_atoms;
    unsigned long long near_tie_leaves;
    unsigned long long attempts[kMaxLevels];
    unsigned long long iterations[kMaxLevels];
    unsigned long long window_steps[kMaxLevels];   // steps decided in full precision
    unsigned int max_steps[kMaxLevels];     // longest pursuit of the level (steps)
    unsigned int queue_count[kMaxLevels + 1];
    unsigned int work_next[kMaxLevels];     // dynamic leaf assignment per level
    // BF16 form with rescore: atoms whose exact initial correlation was
    // computed, leaves handed to the exact path, and that path's queue count
    // and leaf counter
    unsigned long long rescored[kMaxLevels];
    unsigned long long resc_rounds[kMaxLevels];
    unsigned int fallbacks[kMaxLevels];
    unsigned int fb_count[kMaxLevels];
    unsigned int work_fb[kMaxLevels];
    unsigned int error;                // first AQMP_E_* code raised on the device
    unsigned int error_info;
};

// Per-level view handed to the kernels.
struct LevelArgs {
    int b, n, M, Mpad, Kpad, k, level, is_last;
    const QueueEntry *queue;           // this level's entries
    const unsigned *count;             // this level's entry count (device)
    unsigned capacity;                 // room in `queue`
    QueueEntry *next_queue;            // children go here
    unsigned *next_count;
    unsigned next_capacity;
};

// Exact fixed-point sum T = A 2^24 + B (any int64 A, B with |T| < 2^71)
// converted to double-float T 2^-48, rounded once.  The pair is first put
// in the canonical form B in [-2^23, 2^23), so the result depends only on
// T: the tensor-core and SIMT kernels, which split T differently, agree
// bit for bit.
__device__ __forceinline__ df fixed_to_df(long long A, long long B) {
    long long carry = (B + (1ll << 23)) >> 24;     // floor((B + 2^23) / 2^24)
    A += carry;
    B -= carry * (1ll << 24);
    df x = df_scale(df_from_i64(A), 0x1p-24f);
    return df_add_float(x, __ll2float_rn(B) * 0x1p-48f);
}

// Map of min-block cells in the canonical order of the output list:
// planes ascending, roots in raster order, then the Z-order (TL, TR, BL, BR
// recursively) of the cell inside its root.  The leaves of a root tile it,
// so the depth-first position of a leaf is that of its top-left cell.  The
// pursuit kernels store slot + 1 of every emitted leaf at its cell.
struct CellMap {
    uint32_t *cell;                    // n_cells words, zeroed before the encode
    unsigned long long n_cells;
    int max_block, min_block, zbits;   // zbits = 2 log2(max_block / min_block)
};

// Cell index of the block at (y, x) of plane p, or ~0 when it lies outside.
__device__ __forceinline__ unsigned long long cell_of(const CellMap &m, const PlaneDesc &p, uint32_t y, uint32_t x) {
    if (y >= (uint32_t)p.h || x >= (uint32_t)p.w) return ~0ull;
    const uint32_t mb = (uint32_t)m.max_block, nb = (uint32_t)m.min_block;
    const unsigned long long root = (unsigned long long)p.root_off + (y / mb) * p.roots_x + x / mb;
    const uint32_t cy = (y % mb) / nb, cx = (x % mb) / nb;
    uint32_t z = 0;
    for (int bit = m.zbits / 2 - 1; bit >= 0; --bit) z = (z << 2) | (((cy >> bit) & 1u) << 1) | ((cx >> bit) & 1u);
    const unsigned long long c = (root << m.zbits) | z;
    return c < m.n_cells ? c : ~0ull;
}

__device__ __forceinline__ void raise_error(Counters *ctr, unsigned code, unsigned info) {
    if (atomicCAS(&ctr->error, 0u, code) == 0u) ctr->error_info = info;
}

// Error codes raised on the device (positive; the host negates them).
constexpr unsigned kDevErrQueueOverflow = 6;
constexpr unsigned kDevErrTimeout = 7;

}  // namespace aqmp
