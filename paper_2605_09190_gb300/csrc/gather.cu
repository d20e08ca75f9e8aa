// gather.cu -- (a1) block gather and the level-0 root queue.
//
// A leaf vector is the column-major unravel of its block (Appendix A:
// concatenate the columns): element v = m b + i holds pixel (row i, col m).
// The correlation kernels take it centred, y - 128, as BF16: every value in
// [-128, 127] is exact in BF16; the centring is undone exactly inside the
// correlation by adding 128 sum_v D_fix[j][v].
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

// One warp per leaf, grid-stride over the level's entries.
__global__ void gather_kernel(GatherArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned warps = (gridDim.x * blockDim.x) >> 5;
    const unsigned count = *a.count;
    for (unsigned leaf = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < count; leaf += warps) {
        const QueueEntry q = a.queue[leaf];
        const PlaneDesc pd = a.planes[q.plane];
        const uint8_t *base = pd.pix + (long long)q.y * pd.pitch + q.x;
        __nv_bfloat16 *dst = a.Y + (size_t)leaf * a.Kpad;
        uint32_t ss = 0;
        for (int v = lane; v < a.Kpad; v += 32) {
            float val = 0.0f;
            if (v < a.n) {
                const int m = v / a.b, i = v - m * a.b;
                const uint32_t p = base[(long long)i * pd.pitch + m];
                ss += p * p;
                val = (float)((int)p - 128);
            }
            dst[v] = __float2bfloat16_rn(val);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (lane == 0) a.e0[leaf] = ss;
    }
}

cudaError_t launch_gather(const GatherArgs &a, int num_sms, cudaStream_t st) {
    long long warps_needed = a.capacity;
    long long blocks = (warps_needed + 7) / 8;
    long long cap = (long long)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    gather_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// L contiguous row-major b x b blocks.
__global__ void gather_blocks_kernel(int b, int Kpad, const uint8_t *blocks, long long L,
                                     __nv_bfloat16 *Y, uint32_t *e0) {
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n = b * b;
    for (long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < L; leaf += warps) {
        const uint8_t *base = blocks + leaf * n;
        __nv_bfloat16 *dst = Y + leaf * Kpad;
        uint32_t ss = 0;
        for (int v = lane; v < Kpad; v += 32) {
            float val = 0.0f;
            if (v < n) {
                const int m = v / b, i = v - m * b;
                const uint32_t p = base[i * b + m];
                ss += p * p;
                val = (float)((int)p - 128);
            }
            dst[v] = __float2bfloat16_rn(val);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (lane == 0 && e0) e0[leaf] = ss;
    }
}

cudaError_t launch_gather_blocks(int b, int Kpad, const uint8_t *blocks, long long L,
                                 __nv_bfloat16 *Y, uint32_t *e0, int num_sms, cudaStream_t st) {
    long long blocks_needed = (L + 7) / 8;
    long long cap = (long long)num_sms * 8;
    if (blocks_needed > cap) blocks_needed = cap;
    if (blocks_needed < 1) blocks_needed = 1;
    gather_blocks_kernel<<<(unsigned)blocks_needed, 256, 0, st>>>(b, Kpad, blocks, L, Y, e0);
    return cudaGetLastError();
}

// Roots of every plane in row-major order (Algorithm 1 loops over channels;
// Algorithm 2 starts from the N_max blocks of each).
__global__ void seed_roots_kernel(const PlaneDesc *planes, int n_planes, int max_block,
                                  unsigned total, QueueEntry *queue, unsigned *count) {
    for (unsigned r = blockIdx.x * blockDim.x + threadIdx.x; r < total; r += gridDim.x * blockDim.x) {
        int p = 0;
        while (p + 1 < n_planes && planes[p + 1].root_off <= r) ++p;
        const unsigned local = r - planes[p].root_off;
        const unsigned ry = local / planes[p].roots_x, rx = local - ry * planes[p].roots_x;
        queue[r] = QueueEntry{(uint32_t)p, ry * (uint32_t)max_block, rx * (uint32_t)max_block, 0u};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = total;
}

cudaError_t launch_seed_roots(const PlaneDesc *planes, int n_planes, int max_block,
                              unsigned total_roots, QueueEntry *queue, unsigned *count,
                              cudaStream_t st) {
    unsigned blocks = (total_roots + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    seed_roots_kernel<<<blocks, 256, 0, st>>>(planes, n_planes, max_block, total_roots, queue, count);
    return cudaGetLastError();
}

}  // namespace aqmp
