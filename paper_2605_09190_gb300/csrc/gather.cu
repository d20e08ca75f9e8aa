// gather.cu -- (a1) block gather and the level-0 root queue.
//
// A leaf vector is the column-major unravel of its block (Appendix A:
// concatenate the columns): element v = m b + i holds pixel (row i, col m).
// The correlation kernels take it centred, y - 128, as BF16: every value in
// [-128, 127] is exact in BF16; the centring is undone exactly inside the
// correlation by adding 128 sum_v D_fix[j][v].  The BF16 form with rescore
// centres on the block's mean rounded to an integer instead (values in
// [-255, 255], still exact in BF16), recorded per leaf.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

// TPL threads per leaf (a warp below side 32, the whole 256-thread CTA at
// sides 32 to 128), grid-stride over the level's entries.  The block's rows
// are read coalesced into the group's shared-memory tile (row stride B + 4
// bytes), then written in unravel order v = m B + i as BF16 pairs, so both
// the pixel reads and the BF16 writes are contiguous.
template <int B, int TPL>
__global__ void __launch_bounds__(256) gather_kernel(GatherArgs a) {
    constexpr int n = B * B, stride = B + 4, GROUPS = 256 / TPL, NW = TPL / 32;
    extern __shared__ uint8_t gather_tile[];
    __shared__ uint32_t s_ss[8];
    const int t = threadIdx.x % TPL, g = threadIdx.x / TPL, lane = threadIdx.x & 31;
    uint8_t *tile = gather_tile + (size_t)g * B * stride;
    const unsigned count = *a.count;
    for (unsigned leaf = blockIdx.x * GROUPS + g; leaf < count; leaf += gridDim.x * GROUPS) {
        const QueueEntry q = a.queue[leaf];
        const PlaneDesc pd = a.planes[q.plane];
        const uint8_t *base = pd.pix + (long long)q.y * pd.pitch + q.x;
        uint32_t ss = 0, sy = 0;
#pragma unroll 4
        for (int idx = t; idx < n; idx += TPL) {               // rows, coalesced
            const int i = idx / B, m = idx % B;
            const uint32_t p = base[(long long)i * pd.pitch + m];
            ss += p * p;
            sy += p;
            tile[i * stride + m] = (uint8_t)p;
        }
        if (TPL == 32) __syncwarp(); else __syncthreads();
        // the centre: 128, or (BF16 form with rescore) the block's mean
        // rounded to an integer, so that y - centre stays exact in BF16
        int centre = 128;
        if (a.mu) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sy += __shfl_xor_sync(0xffffffffu, sy, off);
            if (NW > 1) {
                if (lane == 0) s_ss[threadIdx.x >> 5] = sy;
                __syncthreads();
                sy = 0;
                for (int w = 0; w < NW; ++w) sy += s_ss[w];
                __syncthreads();
            }
            centre = (int)((sy + (uint32_t)(n / 2)) / (uint32_t)n);
            if (t == 0) a.mu[leaf] = (uint8_t)centre;
        }
        if (a.Y8) {
            // FP8 form: centred pixels times the block's power-of-two scale
            // s_l (the largest with max |y~| s_l <= 448), rounded to E4M3
            uint32_t amax = 0;
            for (int idx = t; idx < n; idx += TPL) {
                const int d = (int)tile[(idx / B) * stride + idx % B] - 128;
                amax = max(amax, (uint32_t)(d < 0 ? -d : d));
            }
            for (int off = 16; off > 0; off >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, off));
            if (NW > 1) {
                if (lane == 0) s_ss[threadIdx.x >> 5] = amax;
                __syncthreads();
                amax = 0;
                for (int w = 0; w < NW; ++w) amax = max(amax, s_ss[w]);
                __syncthreads();
            }
            int ex = 0;
            while (amax > 0 && ((unsigned long long)amax << (ex + 1)) <= 448ull) ++ex;
            const float sl = (float)(1 << ex);
            const int K8 = kpad_fp8(n);
            uint8_t *dst8 = a.Y8 + (size_t)leaf * K8;
            for (int v = t; v < K8; v += TPL) {
                __nv_fp8_storage_t q8 = 0;
                if (v < n)
                    q8 = __nv_cvt_float_to_fp8((float)((int)tile[(v % B) * stride + v / B] - 128) * sl,
                                               __NV_SATFINITE, __NV_E4M3);
                dst8[v] = q8;
            }
            if (t == 0) a.inv_sl[leaf] = 1.0f / sl;
        } else {
            __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(a.Y + (size_t)leaf * a.Kpad);
            for (int v = 2 * t; v < a.Kpad; v += 2 * TPL) {      // unravel order, BF16 pairs
                float v0 = 0.0f, v1 = 0.0f;
                if (v < n) v0 = (float)((int)tile[(v % B) * stride + v / B] - centre);
                if (v + 1 < n) v1 = (float)((int)tile[((v + 1) % B) * stride + (v + 1) / B] - centre);
                dst[v >> 1] = __floats2bfloat162_rn(v0, v1);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (NW == 1) {
            if (lane == 0) a.e0[leaf] = ss;
            __syncwarp();
        } else {
            if (lane == 0) s_ss[threadIdx.x >> 5] = ss;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t tot = 0;
                for (int w = 0; w < NW; ++w) tot += s_ss[w];
                a.e0[leaf] = tot;
            }
            __syncthreads();
        }
    }
}

template <int B>
static cudaError_t launch_gather_t(const GatherArgs &a, int num_sms, cudaStream_t st) {
    constexpr int TPL = B >= 32 ? 256 : 32;
    constexpr int GROUPS = 256 / TPL;
    long long blocks = ((long long)a.capacity + GROUPS - 1) / GROUPS;
    const long long cap = (long long)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const size_t smem = (size_t)GROUPS * B * (B + 4);
    gather_kernel<B, TPL><<<(unsigned)blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather(const GatherArgs &a, int num_sms, cudaStream_t st) {
    switch (a.b) {
        case 4: return launch_gather_t<4>(a, num_sms, st);
        case 8: return launch_gather_t<8>(a, num_sms, st);
        case 16: return launch_gather_t<16>(a, num_sms, st);
        case 32: return launch_gather_t<32>(a, num_sms, st);
        case 64: return launch_gather_t<64>(a, num_sms, st);
        case 128: return launch_gather_t<128>(a, num_sms, st);
    }
    return cudaErrorInvalidValue;
}

// L contiguous row-major b x b blocks (centred on 128, or with `mu` on each
// block's integer mean, recorded in mu[leaf]).
__global__ void gather_blocks_kernel(int b, int Kpad, const uint8_t *blocks, long long L,
                                     __nv_bfloat16 *Y, uint32_t *e0, uint8_t *mu) {
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n = b * b;
    for (long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < L; leaf += warps) {
        const uint8_t *base = blocks + leaf * n;
        __nv_bfloat16 *dst = Y + leaf * Kpad;
        int centre = 128;
        if (mu) {
            uint32_t sy = 0;
            for (int v = lane; v < n; v += 32) sy += base[v];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sy += __shfl_xor_sync(0xffffffffu, sy, off);
            centre = (int)((sy + (uint32_t)(n / 2)) / (uint32_t)n);
            if (lane == 0) mu[leaf] = (uint8_t)centre;
        }
        uint32_t ss = 0;
        for (int v = lane; v < Kpad; v += 32) {
            float val = 0.0f;
            if (v < n) {
                const int m = v / b, i = v - m * b;
                const uint32_t p = base[i * b + m];
                ss += p * p;
                val = (float)((int)p - centre);
            }
            dst[v] = __float2bfloat16_rn(val);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (lane == 0 && e0) e0[leaf] = ss;
    }
}

cudaError_t launch_gather_blocks(int b, int Kpad, const uint8_t *blocks, long long L,
                                 __nv_bfloat16 *Y, uint32_t *e0, int num_sms, cudaStream_t st, uint8_t *mu) {
    long long blocks_needed = (L + 7) / 8;
    long long cap = (long long)num_sms * 8;
    if (blocks_needed > cap) blocks_needed = cap;
    if (blocks_needed < 1) blocks_needed = 1;
    gather_blocks_kernel<<<(unsigned)blocks_needed, 256, 0, st>>>(b, Kpad, blocks, L, Y, e0, mu);
    return cudaGetLastError();
}

// The same for the FP8 form: e4m3(y~ s_l) with the block's power-of-two
// scale s_l (max |y~| s_l <= 448), zero padded to kpad_fp8(n), and 1 / s_l.
__global__ void gather_blocks_fp8_kernel(int b, const uint8_t *blocks, long long L, uint8_t *Y8, float *inv_sl) {
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n = b * b, K8 = kpad_fp8(n);
    for (long long leaf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; leaf < L; leaf += warps) {
        const uint8_t *base = blocks + leaf * n;
        uint32_t amax = 0;
        for (int v = lane; v < n; v += 32) {
            const int d = (int)base[v] - 128;
            amax = max(amax, (uint32_t)(d < 0 ? -d : d));
        }
        for (int off = 16; off > 0; off >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        int ex = 0;
        while (amax > 0 && ((unsigned long long)amax << (ex + 1)) <= 448ull) ++ex;
        const float sl = (float)(1 << ex);
        for (int v = lane; v < K8; v += 32) {
            __nv_fp8_storage_t q8 = 0;
            if (v < n) {
                const int m = v / b, i = v - m * b;
                q8 = __nv_cvt_float_to_fp8((float)((int)base[i * b + m] - 128) * sl, __NV_SATFINITE, __NV_E4M3);
            }
            Y8[leaf * K8 + v] = q8;
        }
        if (lane == 0) inv_sl[leaf] = 1.0f / sl;
    }
}

cudaError_t launch_gather_blocks_fp8(int b, const uint8_t *blocks, long long L, uint8_t *Y8, float *inv_sl,
                                     int num_sms, cudaStream_t st) {
    long long blocks_needed = (L + 7) / 8;
    long long cap = (long long)num_sms * 8;
    if (blocks_needed > cap) blocks_needed = cap;
    if (blocks_needed < 1) blocks_needed = 1;
    gather_blocks_fp8_kernel<<<(unsigned)blocks_needed, 256, 0, st>>>(b, blocks, L, Y8, inv_sl);
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
