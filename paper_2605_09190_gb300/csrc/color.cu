// color.cu -- colour pre-processing (Section 2.3, encoder step (i)) and
// post-processing (decoder step (iii)) of the codec.
//
// The paper converts the channels to RGB or YCbCr and codes each channel on
// its own, without fixing the YCbCr variant.  This build uses the full-range
// JFIF matrix (ITU-T T.871):
//   Y  = 0.299 R + 0.587 G + 0.114 B
//   Cb = 128 - 0.168736 R - 0.331264 G + 0.5 B
//   Cr = 128 + 0.5 R - 0.418688 G - 0.081312 B
// and its inverse R = Y + 1.402 (Cr-128), G = Y - 0.344136 (Cb-128) -
// 0.714136 (Cr-128), B = Y + 1.772 (Cb-128), evaluated exactly in integers
// with each coefficient rounded to 16 fractional bits (the pairs that meet
// at 128 are chosen to sum to 2^15, so greys map to themselves and to
// Cb = Cr = 128), rounding half up, clamped to [0, 255].  Decoded planes are
// real-valued; they are rounded to the nearest integer (ties to even) and
// clamped before the inverse conversion.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

__device__ __forceinline__ uint8_t clamp_u8(int v) { return (uint8_t)min(max(v, 0), 255); }

__device__ __forceinline__ void rgb_to_ycc(int r, int g, int b, uint8_t &y, uint8_t &cb, uint8_t &cr) {
    y = clamp_u8((19595 * r + 38470 * g + 7471 * b + 32768) >> 16);
    cb = clamp_u8((-11058 * r - 21710 * g + 32768 * b + (128 << 16) + 32768) >> 16);
    cr = clamp_u8((32768 * r - 27439 * g - 5329 * b + (128 << 16) + 32768) >> 16);
}

__device__ __forceinline__ void ycc_to_rgb(int y, int cb, int cr, uint8_t &r, uint8_t &g, uint8_t &b) {
    const int db = cb - 128, dr = cr - 128;
    r = clamp_u8(y + ((91881 * dr + 32768) >> 16));
    g = clamp_u8(y + ((-22553 * db - 46802 * dr + 32768) >> 16));
    b = clamp_u8(y + ((116130 * db + 32768) >> 16));
}

__device__ __forceinline__ int round_to_u8(float v) {
    return (int)fminf(fmaxf(rintf(v), 0.0f), 255.0f);      // NaN -> 0
}

// One thread per pixel: interleaved h x w x C bytes -> C planes.
__global__ void image_to_planes_kernel(ColorArgs a) {
    const long long n = (long long)a.h * a.w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int yy = (int)(i / a.w), xx = (int)(i - (long long)yy * a.w);
        const uint8_t *px = a.img + (long long)yy * a.pitch + (long long)xx * a.channels;
        uint8_t *dst = a.planes_u8 + (long long)yy * a.plane_pitch + xx;
        const long long stride = (long long)a.h * a.plane_pitch;
        if (a.color == 2) {
            uint8_t y, cb, cr;
            rgb_to_ycc(px[0], px[1], px[2], y, cb, cr);
            dst[0] = y;
            dst[stride] = cb;
            dst[2 * stride] = cr;
        } else {
            for (int c = 0; c < a.channels; ++c) dst[c * stride] = px[c];
        }
    }
}

// One thread per pixel: C real-valued planes -> interleaved bytes.
__global__ void planes_to_image_kernel(ColorArgs a) {
    const long long n = (long long)a.h * a.w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int yy = (int)(i / a.w), xx = (int)(i - (long long)yy * a.w);
        const float *src = a.planes_f32 + (long long)yy * a.plane_pitch + xx;
        uint8_t *px = a.img_out + (long long)yy * a.pitch + (long long)xx * a.channels;
        const long long stride = (long long)a.h * a.plane_pitch;
        if (a.color == 2) {
            uint8_t r, g, b;
            ycc_to_rgb(round_to_u8(src[0]), round_to_u8(src[stride]), round_to_u8(src[2 * stride]), r, g, b);
            px[0] = r;
            px[1] = g;
            px[2] = b;
        } else {
            for (int c = 0; c < a.channels; ++c) px[c] = (uint8_t)round_to_u8(src[c * stride]);
        }
    }
}

cudaError_t launch_color(const ColorArgs &a, bool to_planes, int num_sms, cudaStream_t st) {
    const long long n = (long long)a.h * a.w;
    long long blocks = (n + 255) / 256;
    const long long most = (long long)num_sms * 16;
    if (blocks > most) blocks = most;
    if (blocks < 1) blocks = 1;
    if (to_planes) image_to_planes_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    else planes_to_image_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace aqmp
