// selftest.cu -- device entry for tests of the rounding every exact
// correlation ends in (int128_to_df, sep.cuh), on caller-given integers.
#include <cuda_runtime.h>

#include "selftest.h"
#include "sep.cuh"

namespace aqmp {

namespace {
__global__ void round_selftest_kernel(const long long *__restrict__ words, long long n, float2 *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned __int128 u = ((unsigned __int128)(unsigned long long)words[2 * i + 1] << 64) |
                                    (unsigned long long)words[2 * i];
        const df c = int128_to_df((__int128)u);
        out[i] = make_float2(c.hi, c.lo);
    }
}
}  // namespace

cudaError_t launch_round_selftest(const long long *words, long long n, float2 *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    round_selftest_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(words, n, out);
    return cudaGetLastError();
}

}  // namespace aqmp
