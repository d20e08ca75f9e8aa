// selftest.h -- the rounding self-test's launcher (selftest.cu).
#pragma once
#include <cuda_runtime.h>

namespace aqmp {

// int128_to_df on n caller-given integers ((lo, hi) 64-bit words each).
cudaError_t launch_round_selftest(const long long *words, long long n, float2 *out, cudaStream_t st);

}  // namespace aqmp
