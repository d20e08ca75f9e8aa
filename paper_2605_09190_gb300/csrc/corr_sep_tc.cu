// corr_sep_tc.cu -- the separable exact correlation on the tensor cores.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace aqmp {

bool corr_sep_tc_available(int, int) { return false; }

cudaError_t launch_corr_sep_tc(const CorrArgs &, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace aqmp
