// Tensor-core GEMM on tcgen05 (placeholder until the sm_103a kernel lands).
#include "kernels.h"

namespace ajf {

bool tc_gemm_supported(int64_t, int64_t, int64_t, int) { return false; }

cudaError_t launch_gemm_tc(char*, const int64_t*, const int64_t*, int, float*, int64_t, int64_t, int64_t, int, int*,
                           cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace ajf
