// 3xTF32 tensor-core GEMM (tcgen05) -- placeholder until the kernel lands.
#include "common.h"
#include "engine.h"

namespace ipeps {
void gemm_tf32x3(bool, bool, int64_t, int64_t, int64_t, double, const double *, int64_t, const double *,
                 int64_t, double, double *, int64_t, cudaStream_t) {
  throw Error(IPEPS_ERR_ARG, "3xTF32 tensor-core GEMM is not available in this build");
}
}  // namespace ipeps
