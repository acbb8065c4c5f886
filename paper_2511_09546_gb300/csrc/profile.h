// Live per-kernel timing (CUDA events on the launching stream).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

namespace ipeps {

bool profiling();
void profile_enable(bool on);
bool profile_query(const char *name, uint64_t *count, double *ms, double *flops, double *bytes);
std::string profile_names();
// With IPEPS_PROF_SHAPES=1 in the environment, a persistent class name
// "<base>[MxNxK]" per GEMM shape (shape histogram of a run); otherwise base.
const char *shape_class(const char *base, int64_t M, int64_t N, int64_t K);

// Records an event pair around the launches issued in its scope when
// profiling is on; flops and bytes are the algorithmic work of the scope.
class ProfScope {
 public:
  ProfScope(const char *name, cudaStream_t s, double flops, double bytes);
  ~ProfScope();
  ProfScope(const ProfScope &) = delete;
  ProfScope &operator=(const ProfScope &) = delete;

 private:
  const char *name_;
  cudaStream_t s_;
  double flops_, bytes_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool active_ = false;
};

}  // namespace ipeps
