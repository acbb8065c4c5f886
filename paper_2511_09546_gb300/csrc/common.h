// Internal runtime shared by the translation units of libipeps.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ipeps.h"

namespace ipeps {

// Errors travel as exceptions inside the library and become ipeps_status at
// the C boundary.
struct Error : std::runtime_error {
  ipeps_status code;
  Error(ipeps_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define IPEPS_CUDA(call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::ipeps::Error(e_ == cudaErrorMemoryAllocation ? IPEPS_ERR_NOMEM : IPEPS_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

#define IPEPS_REQUIRE(cond, msg)                                         \
  do {                                                                   \
    if (!(cond)) throw ::ipeps::Error(IPEPS_ERR_ARG, std::string(msg)); \
  } while (0)

// Count of kernel launches issued by this thread (reported by the bench).
uint64_t &launch_counter();
inline void count_launch(uint64_t n = 1) { launch_counter() += n; }
void check_launch(const char *what);

// cudaStreamSynchronize that counts the host waits of this thread (reports)
cudaError_t stream_sync(cudaStream_t s);
uint64_t &sync_counter();

// Per-device state.  The library keeps nothing per process that belongs to
// one GPU: SM counts, kernel attributes, the memory-pool setting and the
// tensor-core error word are looked up by the calling thread's current device
// (indices below kMaxDevices), so one process may drive several devices.
constexpr int kMaxDevices = 64;
int current_device();
// SM count of the current device (queried once per device)
int device_sm_count();
// runs f() once per (current device, key), e.g. a kernel's shared-memory
// attribute; a throwing f() is retried on the next call
void once_per_device(const void *key, void (*f)(void *), void *arg);
template <class F>
void once_per_device(const void *key, F &&f) {
  once_per_device(key, [](void *a) { (*static_cast<F *>(a))(); }, static_cast<void *>(&f));
}

// Stream-ordered device allocations (the pool keeps freed blocks cached).
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// RAII device buffer of doubles.
struct DBuf {
  double *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t n_, cudaStream_t s_) : n(n_), s(s_) {
    if (n) p = static_cast<double *>(dev_alloc(n * sizeof(double), s));
  }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; s = o.s;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) dev_free(p, s);
    p = nullptr;
    n = 0;
  }
};

inline int64_t prod(const std::vector<int64_t> &d) {
  int64_t n = 1;
  for (auto v : d) n *= v;
  return n;
}

}  // namespace ipeps
