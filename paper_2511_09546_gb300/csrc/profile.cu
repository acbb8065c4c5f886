// Live kernel timing with CUDA events on the launching stream (enabled by
// ipeps_profile; off by default).  Each instrumented launch records an event
// pair; durations are resolved when the statistics are read.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"
#include "profile.h"

namespace ipeps {

namespace {
struct Stat {
  uint64_t count = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
std::mutex g_mu;
std::map<std::string, Stat> g_stats;
bool g_on = false;

void resolve(Stat &st) {
  for (auto &pr : st.pending) {
    cudaEventSynchronize(pr.second);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) st.ms += ms;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  st.pending.clear();
}
}  // namespace

bool profiling() { return g_on; }

ProfScope::ProfScope(const char *name, cudaStream_t s, double flops, double bytes)
    : name_(name), s_(s), flops_(flops), bytes_(bytes) {
  if (!g_on) return;
  cudaEventCreate(&a_);
  cudaEventCreate(&b_);
  cudaEventRecord(a_, s_);
  active_ = true;
}

ProfScope::~ProfScope() {
  if (!active_) return;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> lk(g_mu);
  Stat &st = g_stats[name_];
  st.count += 1;
  st.flops += flops_;
  st.bytes += bytes_;
  st.pending.emplace_back(a_, b_);
  if (st.pending.size() > 4096) resolve(st);
}

void profile_enable(bool on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &kv : g_stats) resolve(kv.second);
  g_stats.clear();
  g_on = on;
}

bool profile_query(const char *name, uint64_t *count, double *ms, double *flops, double *bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_stats.find(name);
  if (it == g_stats.end()) return false;
  resolve(it->second);
  *count = it->second.count;
  *ms = it->second.ms;
  *flops = it->second.flops;
  *bytes = it->second.bytes;
  return true;
}

std::string profile_names() {
  std::lock_guard<std::mutex> lk(g_mu);
  std::string out;
  for (auto &kv : g_stats) {
    if (!out.empty()) out += ",";
    out += kv.first;
  }
  return out;
}

}  // namespace ipeps
