// Live kernel timing with CUDA events on the launching stream (enabled by
// ipeps_profile; off by default).  Each instrumented launch records an event
// pair; durations are resolved when the statistics are read.
#include <cuda_runtime.h>

#include <cstdlib>
#include <map>
#include <set>
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
std::vector<cudaEvent_t> g_free;  // recycled events (creating one per launch costs host time)

cudaEvent_t take_event() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// caller holds g_mu
void resolve(Stat &st) {
  for (auto &pr : st.pending) {
    cudaEventSynchronize(pr.second);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) st.ms += ms;
    g_free.push_back(pr.first);
    g_free.push_back(pr.second);
  }
  st.pending.clear();
}
}  // namespace

bool profiling() { return g_on; }

const char *shape_class(const char *base, int64_t M, int64_t N, int64_t K) {
  static const bool on = [] {
    const char *e = std::getenv("IPEPS_PROF_SHAPES");
    return e && e[0] == '1';
  }();
  if (!on || !g_on) return base;
  static std::mutex mu;
  static std::set<std::string> names;  // stable storage for the returned pointers
  std::lock_guard<std::mutex> lk(mu);
  std::string n = std::string(base) + "[" + std::to_string(M) + "x" + std::to_string(N) + "x" + std::to_string(K) + "]";
  return names.insert(n).first->c_str();
}

ProfScope::ProfScope(const char *name, cudaStream_t s, double flops, double bytes)
    : name_(name), s_(s), flops_(flops), bytes_(bytes) {
  if (!g_on) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s_, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;  // graph capture
  a_ = take_event();
  b_ = take_event();
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
