// Serving: many independent optimisation jobs on one GPU (continuous batching
// at the granularity of L-BFGS iterations).
//
// The paper optimises one iPEPS at a time (Sec. IV); a service that takes
// optimisation requests as they arrive keeps the device busy with several.
//   * Jobs arrive at any time (ipeps_server_submit) with their own shape, chi,
//     Hamiltonian and options; their tensors, environment, L-BFGS history and
//     tapes stay on the device from admission to the end of the run.
//   * Admission by HBM footprint: a job is admitted when the estimated device
//     memory of all admitted jobs plus its own fits the server's budget (the
//     oldest queued job first; a job larger than the whole budget runs alone).
//   * `slots` worker threads each take the admitted job whose last iteration is
//     oldest, run its next iteration on the job's own CUDA stream and put it
//     back, so the iterations of different jobs overlap on the device and a new
//     job starts as soon as memory and a slot free up.
//   * Autotuner: the first job of every (d, D, chi, cell, precision) class
//     times one CTMRG iteration with three settings of the tensor-core
//     crossover (the M N K above which a GEMM takes the BF16-digit kernel) and
//     the class keeps the fastest.
//   * Per job: the wall time of every iteration (p50 / p99), queue time, run
//     time; per server: the same over all iterations.
// A job's result does not depend on what else runs: every kernel is
// deterministic (fixed reduction orders) and each job has private buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/ipeps.h"
#include "common.h"
#include "engine.h"
#include "ipeps_impl.h"
#include "kernels.h"

namespace ipeps {

namespace {
using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * double(v.size() - 1);
  const size_t i = size_t(pos);
  const double f = pos - double(i);
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}
}  // namespace

// Device bytes one job holds while it runs: the environment, and the tapes of
// one recorded CTMRG iteration with their cotangents (per projector pair
// about 50 (chi D^2)^2 doubles: enlarged corners and their intermediates,
// half systems, four-corner product, absorption), the line search's second
// environment, and the digit packs of the largest products.
size_t job_footprint(const Cell &c, int chi) {
  const double N = double(chi) * c.D * c.D;
  const double pairs = 4.0 * c.nsites();
  const double env = 8.0 * c.nsites() * (4.0 * chi * chi + 4.0 * chi * chi * c.D * c.D);
  const double tape = 50.0 * N * N * pairs;
  const double packs = 2.0 * 16.0 / 8.0 * N * N;
  return size_t(8.0 * (tape + 3.0 * env + packs)) + (size_t(64) << 20);
}

}  // namespace ipeps

struct ipeps_server_s {
  struct Job {
    uint64_t id = 0;
    ipeps::Cell c;
    ipeps::HamImpl H;
    ipeps_opts o{};
    std::vector<double> A0, Afinal;
    size_t footprint = 0;
    int state = IPEPS_JOB_QUEUED;
    bool busy = false, cancel = false;
    int error = IPEPS_OK;
    std::string message;
    std::unique_ptr<ipeps::LbfgsRun> run;
    cudaStream_t stream = nullptr;
    double *A_dev = nullptr;
    ipeps::Clock::time_point submitted, started, last;
    double queued_ms = 0.0, run_ms = 0.0;
    std::vector<double> iter_ms;
    ipeps_iter_info info{};
    std::tuple<int, int, int, int, int, int> cls;  // (d, D, chi, Lx, Ly, prec)
  };

  ipeps_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::deque<uint64_t> queue;
  std::vector<std::thread> workers;
  std::map<std::tuple<int, int, int, int, int, int>, double> tuned;  // class -> crossover
  std::map<std::tuple<int, int, int, int, int, int>, bool> tuning;
  bool stop = false;
  size_t in_use = 0;
  uint64_t next_id = 1;
  std::vector<double> all_iter_ms;
  int done_jobs = 0;

  void admit_locked() {
    while (!queue.empty()) {
      Job &j = *jobs[queue.front()];
      if (j.cancel) {
        j.state = IPEPS_JOB_CANCELLED;
        queue.pop_front();
        continue;
      }
      const bool alone = in_use == 0;
      if (!alone && in_use + j.footprint > opts.hbm_budget_bytes) break;
      in_use += j.footprint;
      j.state = IPEPS_JOB_RUNNING;
      j.started = ipeps::Clock::now();
      j.queued_ms = std::chrono::duration<double, std::milli>(j.started - j.submitted).count();
      queue.pop_front();
    }
  }

  Job *pick_locked() {
    Job *best = nullptr;
    for (auto &kv : jobs) {
      Job &j = *kv.second;
      if (j.state != IPEPS_JOB_RUNNING || j.busy) continue;
      // a class being tuned by another worker waits for its crossover
      if (opts.autotune && !tuned.count(j.cls) && tuning.count(j.cls)) continue;
      if (!best || j.last < best->last) best = &j;
    }
    return best;
  }

  void finish_locked(Job &j, int state) {
    j.state = state;
    j.run_ms = ipeps::ms_since(j.started);
    in_use -= j.footprint;
    ++done_jobs;
  }

  // one unit of work of job j (no lock held): start, or one iteration
  void work(Job &j) {
    ipeps::PolicyScope policy(ipeps::fp64_grade_of(ipeps::Prec(j.o.prec)));
    double thr = ipeps::oz_threshold();
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = tuned.find(j.cls);
      if (it != tuned.end()) thr = it->second;
    }
    struct ThrScope {
      double old;
      explicit ThrScope(double t) : old(ipeps::oz_threshold()) { ipeps::oz_threshold() = t; }
      ~ThrScope() { ipeps::oz_threshold() = old; }
    } thr_scope(thr);
    if (!j.run) {
      IPEPS_CUDA(cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking));
      const size_t n = j.A0.size();
      j.A_dev = static_cast<double *>(ipeps::dev_alloc(n * sizeof(double), j.stream));
      IPEPS_CUDA(cudaMemcpyAsync(j.A_dev, j.A0.data(), n * sizeof(double), cudaMemcpyHostToDevice, j.stream));
      if (opts.autotune) autotune(j);
      j.run.reset(new ipeps::LbfgsRun(j.c, j.H, j.o, j.stream));
      auto t0 = ipeps::Clock::now();
      j.info = j.run->start(j.A_dev);
      j.iter_ms.push_back(ipeps::ms_since(t0));
      return;
    }
    auto t0 = ipeps::Clock::now();
    ipeps_iter_info inf{};
    if (j.run->step(&inf)) {
      j.info = inf;
      j.iter_ms.push_back(ipeps::ms_since(t0));
    }
  }

  // time one CTMRG iteration of this class at three crossovers, keep the best
  void autotune(Job &j) {
    {
      std::lock_guard<std::mutex> lk(mu);
      if (tuned.count(j.cls) || tuning.count(j.cls)) return;
      tuning[j.cls] = true;
    }
    double best_thr = ipeps::oz_threshold(), best_ms = INFINITY;
    // the class always gets a crossover, also when a timing run fails
    struct Publish {
      ipeps_server_s &srv;
      Job &j;
      double &thr;
      ~Publish() {
        std::lock_guard<std::mutex> lk(srv.mu);
        srv.tuned[j.cls] = thr;
        srv.cv.notify_all();
      }
    } publish{*this, j, best_thr};
    if (ipeps::Prec(j.o.prec) == ipeps::Prec::FP64_TC || ipeps::Prec(j.o.prec) == ipeps::Prec::BF16X3) {
      ipeps::EnvImpl e;
      e.cell = j.c;
      e.chi = j.o.chi;
      e.s = j.stream;
      e.buf = ipeps::DBuf(size_t(e.total()), j.stream);
      ipeps::env_init(e, j.A_dev, j.stream);
      double err = 0.0;
      ipeps::ctmrg_run(e, j.A_dev, 0.0, 1, ipeps::Prec(j.o.prec), &err, j.stream);  // warm-up
      for (double thr : {double(1 << 20), double(1 << 23), double(1 << 26)}) {
        ipeps::oz_threshold() = thr;
        IPEPS_CUDA(cudaStreamSynchronize(j.stream));
        auto t0 = ipeps::Clock::now();
        ipeps::ctmrg_run(e, j.A_dev, 0.0, 1, ipeps::Prec(j.o.prec), &err, j.stream);
        IPEPS_CUDA(cudaStreamSynchronize(j.stream));
        const double ms = ipeps::ms_since(t0);
        if (ms < best_ms) {
          best_ms = ms;
          best_thr = thr;
        }
      }
    }
    ipeps::oz_threshold() = best_thr;
  }

  void release(Job &j) {
    if (j.run) {
      const size_t n = j.A0.size();
      j.Afinal.assign(n, 0.0);
      try {
        j.run->copy_tensor(j.A_dev);
        cudaMemcpyAsync(j.Afinal.data(), j.A_dev, n * sizeof(double), cudaMemcpyDeviceToHost, j.stream);
        cudaStreamSynchronize(j.stream);
      } catch (...) {
      }
      j.run.reset();
    }
    if (j.A_dev) ipeps::dev_free(j.A_dev, j.stream);
    j.A_dev = nullptr;
    if (j.stream) {
      cudaStreamSynchronize(j.stream);
      cudaStreamDestroy(j.stream);
      j.stream = nullptr;
    }
  }

  void worker() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      Job *j = nullptr;
      cv.wait(lk, [&] {
        if (stop) return true;
        admit_locked();
        j = pick_locked();
        return j != nullptr;
      });
      if (stop) return;
      j->busy = true;
      const bool cancel = j->cancel;
      lk.unlock();
      int end_state = -1, err = IPEPS_OK;
      std::string msg;
      if (cancel) {
        end_state = IPEPS_JOB_CANCELLED;
      } else {
        try {
          work(*j);
          if (j->run && j->run->finished()) end_state = IPEPS_JOB_DONE;
        } catch (const ipeps::Error &e) {
          end_state = IPEPS_JOB_FAILED;
          err = e.code;
          msg = e.what();
        } catch (const std::exception &e) {
          end_state = IPEPS_JOB_FAILED;
          err = IPEPS_ERR_CUDA;
          msg = e.what();
        }
      }
      if (end_state >= 0) release(*j);
      lk.lock();
      j->busy = false;
      j->last = ipeps::Clock::now();
      if (end_state >= 0) {
        j->error = err;
        j->message = msg;
        for (double t : j->iter_ms) all_iter_ms.push_back(t);
        finish_locked(*j, end_state);
      }
      cv.notify_all();
    }
  }
};

namespace {
thread_local std::string g_serve_error;

template <class F>
ipeps_status sguard(F &&f) {
  try {
    return f();
  } catch (const ipeps::Error &e) {
    g_serve_error = e.what();
    return e.code;
  } catch (const std::exception &e) {
    g_serve_error = e.what();
    return IPEPS_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

const char *ipeps_server_last_error(void) { return g_serve_error.c_str(); }

void ipeps_server_opts_default(ipeps_server_opts *o) {
  if (!o) return;
  o->slots = 3;
  o->hbm_budget_bytes = 0;
  o->autotune = 1;
}

size_t ipeps_job_footprint(const ipeps_shape *shape, int chi) {
  if (!shape || shape->Lx < 1 || shape->Ly < 1 || shape->d < 1 || shape->D < 1 || chi < 1) return 0;
  ipeps::Cell c;
  c.Lx = shape->Lx;
  c.Ly = shape->Ly;
  c.d = shape->d;
  c.D = shape->D;
  return ipeps::job_footprint(c, chi);
}

ipeps_status ipeps_server_create(const ipeps_server_opts *opts, ipeps_server *out) {
  return sguard([&]() {
    IPEPS_REQUIRE(out, "server_create: NULL out");
    ipeps_server_opts o;
    ipeps_server_opts_default(&o);
    if (opts) o = *opts;
    IPEPS_REQUIRE(o.slots >= 1 && o.slots <= 64, "server_create: slots must be in 1 .. 64");
    auto srv = std::make_unique<ipeps_server_s>();
    IPEPS_CUDA(cudaGetDevice(&srv->device));
    if (o.hbm_budget_bytes == 0) {
      size_t free_b = 0, total_b = 0;
      IPEPS_CUDA(cudaMemGetInfo(&free_b, &total_b));
      o.hbm_budget_bytes = size_t(0.8 * double(free_b));
    }
    srv->opts = o;
    for (int i = 0; i < o.slots; ++i) srv->workers.emplace_back([p = srv.get()] { p->worker(); });
    *out = srv.release();
    return IPEPS_OK;
  });
}

ipeps_status ipeps_server_submit(ipeps_server srv, const ipeps_job_desc *desc, uint64_t *job_id) {
  return sguard([&]() {
    IPEPS_REQUIRE(srv && desc && job_id && desc->A_host && desc->ham, "server_submit: NULL argument");
    const ipeps_shape &sh = desc->shape;
    IPEPS_REQUIRE(sh.Lx >= 1 && sh.Ly >= 1 && sh.d >= 1 && sh.D >= 1 && sh.Lx <= 64 && sh.Ly <= 64 &&
                      sh.d <= 64 && sh.D <= 64,
                  "server_submit: bad shape");
    const ipeps_opts &o = desc->opts;
    IPEPS_REQUIRE(o.chi >= 1 && o.ctm_maxit >= 1 && o.history >= 0 && o.maxiter >= 0 && o.krylov >= 1 &&
                      o.restarts >= 1 && o.prec >= IPEPS_FP64 && o.prec <= IPEPS_BF16X3 &&
                      o.precondition >= 0 && o.precondition <= 2 && (o.precondition != 2 || sh.D <= 32),
                  "server_submit: bad options");
    const ipeps::HamImpl &H = desc->ham->impl;
    IPEPS_REQUIRE(H.d == sh.d, "server_submit: Hamiltonian has a different d");
    auto j = std::make_unique<ipeps_server_s::Job>();
    j->c.Lx = sh.Lx;
    j->c.Ly = sh.Ly;
    j->c.d = sh.d;
    j->c.D = sh.D;
    const size_t n = size_t(j->c.nsites()) * size_t(j->c.tsize());
    j->A0.assign(desc->A_host, desc->A_host + n);
    for (double v : j->A0) IPEPS_REQUIRE(std::isfinite(v), "server_submit: A contains NaN or Inf");
    j->H = H;
    j->o = o;
    j->footprint = ipeps::job_footprint(j->c, o.chi);
    j->cls = std::make_tuple(sh.d, sh.D, o.chi, sh.Lx, sh.Ly, int(o.prec));
    j->submitted = j->last = ipeps::Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    j->id = srv->next_id++;
    *job_id = j->id;
    srv->queue.push_back(j->id);
    srv->jobs[j->id] = std::move(j);
    srv->cv.notify_all();
    return IPEPS_OK;
  });
}

ipeps_status ipeps_server_poll(ipeps_server srv, uint64_t job_id, ipeps_job_result *res) {
  return sguard([&]() {
    IPEPS_REQUIRE(srv && res, "server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    IPEPS_REQUIRE(it != srv->jobs.end(), "server_poll: unknown job");
    const auto &j = *it->second;
    res->state = j.state;
    res->iterations = j.info.iter;
    res->E = j.info.E;
    res->gnorm = j.info.gnorm;
    res->queued_ms = j.state == IPEPS_JOB_QUEUED ? ipeps::ms_since(j.submitted) : j.queued_ms;
    res->run_ms = (j.state == IPEPS_JOB_RUNNING) ? ipeps::ms_since(j.started) : j.run_ms;
    res->iter_ms_p50 = ipeps::percentile(j.iter_ms, 0.5);
    res->iter_ms_p99 = ipeps::percentile(j.iter_ms, 0.99);
    res->footprint_bytes = j.footprint;
    res->error = j.error;
    return IPEPS_OK;
  });
}

ipeps_status ipeps_server_wait(ipeps_server srv, uint64_t job_id, double timeout_s) {
  return sguard([&]() {
    IPEPS_REQUIRE(srv, "server_wait: NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    IPEPS_REQUIRE(it != srv->jobs.end(), "server_wait: unknown job");
    auto &j = *it->second;
    const bool ok = srv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
      return j.state == IPEPS_JOB_DONE || j.state == IPEPS_JOB_FAILED || j.state == IPEPS_JOB_CANCELLED;
    });
    if (!ok) throw ipeps::Error(IPEPS_ERR_TIMEOUT, "server_wait: the job is still running");
    return IPEPS_OK;
  });
}

ipeps_status ipeps_server_cancel(ipeps_server srv, uint64_t job_id) {
  return sguard([&]() {
    IPEPS_REQUIRE(srv, "server_cancel: NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    IPEPS_REQUIRE(it != srv->jobs.end(), "server_cancel: unknown job");
    auto &j = *it->second;
    j.cancel = true;
    if (j.state == IPEPS_JOB_QUEUED) {
      srv->queue.erase(std::remove(srv->queue.begin(), srv->queue.end(), job_id), srv->queue.end());
      j.state = IPEPS_JOB_CANCELLED;
    }
    srv->cv.notify_all();
    return IPEPS_OK;
  });
}

ipeps_status ipeps_server_tensor(ipeps_server srv, uint64_t job_id, double *A_host, size_t n) {
  return sguard([&]() {
    IPEPS_REQUIRE(srv && A_host, "server_tensor: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    IPEPS_REQUIRE(it != srv->jobs.end(), "server_tensor: unknown job");
    const auto &j = *it->second;
    IPEPS_REQUIRE(j.state == IPEPS_JOB_DONE || j.state == IPEPS_JOB_CANCELLED || j.state == IPEPS_JOB_FAILED,
                  "server_tensor: the job has not ended");
    const auto &src = j.Afinal.empty() ? j.A0 : j.Afinal;
    IPEPS_REQUIRE(n >= src.size(), "server_tensor: output too small");
    std::copy(src.begin(), src.end(), A_host);
    return IPEPS_OK;
  });
}

ipeps_status ipeps_server_get_stats(ipeps_server srv, ipeps_server_stats *st) {
  return sguard([&]() {
    IPEPS_REQUIRE(srv && st, "server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    st->jobs_done = srv->done_jobs;
    st->jobs_queued = int(srv->queue.size());
    int running = 0;
    for (auto &kv : srv->jobs) running += kv.second->state == IPEPS_JOB_RUNNING;
    st->jobs_running = running;
    st->iterations = int64_t(srv->all_iter_ms.size());
    st->iter_ms_p50 = ipeps::percentile(srv->all_iter_ms, 0.5);
    st->iter_ms_p99 = ipeps::percentile(srv->all_iter_ms, 0.99);
    st->hbm_in_use_bytes = srv->in_use;
    st->hbm_budget_bytes = srv->opts.hbm_budget_bytes;
    return IPEPS_OK;
  });
}

void ipeps_server_destroy(ipeps_server srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  for (auto &t : srv->workers) t.join();
  for (auto &kv : srv->jobs) srv->release(*kv.second);
  delete srv;
}

}  // extern "C"
