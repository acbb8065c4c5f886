// Plain and preconditioned L-BFGS with the Hager-Zhang line search (Sec. II:
// the preconditioned gradient P^-1 g inside a quasi-Newton method; Sec. IV.A:
// L-BFGS with m = 200 and the Hager-Zhang line search; Sec. III.B: delta).
// P is the local metric (precondition = 1, precond.cu) or the mean-field
// chi = 1 metric (precondition = 2, bp.cu).
//
// Host control, device vectors: the history pairs (s, y) live in HBM, every
// inner product is a device reduction read back as one scalar, and each
// objective evaluation is a warm-started CTMRG run plus the fixed-point
// gradient.  Readings where the paper is silent:
//   * initial inverse Hessian gamma_k P_k^-1, gamma_k = s^T y / (y^T P_k^-1 y)
//     of the newest pair (P = I when plain), gamma = 1 without history;
//   * (s, y) stored only when s^T y > 1e-16 |s| |y|;
//   * first trial step 1 with a preconditioner or history, otherwise
//     0.01 |x|_inf / |d|_inf (Hager & Zhang's I0);
//   * Hager & Zhang's bracket / update / secant^2 with delta = 0.1,
//     sigma = 0.9, epsilon = 1e-6, theta = 0.5, gamma = 0.66, rho = 5; the
//     first trial point meeting the Wolfe or approximate Wolfe conditions is
//     accepted; a trial point whose CTMRG or adjoint solve fails counts as
//     lying beyond the minimiser (value and slope +inf).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include "bp.h"
#include "common.h"
#include "ipeps_impl.h"
#include "kernels.h"

namespace ipeps {

namespace {

struct Point {
  double f = INFINITY;
  DBuf x, g;
  EnvImpl env;
  int ctm_iters = 0;
  bool ok = false;
  std::unique_ptr<BpMetric> bp;  // mean-field metric of x, built on first use
};

double ddot(int64_t n, const double *a, const double *b, cudaStream_t s) {
  DBuf r(1, s);
  dot(n, a, b, r.p, s);
  double h;
  IPEPS_CUDA(cudaMemcpyAsync(&h, r.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  IPEPS_CUDA(stream_sync(s));
  return h;
}

__global__ void absmax_kernel(int64_t n, const double *x, double *out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(x[i]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

double absmax(int64_t n, const double *x, cudaStream_t s) {
  DBuf r(1, s);
  absmax_kernel<<<1, 256, 0, s>>>(n, x, r.p);
  count_launch();
  double h;
  IPEPS_CUDA(cudaMemcpyAsync(&h, r.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  IPEPS_CUDA(stream_sync(s));
  return h;
}

struct Driver {
  Cell c;
  const HamImpl &H;
  ipeps_opts o;
  cudaStream_t s;
  int64_t n;

  // evaluate f, g at x warm-started from env0
  void evaluate(Point &p, const EnvImpl &env0) {
    p.env.cell = c;
    p.env.chi = o.chi;
    p.env.s = s;
    p.env.buf = DBuf(size_t(env0.total()), s);
    IPEPS_CUDA(cudaMemcpyAsync(p.env.buf.p, env0.buf.p, env0.total() * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    p.env.have_spectra = false;
    p.env.svd_cache.clear();
    for (auto &kv : env0.svd_cache) {
      DBuf b(kv.second.n, s);
      IPEPS_CUDA(cudaMemcpyAsync(b.p, kv.second.p, kv.second.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      p.env.svd_cache.emplace(kv.first, std::move(b));
    }
    double err = INFINITY;
    p.ctm_iters = ctmrg_run(p.env, p.x.p, o.ctm_tol, o.ctm_maxit, Prec(o.prec), &err, s);
    p.ok = err < o.ctm_tol;
    if (!p.ok) {
      p.f = INFINITY;
      return;
    }
    p.g = DBuf(size_t(n), s);
    double ares = 0.0;
    int amv = 0;
    p.f = energy_grad(c, p.x.p, p.env, H, p.g.p, s, &ares, &amv, nullptr);
    p.ok = std::isfinite(p.f) && ares < 1e-8;
    if (!p.ok) p.f = INFINITY;
  }

  void precond(Point &p, const double *v, double delta, double *out) {
    if (o.precondition == 2) {
      // the mean-field metric depends on the tensor only: one build per point
      if (!p.bp) {
        p.bp = std::make_unique<BpMetric>();
        bp_metric(c, p.x.p, kBpTol, kBpMaxit, *p.bp, s);
      }
      bp_apply(*p.bp, v, delta, out, s);
      return;
    }
    precondition_all(p.env, p.x.p, v, delta, o.krylov, o.restarts, out, s);
  }
};

}  // namespace

// One optimisation as a resumable state machine: start() evaluates the
// starting point, every step() runs one L-BFGS iteration (two-loop direction,
// Hager-Zhang line search, history update).  optimize_impl drives one run to
// its end; the server interleaves the steps of many runs.
struct LbfgsRun::Impl {
  Driver drv;
  int64_t n;
  std::unique_ptr<Point> cur;
  struct Pair { DBuf s, y; double rho; };
  std::deque<Pair> hist;
  double f_prev = NAN;
  int k = 0;
  bool done = false;
  DBuf d, q, r, tmp;
  std::chrono::steady_clock::time_point t0;
  Impl(const Cell &c, const HamImpl &H, const ipeps_opts &o, cudaStream_t s)
      : drv{c, H, o, s, int64_t(c.nsites()) * c.tsize()}, n(int64_t(c.nsites()) * c.tsize()) {}

  ipeps_iter_info info(int it, double alpha, double delta, int evals) {
    ipeps_iter_info inf{};
    inf.iter = it;
    inf.E = cur->f;
    inf.gnorm = std::sqrt(ddot(n, cur->g.p, cur->g.p, drv.s));
    inf.alpha = alpha;
    inf.delta = delta;
    inf.evals = evals;
    inf.ctm_iters = cur->ctm_iters;
    auto t1 = std::chrono::steady_clock::now();
    inf.wall_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    t0 = t1;
    return inf;
  }
};

LbfgsRun::LbfgsRun(const Cell &c, const HamImpl &H, const ipeps_opts &o, cudaStream_t s)
    : impl_(new Impl(c, H, o, s)) {}
LbfgsRun::~LbfgsRun() = default;

ipeps_iter_info LbfgsRun::start(const double *A_dev) {
  Impl &m = *impl_;
  Driver &drv = m.drv;
  const cudaStream_t s = drv.s;
  const int64_t n = m.n;
  m.t0 = std::chrono::steady_clock::now();
  m.cur = std::make_unique<Point>();
  m.cur->x = DBuf(size_t(n), s);
  IPEPS_CUDA(cudaMemcpyAsync(m.cur->x.p, A_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  {
    EnvImpl e0;
    e0.cell = drv.c;
    e0.chi = drv.o.chi;
    e0.s = s;
    e0.buf = DBuf(size_t(e0.total()), s);
    env_init(e0, m.cur->x.p, s);
    drv.evaluate(*m.cur, e0);
  }
  if (!m.cur->ok) throw Error(IPEPS_ERR_NOT_CONVERGED, "optimize: starting point did not converge");
  m.d = DBuf(size_t(n), s);
  m.q = DBuf(size_t(n), s);
  m.r = DBuf(size_t(n), s);
  m.tmp = DBuf(size_t(n), s);
  return m.info(0, 0.0, 0.0, 1);
}

bool LbfgsRun::finished() const { return impl_->done; }
int LbfgsRun::iteration() const { return impl_->k; }
double LbfgsRun::energy() const { return impl_->cur ? impl_->cur->f : NAN; }

void LbfgsRun::copy_tensor(double *A_dev) const {
  const Impl &m = *impl_;
  if (!m.cur || !m.cur->x.p) return;
  IPEPS_CUDA(cudaMemcpyAsync(A_dev, m.cur->x.p, m.n * sizeof(double), cudaMemcpyDeviceToDevice, m.drv.s));
}

bool LbfgsRun::step(ipeps_iter_info *out) {
  Impl &m = *impl_;
  if (m.done) return false;
  Driver &drv = m.drv;
  const ipeps_opts &o = drv.o;
  const cudaStream_t s = drv.s;
  const int64_t n = m.n;
  auto &cur = m.cur;
  auto &hist = m.hist;
  DBuf &d = m.d, &q = m.q, &r = m.r, &tmp = m.tmp;
  if (m.k >= o.maxiter) {
    m.done = true;
    return false;
  }
  const double gg = ddot(n, cur->g.p, cur->g.p, s);
  if (std::sqrt(gg) < o.gtol || cur->f <= o.E_target) {
    m.done = true;
    return false;
  }
  const double f_prev = m.f_prev;
  double delta = (o.delta_rule == 0 || std::isnan(f_prev)) ? std::max(gg, 1e-12)
                                                           : std::max(std::fabs(cur->f - f_prev), 1e-12);
  // ---- two-loop recursion
  IPEPS_CUDA(cudaMemcpyAsync(q.p, cur->g.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<double> alphas;
  for (auto it = hist.rbegin(); it != hist.rend(); ++it) {
    double a = it->rho * ddot(n, it->s.p, q.p, s);
    axpy(n, -a, it->y.p, q.p, s);
    alphas.push_back(a);
  }
  double gamma = 1.0;
  if (o.precondition) {
    drv.precond(*cur, q.p, delta, r.p);
    if (!hist.empty()) {
      drv.precond(*cur, hist.back().y.p, delta, tmp.p);
      gamma = ddot(n, hist.back().s.p, hist.back().y.p, s) / ddot(n, hist.back().y.p, tmp.p, s);
    }
  } else {
    IPEPS_CUDA(cudaMemcpyAsync(r.p, q.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (!hist.empty())
      gamma = ddot(n, hist.back().s.p, hist.back().y.p, s) / ddot(n, hist.back().y.p, hist.back().y.p, s);
  }
  scal(n, gamma, r.p, s);
  {
    size_t i = 0;
    for (auto it = hist.begin(); it != hist.end(); ++it, ++i) {
      double a = alphas[alphas.size() - 1 - i];
      double b = it->rho * ddot(n, it->y.p, r.p, s);
      axpy(n, a - b, it->s.p, r.p, s);
    }
  }
  axpby(n, -1.0, r.p, 0.0, d.p, s);
  double dg = ddot(n, d.p, cur->g.p, s);
  if (!(dg < 0.0)) {  // not a descent direction: restart
    hist.clear();
    if (o.precondition) drv.precond(*cur, cur->g.p, delta, r.p);
    else IPEPS_CUDA(cudaMemcpyAsync(r.p, cur->g.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    axpby(n, -1.0, r.p, 0.0, d.p, s);
    dg = ddot(n, d.p, cur->g.p, s);
  }
  double c0 = (!hist.empty() || o.precondition) ? 1.0 : 0.01 * absmax(n, cur->x.p, s) / absmax(n, d.p, s);
  // ---- Hager-Zhang line search
  const double phi0 = cur->f, dphi0 = dg;
  const double hz_delta = 0.1, hz_sigma = 0.9, hz_eps = 1e-6, hz_theta = 0.5, hz_gamma = 0.66,
               hz_rho = 5.0;
  const int max_evals = 40;
  const double fmax = phi0 + hz_eps * std::fabs(phi0);
  std::map<double, std::unique_ptr<Point>> cache;
  std::map<double, std::pair<double, double>> vals;  // a -> (phi, dphi)
  vals[0.0] = {phi0, dphi0};
  double found = -1.0;
  struct Stop {};
  int repeats = 0;  // consecutive requests of points already evaluated
  auto ev = [&](double a) -> std::pair<double, double> {
    auto it = vals.find(a);
    if (it != vals.end()) {
      // an interval shrunk to adjacent doubles keeps asking for its own ends:
      // end the search with the best point, as when the budget is spent
      if (++repeats > 50) throw Stop{};
      return it->second;
    }
    repeats = 0;
    if (int(vals.size()) > max_evals) throw Stop{};
    auto p = std::make_unique<Point>();
    p->x = DBuf(size_t(n), s);
    IPEPS_CUDA(cudaMemcpyAsync(p->x.p, cur->x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    axpy(n, a, d.p, p->x.p, s);
    drv.evaluate(*p, cur->env);
    std::pair<double, double> v{INFINITY, INFINITY};
    if (p->ok) v = {p->f, ddot(n, p->g.p, d.p, s)};
    vals[a] = v;
    cache[a] = std::move(p);
    bool t1 = (v.first - phi0 <= hz_delta * a * dphi0) && (v.second >= hz_sigma * dphi0);
    bool t2 = ((2.0 * hz_delta - 1.0) * dphi0 >= v.second) && (v.second >= hz_sigma * dphi0) &&
              (v.first <= fmax);
    if (std::isfinite(v.first) && (t1 || t2)) {
      found = a;
      throw Stop{};
    }
    return v;
  };
  auto bisect = [&](double a, double b) -> std::pair<double, double> {
    for (;;) {
      double dd = (1.0 - hz_theta) * a + hz_theta * b;
      auto v = ev(dd);
      if (v.second >= 0) return {a, dd};
      if (v.first <= fmax) a = dd;
      else b = dd;
    }
  };
  auto update = [&](double a, double b, double cc) -> std::pair<double, double> {
    if (!(a < cc && cc < b)) return {a, b};
    auto v = ev(cc);
    if (v.second >= 0) return {a, cc};
    if (v.first <= fmax) return {cc, b};
    return bisect(a, cc);
  };
  auto secant = [&](double a, double b) {
    double da = vals[a].second, db = vals[b].second;
    if (db == da || !std::isfinite(da) || !std::isfinite(db)) return 0.5 * (a + b);
    return (a * db - b * da) / (db - da);
  };
  try {
    // bracket
    double a = 0.0, b = 0.0, cc = c0, good = 0.0;
    for (;;) {
      auto v = ev(cc);
      if (v.second >= 0) { a = good; b = cc; break; }
      if (v.first > fmax) { auto ab = bisect(0.0, cc); a = ab.first; b = ab.second; break; }
      good = cc;
      cc *= hz_rho;
    }
    for (;;) {
      double cs = secant(a, b);
      auto AB = update(a, b, cs);
      if (cs == AB.second) AB = update(AB.first, AB.second, secant(b, AB.second));
      else if (cs == AB.first) AB = update(AB.first, AB.second, secant(a, AB.first));
      if (AB.second - AB.first > hz_gamma * (b - a))
        AB = update(AB.first, AB.second, 0.5 * (AB.first + AB.second));
      a = AB.first;
      b = AB.second;
    }
  } catch (Stop &) {
  }
  int nev = int(vals.size()) - 1;
  if (found < 0.0) {  // budget spent: best finite point, if any
    double bestf = INFINITY;
    for (auto &kv : vals)
      if (kv.first > 0.0 && kv.second.first < bestf) { bestf = kv.second.first; found = kv.first; }
    if (!(bestf < phi0)) {
      m.done = true;
      throw Error(IPEPS_ERR_NOT_CONVERGED, "optimize: line search found no decrease");
    }
  }
  std::unique_ptr<Point> nxt = std::move(cache[found]);
  cache.clear();
  // ---- history update
  Impl::Pair pr{DBuf(size_t(n), s), DBuf(size_t(n), s), 0.0};
  axpby(n, found, d.p, 0.0, pr.s.p, s);
  IPEPS_CUDA(cudaMemcpyAsync(pr.y.p, nxt->g.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  axpy(n, -1.0, cur->g.p, pr.y.p, s);
  double sy = ddot(n, pr.s.p, pr.y.p, s);
  double ns = std::sqrt(ddot(n, pr.s.p, pr.s.p, s)), ny = std::sqrt(ddot(n, pr.y.p, pr.y.p, s));
  if (sy > 1e-16 * ns * ny) {
    pr.rho = 1.0 / sy;
    hist.push_back(std::move(pr));
    while (int(hist.size()) > o.history) hist.pop_front();
  }
  m.f_prev = cur->f;
  cur = std::move(nxt);
  ++m.k;
  if (out) *out = m.info(m.k, found, delta, nev);
  return true;
}

ipeps_status optimize_impl(const Cell &c, double *A_dev, const HamImpl &H, const ipeps_opts &o,
                           ipeps_iter_cb cb, void *user, cudaStream_t s) {
  LbfgsRun run(c, H, o, s);
  ipeps_iter_info info = run.start(A_dev);
  auto finish = [&]() {
    run.copy_tensor(A_dev);
    IPEPS_CUDA(stream_sync(s));
  };
  if (cb && cb(&info, user)) {
    finish();
    return IPEPS_ERR_CANCELLED;
  }
  try {
    while (run.step(&info)) {
      if (cb && cb(&info, user)) {
        finish();
        return IPEPS_ERR_CANCELLED;
      }
    }
  } catch (...) {
    finish();
    throw;
  }
  finish();
  return IPEPS_OK;
}

}  // namespace ipeps
