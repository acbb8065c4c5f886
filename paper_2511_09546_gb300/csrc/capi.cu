// C ABI of libipeps (include/ipeps.h): argument checks, error translation and
// the runtime helpers shared by the translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <set>
#include <mutex>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "../../include/ipeps.h"
#include "bp.h"
#include "common.h"
#include "ipeps_impl.h"
#include "kernels.h"
#include "profile.h"
#include "engine.h"


namespace ipeps {

ipeps_status optimize_impl(const Cell &c, double *A_dev, const HamImpl &H, const ipeps_opts &o,
                           ipeps_iter_cb cb, void *user, cudaStream_t s);

uint64_t &launch_counter() {
  static thread_local uint64_t n = 0;
  return n;
}

uint64_t &sync_counter() {
  static thread_local uint64_t n = 0;
  return n;
}

cudaError_t stream_sync(cudaStream_t s) {
  ++sync_counter();
  return cudaStreamSynchronize(s);
}

void check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(IPEPS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int current_device() {
  int d = 0;
  IPEPS_CUDA(cudaGetDevice(&d));
  IPEPS_REQUIRE(d >= 0 && d < kMaxDevices, "device index above the library's limit of 64");
  return d;
}

int device_sm_count() {
  static std::atomic<int> sms[kMaxDevices];  // zero-initialised
  const int d = current_device();
  int v = sms[d].load(std::memory_order_relaxed);
  if (!v) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    sms[d].store(v, std::memory_order_relaxed);
  }
  return v;
}

void once_per_device(const void *key, void (*f)(void *), void *arg) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  const int d = current_device();
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({d, key})) return;
  f(arg);
  done.insert({d, key});
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
  // keep freed blocks in the current device's pool (its release threshold)
  static std::atomic<bool> pool_ready[kMaxDevices];
  const int dev = current_device();
  if (!pool_ready[dev].load(std::memory_order_acquire)) {
    once_per_device(&pool_ready, [dev]() {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      cudaGetLastError();
    });
    pool_ready[dev].store(true, std::memory_order_release);
  }
  void *p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(IPEPS_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  return p;
}

void dev_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

}  // namespace ipeps

namespace {
thread_local std::string g_last_error;

template <class F>
ipeps_status guarded(F &&f) {
  try {
    return f();
  } catch (const ipeps::Error &e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return IPEPS_ERR_CUDA;
  }
}

ipeps::Cell cell_of(const ipeps_shape *sh) {
  IPEPS_REQUIRE(sh, "shape is NULL");
  IPEPS_REQUIRE(sh->Lx >= 1 && sh->Ly >= 1 && sh->d >= 1 && sh->D >= 1, "shape fields must be >= 1");
  IPEPS_REQUIRE(sh->Lx <= 64 && sh->Ly <= 64 && sh->d <= 64 && sh->D <= 64, "shape too large");
  ipeps::Cell c;
  c.Lx = sh->Lx;
  c.Ly = sh->Ly;
  c.d = sh->d;
  c.D = sh->D;
  return c;
}

void check_finite(const double *p, int64_t n, cudaStream_t s, const char *what) {
  int *cnt = static_cast<int *>(ipeps::dev_alloc(sizeof(int), s));
  ipeps::count_nonfinite(n, p, cnt, s);
  int h = 0;
  cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  ipeps::dev_free(cnt, s);
  if (h) throw ipeps::Error(IPEPS_ERR_NONFINITE, std::string(what) + " contains NaN or Inf");
}

void check_env(ipeps_env env, const ipeps::Cell &c) {
  IPEPS_REQUIRE(env, "env is NULL");
  const auto &e = env->impl;
  IPEPS_REQUIRE(e.cell.Lx == c.Lx && e.cell.Ly == c.Ly && e.cell.d == c.d && e.cell.D == c.D,
                "env was built for a different shape");
}

void kron4(const double *a, const double *b, const double *c, const double *d, double *out) {
  // out = a (x) b (x) c (x) d, all 2 x 2
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 16; ++j) {
      int i0 = (i >> 3) & 1, i1 = (i >> 2) & 1, i2 = (i >> 1) & 1, i3 = i & 1;
      int j0 = (j >> 3) & 1, j1 = (j >> 2) & 1, j2 = (j >> 1) & 1, j3 = j & 1;
      out[i * 16 + j] = a[i0 * 2 + j0] * b[i1 * 2 + j1] * c[i2 * 2 + j2] * d[i3 * 2 + j3];
    }
}
}  // namespace

extern "C" {

const char *ipeps_last_error(void) { return g_last_error.c_str(); }

void ipeps_profile(int enable) { ipeps::profile_enable(enable != 0); }

int ipeps_profile_query(const char *name, uint64_t *count, double *ms, double *flops, double *bytes) {
  if (!name || !count || !ms || !flops || !bytes) return 0;
  return ipeps::profile_query(name, count, ms, flops, bytes) ? 1 : 0;
}

const char *ipeps_profile_names(void) {
  static thread_local std::string names;
  names = ipeps::profile_names();
  return names.c_str();
}

uint64_t ipeps_launch_count(int reset) {
  uint64_t n = ipeps::launch_counter();
  if (reset) ipeps::launch_counter() = 0;
  return n;
}

uint64_t ipeps_sync_count(int reset) {
  uint64_t n = ipeps::sync_counter();
  if (reset) ipeps::sync_counter() = 0;
  return n;
}

ipeps_status ipeps_ham_create(int d, const double *h_h, const double *h_v, const double *h_site,
                              double scale, ipeps_ham *out) {
  return guarded([&]() {
    IPEPS_REQUIRE(out && h_h && h_v && d >= 1 && d <= 64, "ham_create: bad arguments");
    auto H = std::make_unique<ipeps_ham_s>();
    H->impl.d = d;
    H->impl.scale = scale;
    size_t n2 = size_t(d) * d * d * d;
    H->impl.h.assign(h_h, h_h + n2);
    H->impl.v.assign(h_v, h_v + n2);
    if (h_site) {
      H->impl.site.assign(h_site, h_site + size_t(d) * d);
      H->impl.has_site = true;
    }
    for (double x : H->impl.h) IPEPS_REQUIRE(std::isfinite(x), "ham_create: non-finite h");
    for (double x : H->impl.v) IPEPS_REQUIRE(std::isfinite(x), "ham_create: non-finite v");
    *out = H.release();
    return IPEPS_OK;
  });
}

ipeps_status ipeps_ham_set_nnn(ipeps_ham ham, const double *h_d1, const double *h_d2) {
  return guarded([&]() {
    IPEPS_REQUIRE(ham, "ham_set_nnn: NULL Hamiltonian");
    const int d = ham->impl.d;
    const size_t n2 = size_t(d) * d * d * d;
    ham->impl.has_d1 = h_d1 != nullptr;
    ham->impl.has_d2 = h_d2 != nullptr;
    if (h_d1) ham->impl.d1.assign(h_d1, h_d1 + n2);
    else ham->impl.d1.clear();
    if (h_d2) ham->impl.d2.assign(h_d2, h_d2 + n2);
    else ham->impl.d2.clear();
    for (double x : ham->impl.d1) IPEPS_REQUIRE(std::isfinite(x), "ham_set_nnn: non-finite d1");
    for (double x : ham->impl.d2) IPEPS_REQUIRE(std::isfinite(x), "ham_set_nnn: non-finite d2");
    return IPEPS_OK;
  });
}

ipeps_status ipeps_ham_heisenberg(int rotated, double J, ipeps_ham *out) {
  // S.S in the basis |00>,|01>,|10>,|11> (0 = up): 1/4 on the aligned states,
  // -1/4 and the 1/2 exchange on the anti-aligned ones.  The rotated bond
  // (second spin turned by i sigma_y: S^x -> -S^x, S^z -> -S^z) is
  // -SxSx + SySy - SzSz.
  double h[16] = {0};
  if (!rotated) {
    h[0] = 0.25; h[15] = 0.25;
    h[5] = -0.25; h[10] = -0.25;
    h[6] = 0.5; h[9] = 0.5;
  } else {
    h[0] = -0.25; h[15] = -0.25;
    h[5] = 0.25; h[10] = 0.25;
    h[3] = -0.5; h[12] = -0.5;
  }
  for (double &x : h) x *= J;
  return ipeps_ham_create(2, h, h, nullptr, 1.0, out);
}

ipeps_status ipeps_ham_j1j2(int rotated, double J1, double J2, ipeps_ham *out) {
  // J1 S.S on nearest neighbours (sublattice-rotated when rotated != 0) and
  // J2 S.S on both plaquette diagonals, never rotated: diagonal neighbours sit
  // on the same sublattice
  return guarded([&]() {
    IPEPS_REQUIRE(out && std::isfinite(J1) && std::isfinite(J2), "ham_j1j2: bad arguments");
    ipeps_ham h = nullptr;
    ipeps_status st = ipeps_ham_heisenberg(rotated, J1, &h);
    if (st != IPEPS_OK) return st;
    double nnn[16] = {0};
    nnn[0] = 0.25 * J2; nnn[15] = 0.25 * J2;
    nnn[5] = -0.25 * J2; nnn[10] = -0.25 * J2;
    nnn[6] = 0.5 * J2; nnn[9] = 0.5 * J2;
    st = ipeps_ham_set_nnn(h, nnn, nnn);
    if (st != IPEPS_OK) {
      ipeps_ham_destroy(h);
      return st;
    }
    *out = h;
    return IPEPS_OK;
  });
}

ipeps_status ipeps_ham_kitaev(double K, ipeps_ham *out) {
  // tensor index s = 2 a + b; two-tensor index (a1, b1, a2, b2)
  const double I2[4] = {1, 0, 0, 1};
  const double Sx[4] = {0, 0.5, 0.5, 0};
  const double Sz[4] = {0.5, 0, 0, -0.5};
  // S^y = i Y with Y = [[0, -1/2], [1/2, 0]] real, so S^y S^y = -Y (x) Y
  const double Y[4] = {0, -0.5, 0.5, 0};
  double site[16], h[256], v[256];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      site[i * 4 + j] = K * Sz[(i >> 1) * 2 + (j >> 1)] * Sz[(i & 1) * 2 + (j & 1)];
  kron4(I2, Sx, Sx, I2, h);
  kron4(I2, Y, Y, I2, v);
  for (int i = 0; i < 256; ++i) {
    h[i] *= K;
    v[i] *= -K;
  }
  return ipeps_ham_create(4, h, v, site, 0.5, out);
}

void ipeps_ham_destroy(ipeps_ham h) { delete h; }

ipeps_status ipeps_ctmrg(const ipeps_shape *shape, const double *A_dev, int chi, double tol, int maxit,
                         ipeps_prec prec, ipeps_env *inout_env, int *iters_out, double *err_out,
                         ipeps_stream_t stream) {
  return guarded([&]() {
    ipeps::Cell c = cell_of(shape);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(A_dev && inout_env, "ctmrg: NULL argument");
    IPEPS_REQUIRE(chi >= 1 && chi <= 4096, "ctmrg: chi out of range");
    IPEPS_REQUIRE(maxit >= 0 && tol >= 0.0, "ctmrg: bad tol / maxit");
    IPEPS_REQUIRE(prec >= IPEPS_FP64 && prec <= IPEPS_BF16X3, "ctmrg: unknown precision");
    ipeps::PolicyScope policy(ipeps::fp64_grade_of(ipeps::Prec(prec)));
    check_finite(A_dev, int64_t(c.nsites()) * c.tsize(), s, "A");
    std::unique_ptr<ipeps_env_s> fresh;
    ipeps_env env = *inout_env;
    if (!env) {
      fresh = std::make_unique<ipeps_env_s>();
      env = fresh.get();
      env->impl.cell = c;
      env->impl.chi = chi;
      env->impl.s = s;
      env->impl.buf = ipeps::DBuf(size_t(env->impl.total()), s);
      ipeps::env_init(env->impl, A_dev, s);
    } else {
      check_env(env, c);
      IPEPS_REQUIRE(env->impl.chi == chi, "ctmrg: env has a different chi");
    }
    double err = 0.0;
    int it = 0;
    if (maxit > 0) it = ipeps::ctmrg_run(env->impl, A_dev, tol, maxit, ipeps::Prec(prec), &err, s);
    ipeps::tc_check_errors(s);
    if (iters_out) *iters_out = it;
    if (err_out) *err_out = err;
    if (fresh) *inout_env = fresh.release();
    if (maxit > 0 && !(err < tol)) {
      g_last_error = "CTMRG reached maxit before tol";
      return IPEPS_ERR_NOT_CONVERGED;
    }
    return IPEPS_OK;
  });
}

ipeps_status ipeps_env_corner_spectra(ipeps_env env, double *out_host, size_t n, ipeps_stream_t stream) {
  return guarded([&]() {
    IPEPS_REQUIRE(env && out_host, "corner_spectra: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto &e = env->impl;
    size_t need = size_t(4) * e.cell.nsites() * e.chi;
    IPEPS_REQUIRE(n >= need, "corner_spectra: output too small");
    ipeps::corner_spectra(e, s);
    IPEPS_CUDA(cudaMemcpyAsync(out_host, e.spectra.p, need * sizeof(double), cudaMemcpyDeviceToHost, s));
    IPEPS_CUDA(cudaStreamSynchronize(s));
    return IPEPS_OK;
  });
}

void ipeps_env_destroy(ipeps_env env) {
  if (!env) return;
  cudaStream_t s = env->impl.s;
  delete env;
  cudaStreamSynchronize(s);
}

ipeps_status ipeps_energy(const ipeps_shape *shape, const double *A_dev, ipeps_env env, ipeps_ham ham,
                          double *E_out, ipeps_stream_t stream) {
  return guarded([&]() {
    ipeps::Cell c = cell_of(shape);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(A_dev && ham && E_out, "energy: NULL argument");
    check_env(env, c);
    IPEPS_REQUIRE(ham->impl.d == c.d, "energy: Hamiltonian has a different d");
    ipeps::PolicyScope policy(ipeps::fp64_grade_of(env->impl.prec));
    *E_out = ipeps::energy_only(c, A_dev, env->impl, ham->impl, s);
    ipeps::tc_check_errors(s);
    if (!std::isfinite(*E_out)) throw ipeps::Error(IPEPS_ERR_NONFINITE, "energy is not finite");
    return IPEPS_OK;
  });
}

ipeps_status ipeps_energy_grad(const ipeps_shape *shape, const double *A_dev, ipeps_env env, ipeps_ham ham,
                               double *E_out, double *grad_dev, ipeps_stream_t stream) {
  return guarded([&]() {
    ipeps::Cell c = cell_of(shape);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(A_dev && ham && E_out && grad_dev, "energy_grad: NULL argument");
    check_env(env, c);
    IPEPS_REQUIRE(ham->impl.d == c.d, "energy_grad: Hamiltonian has a different d");
    check_finite(A_dev, int64_t(c.nsites()) * c.tsize(), s, "A");
    double ares = 0.0, fpres = 0.0;
    int amv = 0;
    ipeps::PolicyScope policy(ipeps::fp64_grade_of(env->impl.prec));
    *E_out = ipeps::energy_grad(c, A_dev, env->impl, ham->impl, grad_dev, s, &ares, &amv, &fpres);
    ipeps::tc_check_errors(s);
    if (!std::isfinite(*E_out)) throw ipeps::Error(IPEPS_ERR_NONFINITE, "energy is not finite");
    if (!(ares < 1e-8)) {
      g_last_error = "adjoint solve did not converge (relative residual " + std::to_string(ares) + ")";
      return IPEPS_ERR_NOT_CONVERGED;
    }
    return IPEPS_OK;
  });
}

ipeps_status ipeps_precondition(const ipeps_shape *shape, const double *A_dev, ipeps_env env,
                                const double *g_dev, double delta, int krylov, int restarts,
                                double *out_dev, double *resid_out, ipeps_stream_t stream) {
  return guarded([&]() {
    ipeps::Cell c = cell_of(shape);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(A_dev && g_dev && out_dev, "precondition: NULL argument");
    IPEPS_REQUIRE(krylov >= 1 && krylov <= 1000 && restarts >= 1 && restarts <= 1000,
                  "precondition: krylov / restarts out of range");
    IPEPS_REQUIRE(std::isfinite(delta), "precondition: delta must be finite");
    IPEPS_REQUIRE(out_dev != g_dev, "precondition: out_dev must not alias g_dev");
    check_env(env, c);
    check_finite(g_dev, int64_t(c.nsites()) * c.tsize(), s, "g");
    if (delta < 0.0) {
      // the |g|^2 rule of Sec. III.B, floored at 1e-12
      ipeps::DBuf nr(1, s);
      ipeps::nrm2(int64_t(c.nsites()) * c.tsize(), g_dev, nr.p, s);
      double h = 0.0;
      IPEPS_CUDA(cudaMemcpyAsync(&h, nr.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      IPEPS_CUDA(cudaStreamSynchronize(s));
      delta = std::max(h * h, 1e-12);
    }
    ipeps::PolicyScope policy(ipeps::fp64_grade_of(env->impl.prec));
    double r = ipeps::precondition_all(env->impl, A_dev, g_dev, delta, krylov, restarts, out_dev, s);
    ipeps::tc_check_errors(s);
    IPEPS_CUDA(cudaStreamSynchronize(s));
    if (resid_out) *resid_out = r;
    return IPEPS_OK;
  });
}

ipeps_status ipeps_precondition_bp(const ipeps_shape *shape, const double *A_dev, const double *g_dev,
                                   double delta, double bp_tol, int bp_maxit, double *out_dev, int *sweeps_out,
                                   double *change_out, ipeps_stream_t stream) {
  return guarded([&]() {
    ipeps::Cell c = cell_of(shape);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(A_dev && g_dev && out_dev, "precondition_bp: NULL argument");
    IPEPS_REQUIRE(c.D <= 32, "precondition_bp: bond dimension above 32");
    IPEPS_REQUIRE(std::isfinite(delta), "precondition_bp: delta must be finite");
    IPEPS_REQUIRE(bp_tol >= 0.0 && bp_maxit >= 1, "precondition_bp: bad sweep limits");
    IPEPS_REQUIRE(out_dev != g_dev && out_dev != A_dev, "precondition_bp: out_dev must not alias A_dev or g_dev");
    const int64_t n = int64_t(c.nsites()) * c.tsize();
    check_finite(A_dev, n, s, "A");
    check_finite(g_dev, n, s, "g");
    if (delta < 0.0) {
      // the |g|^2 rule of Sec. III.B, floored at 1e-12
      ipeps::DBuf nr(1, s);
      ipeps::nrm2(n, g_dev, nr.p, s);
      double h = 0.0;
      IPEPS_CUDA(cudaMemcpyAsync(&h, nr.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      IPEPS_CUDA(cudaStreamSynchronize(s));
      delta = std::max(h * h, 1e-12);
    }
    ipeps::BpMetric m;
    ipeps::bp_metric(c, A_dev, bp_tol, bp_maxit, m, s);
    ipeps::bp_apply(m, g_dev, delta, out_dev, s);
    IPEPS_CUDA(cudaStreamSynchronize(s));
    if (sweeps_out) *sweeps_out = m.sweeps;
    if (change_out) *change_out = m.change;
    return IPEPS_OK;
  });
}

ipeps_status ipeps_gemm(ipeps_prec prec, int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                        const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                        int64_t ldc, ipeps_stream_t stream) {
  return guarded([&]() {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(M >= 0 && N >= 0 && K >= 0, "gemm: negative size");
    IPEPS_REQUIRE((A && B) || K == 0, "gemm: NULL operand");
    IPEPS_REQUIRE(C || M * N == 0, "gemm: NULL output");
    IPEPS_REQUIRE((lda >= (ta ? M : K) && ldb >= (tb ? K : N)) || K == 0, "gemm: leading dimension too small");
    IPEPS_REQUIRE(ldc >= N, "gemm: leading dimension of C too small");
    ipeps::PolicyScope policy(ipeps::Prec::FP64);
    if (prec == IPEPS_TF32X3 || prec == IPEPS_TF32X3_ALL) ipeps::gemm_tf32x3(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    else if (prec == IPEPS_FP64) ipeps::gemm_f64(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    else if (prec == IPEPS_FP64_TC) ipeps::gemm_oz(8, ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    else if (prec == IPEPS_BF16X3) ipeps::gemm_oz(2, ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    else throw ipeps::Error(IPEPS_ERR_ARG, "gemm: unknown precision");
    IPEPS_CUDA(cudaStreamSynchronize(s));
    ipeps::tc_check_errors(s);
    return IPEPS_OK;
  });
}

ipeps_status ipeps_gemm_noalloc(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                                const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                                double *C, int64_t ldc, ipeps_stream_t stream) {
  return guarded([&]() {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(M >= 0 && N >= 0 && K >= 0, "gemm_noalloc: negative size");
    IPEPS_REQUIRE((A && B) || K == 0, "gemm_noalloc: NULL operand");
    IPEPS_REQUIRE(C || M * N == 0, "gemm_noalloc: NULL output");
    IPEPS_REQUIRE((lda >= (ta ? M : K) && ldb >= (tb ? K : N)) || K == 0,
                  "gemm_noalloc: leading dimension too small");
    IPEPS_REQUIRE(ldc >= N, "gemm_noalloc: leading dimension of C too small");
    ipeps::gemm_f64_noalloc(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    IPEPS_CUDA(cudaStreamSynchronize(s));
    return IPEPS_OK;
  });
}

void ipeps_opts_default(ipeps_opts *o) {
  if (!o) return;
  o->chi = 16;
  o->ctm_tol = 1e-10;
  o->ctm_maxit = 300;
  o->prec = IPEPS_FP64;
  o->precondition = 1;
  o->krylov = 30;
  o->restarts = 1;
  o->delta_rule = 0;
  o->history = 200;
  o->maxiter = 100;
  o->gtol = 1e-10;
  o->E_target = -1e300;
}

ipeps_status ipeps_optimize(const ipeps_shape *shape, double *A_dev, ipeps_ham ham, const ipeps_opts *opts,
                            ipeps_iter_cb cb, void *user, ipeps_stream_t stream) {
  return guarded([&]() {
    ipeps::Cell c = cell_of(shape);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    IPEPS_REQUIRE(A_dev && ham && opts, "optimize: NULL argument");
    IPEPS_REQUIRE(opts->chi >= 1 && opts->ctm_maxit >= 1 && opts->history >= 0 && opts->maxiter >= 0 &&
                      opts->krylov >= 1 && opts->restarts >= 1 && opts->prec >= IPEPS_FP64 &&
                      opts->prec <= IPEPS_BF16X3 && opts->precondition >= 0 && opts->precondition <= 2 &&
                      (opts->precondition != 2 || c.D <= 32),
                  "optimize: bad options");
    IPEPS_REQUIRE(ham->impl.d == c.d, "optimize: Hamiltonian has a different d");
    check_finite(A_dev, int64_t(c.nsites()) * c.tsize(), s, "A");
    ipeps::PolicyScope policy(ipeps::fp64_grade_of(ipeps::Prec(opts->prec)));
    ipeps_status st = ipeps::optimize_impl(c, A_dev, ham->impl, *opts, cb, user, s);
    ipeps::tc_check_errors(s);
    return st;
  });
}

}  // extern "C"
