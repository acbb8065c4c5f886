// Local-metric preconditioner (Eq. equ:local_metric, Sec. III.B, III.C) and
// the device GMRES used by it and by the fixed-point adjoint.
//
// M of a site is its single-site environment: the ring C1 T1 C2 T2 C3 T3 C4 T4
// with A and conj(A) removed, M[(u l d r), (u' l' d' r')] (D^4 x D^4); the
// local metric is 1_d (x) M.  M is symmetrised and scaled so that
// <A|1 (x) M|A> = 1.  P = 1_d (x) M + delta I is applied as one GEMM of the
// tensor viewed as d x D^4 with M plus an axpy; P^-1 g comes from GMRES
// (x0 = 0, classical Gram-Schmidt twice, Givens least squares), one tensor of
// the unit cell at a time (Sec. IV.B).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.h"
#include "engine.h"
#include "ipeps_impl.h"
#include "kernels.h"

namespace ipeps {

namespace {
__global__ void symmetrize_kernel(double *M, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * n;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = e / n, j = e % n;
    if (i < j) {
      double a = 0.5 * (M[i * n + j] + M[j * n + i]);
      M[i * n + j] = a;
      M[j * n + i] = a;
    }
  }
}
}  // namespace

void local_metrics(const EnvImpl &e, const double *A_dev, DBuf &Mall, cudaStream_t s) {
  const Cell &c = e.cell;
  const int64_t D4 = int64_t(c.D) * c.D * c.D * c.D;
  Mall = DBuf(size_t(c.nsites()) * D4 * D4, s);
  for (int x = 0; x < c.Lx; ++x)
    for (int y = 0; y < c.Ly; ++y) {
      Tape t(s);
      t.record = false;
      auto L = [&](int n) { return t.leaf(e.ptr(n, x, y), e.dims(n)); };
      int top = t_contract(t, L(C1), "ab", L(T1), "buvc", "auvc");
      top = t_contract(t, top, "auvc", L(C2), "ce", "auve");
      int bot = t_contract(t, L(C3), "fg", L(T3), "gdwh", "fdwh");
      bot = t_contract(t, bot, "fdwh", L(C4), "hi", "fdwi");
      int X = t_contract(t, top, "auve", L(T2), "erzf", "auvrzf");
      X = t_contract(t, X, "auvrzf", bot, "fdwi", "auvrzdwi");
      // ket (u l d r), bra (u' l' d' r')
      X = t_contract(t, X, "auvrzdwi", L(T4), "ilma", "uldrvmwz");
      double *M = Mall.p + int64_t(x * c.Ly + y) * D4 * D4;
      IPEPS_CUDA(cudaMemcpyAsync(M, t.vp(X), D4 * D4 * sizeof(double), cudaMemcpyDeviceToDevice, s));
      symmetrize_kernel<<<256, 256, 0, s>>>(M, D4);
      count_launch();
      check_launch("symmetrize");
      // <A| 1 (x) M |A>
      const double *A = A_dev + int64_t(x * c.Ly + y) * c.tsize();
      DBuf AM(size_t(c.d) * D4, s), nrm(1, s);
      gemm_f64(false, false, c.d, D4, D4, 1.0, A, D4, M, D4, 0.0, AM.p, D4, s);
      dot(c.d * D4, A, AM.p, nrm.p, s);
      div_by_scalar(D4 * D4, M, nrm.p, s);
    }
}

double gmres_dev(int64_t n, const MatVec &mv, const double *b, double *x, int krylov, int restarts,
                 double rtol, cudaStream_t s, int *matvecs) {
  // Arnoldi with classical Gram-Schmidt applied twice, all on the device; the
  // new Hessenberg column (j + 2 numbers) comes back to the host once per
  // step for the Givens rotations and the residual estimate
  IPEPS_REQUIRE(krylov >= 1 && restarts >= 1, "gmres: krylov and restarts must be >= 1");
  const int m = krylov;
  DBuf V(size_t(m + 1) * n, s), w(size_t(n), s), r(size_t(n), s), h(size_t(m + 2), s), h2(size_t(m + 2), s),
      sc(1, s);
  fill(x, n, 0.0, s);
  auto host_scalar = [&](const double *p) {
    double v;
    IPEPS_CUDA(cudaMemcpyAsync(&v, p, sizeof(double), cudaMemcpyDeviceToHost, s));
    IPEPS_CUDA(stream_sync(s));
    return v;
  };
  nrm2(n, b, sc.p, s);
  const double bnorm = host_scalar(sc.p);
  int nmv = 0;
  if (bnorm == 0.0) {
    if (matvecs) *matvecs = 0;
    return 0.0;
  }
  double rel = 1.0;
  std::vector<double> col(size_t(m) + 2);
  for (int cycle = 0; cycle < restarts; ++cycle) {
    if (cycle == 0) {
      IPEPS_CUDA(cudaMemcpyAsync(r.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      mv(x, r.p);
      ++nmv;
      axpby(n, 1.0, b, -1.0, r.p, s);  // r = b - A x
    }
    nrm2(n, r.p, sc.p, s);
    double beta = host_scalar(sc.p);
    rel = beta / bnorm;
    if (rel <= rtol) break;
    std::vector<double> H(size_t(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1, 0.0);
    gv[0] = beta;
    IPEPS_CUDA(cudaMemcpyAsync(V.p, r.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    scal(n, 1.0 / beta, V.p, s);
    int used = 0;
    for (int j = 0; j < m; ++j) {
      mv(V.p + int64_t(j) * n, w.p);
      ++nmv;
      // h = V[0..j] w, w -= V[0..j]^T h, twice; h accumulates both passes
      gemm_f64(false, false, j + 1, 1, n, 1.0, V.p, n, w.p, 1, 0.0, h.p, 1, s);
      gemm_f64(true, false, n, 1, j + 1, -1.0, V.p, n, h.p, 1, 1.0, w.p, 1, s);
      gemm_f64(false, false, j + 1, 1, n, 1.0, V.p, n, w.p, 1, 0.0, h2.p, 1, s);
      gemm_f64(true, false, n, 1, j + 1, -1.0, V.p, n, h2.p, 1, 1.0, w.p, 1, s);
      axpy(j + 1, 1.0, h2.p, h.p, s);
      nrm2(n, w.p, h.p + j + 1, s);
      // next basis vector (a zero norm leaves it zero; the loop stops below)
      IPEPS_CUDA(cudaMemcpyAsync(V.p + int64_t(j + 1) * n, w.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      div_by_scalar(n, V.p + int64_t(j + 1) * n, h.p + j + 1, s);
      IPEPS_CUDA(cudaMemcpyAsync(col.data(), h.p, size_t(j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
      IPEPS_CUDA(stream_sync(s));
      const double hn = col[j + 1];
      for (int i = 0; i <= j; ++i) H[i * m + j] = col[i];
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else { cs[j] = H[j * m + j] / den; sn[j] = H[(j + 1) * m + j] / den; }
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      used = j + 1;
      rel = std::fabs(gv[j + 1]) / bnorm;
      if (std::getenv("IPEPS_DEBUG_GMRES")) {
        static auto tlast = std::chrono::steady_clock::now();
        auto tn = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[ipeps] gmres n=%lld cycle %d step %d rel %.3e (%.1f ms)\n", (long long)n, cycle, j,
                     rel, std::chrono::duration<double, std::milli>(tn - tlast).count());
        tlast = tn;
      }
      if (rel <= rtol || hn == 0.0) break;
    }
    std::vector<double> y(used, 0.0);
    for (int i = used - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int k = i + 1; k < used; ++k) acc -= H[i * m + k] * y[k];
      y[i] = acc / H[i * m + i];
    }
    IPEPS_CUDA(cudaMemcpyAsync(h.p, y.data(), used * sizeof(double), cudaMemcpyHostToDevice, s));
    gemm_f64(true, false, n, 1, used, 1.0, V.p, n, h.p, 1, 1.0, x, 1, s);
    IPEPS_CUDA(stream_sync(s));  // y leaves scope
    if (rel <= rtol) break;
  }
  if (matvecs) *matvecs = nmv;
  return rel;
}

double precondition_all(const EnvImpl &e, const double *A_dev, const double *g, double delta,
                        int krylov, int restarts, double *out, cudaStream_t s) {
  const Cell &c = e.cell;
  const int64_t D4 = int64_t(c.D) * c.D * c.D * c.D;
  DBuf Mall;
  local_metrics(e, A_dev, Mall, s);
  double worst = 0.0;
  for (int i = 0; i < c.nsites(); ++i) {
    const double *M = Mall.p + int64_t(i) * D4 * D4;
    const int64_t n = c.tsize();
    MatVec mv = [&](const double *xv, double *yv) {
      // y = x M^T + delta x for x viewed as d x D^4
      gemm_f64(false, true, c.d, D4, D4, 1.0, xv, D4, M, D4, 0.0, yv, D4, s);
      axpy(n, delta, xv, yv, s);
    };
    int nmv = 0;
    double rel = gmres_dev(n, mv, g + int64_t(i) * n, out + int64_t(i) * n, krylov, restarts, 1e-14, s,
                           &nmv);
    worst = std::max(worst, rel);
  }
  return worst;
}

}  // namespace ipeps
