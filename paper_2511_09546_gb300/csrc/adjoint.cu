// Energy and its gradient at the CTMRG fixed point (Sec. III.A: dE/dA of the
// energy functional), by implicit differentiation of the fixed point.
//
// With F one CTMRG iteration followed by the constant sign gauge sigma that
// makes the converged environment e* an elementwise fixed point,
//   g = dE/dA|_e + (dF/dA)^T lam,   (I - (dF/de)^T) lam = dE/de|_A.
// One F pass and one energy pass are recorded on tapes (their intermediates
// stay resident in HBM); every Krylov step of the device GMRES replays the
// hand-written adjoints of the F tape with a new cotangent.
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

double energy_only(const Cell &c, const double *A_dev, EnvImpl &e, const HamImpl &H, cudaStream_t s) {
  HamDev hd(H, s);
  Tape t(s);
  t.record = false;
  StateVars sv = state_leaves(t, e, A_dev);
  int E = energy_on_tape(t, c, e.chi, sv, H, hd);
  double v;
  IPEPS_CUDA(cudaMemcpyAsync(&v, t.vp(E), sizeof(double), cudaMemcpyDeviceToHost, s));
  IPEPS_CUDA(stream_sync(s));
  return v;
}

double energy_grad(const Cell &c, const double *A_dev, EnvImpl &e, const HamImpl &H, double *grad,
                   cudaStream_t s, double *adj_resid, int *adj_mv, double *fp_resid) {
  const int ns = c.nsites();
  const int64_t nenv = e.total(), ta = c.tsize();
  HamDev hd(H, s);
  const bool dbg = std::getenv("IPEPS_DEBUG") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](const char *what) {
    if (!dbg) return;
    IPEPS_CUDA(stream_sync(s));
    auto t1 = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[ipeps] energy_grad %s: %.1f ms\n", what,
                 std::chrono::duration<double, std::milli>(t1 - t0).count());
    t0 = t1;
  };

  // ---- F tape at e*
  Tape tF(s);
  tF.vcache = &e.svd_cache;
  tF.prec = e.prec;  // the fixed-point map in the precision of the last CTMRG iterations
  StateVars in = state_leaves(tF, e, A_dev);
  StateVars out = in;
  ctmrg_iteration(tF, c, e.chi, out);
  std::vector<const double *> cand(8 * ns);
  for (int n = 0; n < 8; ++n)
    for (int i = 0; i < ns; ++i) cand[n * ns + i] = tF.vp(out.env[n][i]);
  double fpres = 0.0;
  DBuf sig = solve_signs(e, cand, s, &fpres);
  std::vector<int> outs(8 * ns);
  for (int n = 0; n < 8; ++n)
    for (int i = 0; i < ns; ++i) {
      int k = n * ns + i;
      outs[k] = t_signs(tF, out.env[n][i], sig.p + int64_t(2 * k) * e.chi, sig.p + int64_t(2 * k + 1) * e.chi);
    }
  if (fp_resid) *fp_resid = fpres;
  lap("F tape + sign gauge");

  // ---- energy tape: E, dE/de, dE/dA
  Tape tE(s);
  StateVars se = state_leaves(tE, e, A_dev);
  int Ev = energy_on_tape(tE, c, e.chi, se, H, hd);
  fill(tE.grad(Ev), 1, 1.0, s);
  tE.backward();
  double E;
  IPEPS_CUDA(cudaMemcpyAsync(&E, tE.vp(Ev), sizeof(double), cudaMemcpyDeviceToHost, s));
  DBuf ebar(size_t(nenv), s);
  fill(ebar.p, nenv, 0.0, s);
  for (int n = 0; n < 8; ++n)
    for (int i = 0; i < ns; ++i) {
      double *g = tE.grad(se.env[n][i], false);
      if (g)
        IPEPS_CUDA(cudaMemcpyAsync(ebar.p + e.offset(n, i / c.Ly, i % c.Ly), g,
                                   tE.val(se.env[n][i]).size() * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
  fill(grad, int64_t(ns) * ta, 0.0, s);
  for (int i = 0; i < ns; ++i) {
    double *g = tE.grad(se.A[0][i], false);
    if (g) axpy(ta, 1.0, g, grad + int64_t(i) * ta, s);
  }
  tE.clear();
  lap("energy tape");
  if (dbg) {
    DBuf nb(1, s);
    nrm2(nenv, ebar.p, nb.p, s);
    double h;
    IPEPS_CUDA(cudaMemcpyAsync(&h, nb.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    IPEPS_CUDA(stream_sync(s));
    std::fprintf(stderr, "[ipeps] |dE/denv| = %.6e\n", h);
  }

  // ---- vector-Jacobian products of F
  auto vjp = [&](const double *lam, double *out_env, double *out_A) {
    tF.zero_grads();
    for (int n = 0; n < 8; ++n)
      for (int i = 0; i < ns; ++i) {
        int k = n * ns + i;
        IPEPS_CUDA(cudaMemcpyAsync(tF.grad(outs[k]), lam + e.offset(n, i / c.Ly, i % c.Ly),
                                   tF.val(outs[k]).size() * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
    tF.backward();
    if (out_env) {
      fill(out_env, nenv, 0.0, s);
      for (int n = 0; n < 8; ++n)
        for (int i = 0; i < ns; ++i) {
          double *g = tF.grad(in.env[n][i], false);
          if (g)
            IPEPS_CUDA(cudaMemcpyAsync(out_env + e.offset(n, i / c.Ly, i % c.Ly), g,
                                       tF.val(in.env[n][i]).size() * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
        }
    }
    if (out_A)
      for (int i = 0; i < ns; ++i) {
        double *g = tF.grad(in.A[0][i], false);
        if (g) axpy(ta, 1.0, g, out_A + int64_t(i) * ta, s);
      }
  };
  MatVec mv = [&](const double *x, double *y) {
    vjp(x, y, nullptr);
    axpby(nenv, 1.0, x, -1.0, y, s);  // y = x - J^T x
  };
  DBuf lam(size_t(nenv), s);
  int nmv = 0;
  int kry = 40, rst = 6;
  if (const char *v = std::getenv("IPEPS_ADJ_KRYLOV")) kry = std::atoi(v);
  if (const char *v = std::getenv("IPEPS_ADJ_RESTARTS")) rst = std::atoi(v);
  double rel = gmres_dev(nenv, mv, ebar.p, lam.p, kry, rst, 1e-12, s, &nmv);
  lap("adjoint GMRES");
  if (dbg)
    std::fprintf(stderr, "[ipeps] adjoint: %d matvecs, residual %.2e, fixed-point residual %.2e, cg %d\n", nmv,
                 rel, fpres, tF.svd_iters);
  vjp(lam.p, nullptr, grad);
  IPEPS_CUDA(stream_sync(s));
  if (adj_resid) *adj_resid = rel;
  if (adj_mv) *adj_mv = nmv;
  return E;
}

}  // namespace ipeps
