// Internal structures of the iPEPS hot path: the device-resident environment,
// the unit-cell frames used by the directional CTMRG moves, and the
// functions behind the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <functional>
#include <map>
#include <memory>
#include <vector>

#include "common.h"
#include "engine.h"

namespace ipeps {

// Boundary tensor names; legs of a corner are (prev, next), of an edge
// (prev, ket, bra, next), running clockwise C1 T1 C2 T2 C3 T3 C4 T4.
enum Name { C1 = 0, C2, C3, C4, T1, T2, T3, T4 };
constexpr double kSplitSwitch = 1e-6;  // split mode: spectra change at which FP64 takes over
constexpr double kSvCutoff = 1e-12;  // relative cut of the projector spectrum (FP64 GEMMs)
// Relative cut of the projector spectrum for the precision the enlarged corners
// were contracted in: singular values of the four-corner product below the
// GEMM error floor carry no information, and S^-1/2 would amplify that noise
// into the projectors.  IPEPS_SV_CUTOFF_FP64 / IPEPS_SV_CUTOFF_TF32X3 override
// the two cuts (1e-12 and 1e-7).
double sv_cutoff(Prec prec);

struct Cell {
  int Lx = 1, Ly = 1, d = 2, D = 2;
  int nsites() const { return Lx * Ly; }
  int64_t tsize() const { return int64_t(d) * D * D * D * D; }
};

// Frame r: the picture rotated counter-clockwise r times.  Tensors of frame r
// at (n, x, y) are stored as frame-0 tensors at resolve(r, n, x, y).
struct Frame {
  int Lx0, Ly0, r;
  int Lx() const { return (r % 2 == 0) ? Lx0 : Ly0; }
  int Ly() const { return (r % 2 == 0) ? Ly0 : Lx0; }
  // frame-0 (name, x, y) of the frame-r tensor (n, x, y)
  void resolve(int n, int x, int y, int *n0, int *x0, int *y0) const;
  void resolve_site(int x, int y, int *x0, int *y0) const {
    int n0;
    resolve(0, x, y, &n0, x0, y0);
  }
};

struct EnvImpl {
  Cell cell;
  int chi = 0;
  DBuf buf;              // all 8 * Lx * Ly tensors, zero padded to chi
  DBuf spectra;          // last corner spectra (4 * Lx * Ly * chi)
  bool have_spectra = false;
  std::map<int, DBuf> svd_cache;  // warm starts of the projector SVDs
  Prec prec = Prec::FP64;         // precision of the last CTMRG iterations (reused by the adjoint)
  cudaStream_t s = nullptr;
  int64_t csize() const { return int64_t(chi) * chi; }
  int64_t esize() const { return int64_t(chi) * cell.D * cell.D * chi; }
  int64_t site_size() const { return 4 * csize() + 4 * esize(); }
  int64_t total() const { return site_size() * cell.nsites(); }
  int64_t offset(int n, int x, int y) const {
    int64_t o = site_size() * (int64_t(x) * cell.Ly + y);
    return n < 4 ? o + n * csize() : o + 4 * csize() + (n - 4) * esize();
  }
  double *ptr(int n, int x, int y) const { return buf.p + offset(n, x, y); }
  std::vector<int64_t> dims(int n) const {
    if (n < 4) return {chi, chi};
    return {chi, cell.D, cell.D, chi};
  }
};

// Tape variables of a unit-cell state: env[n][site0] and A legs rotated q times
struct StateVars {
  std::array<std::vector<int>, 8> env;  // frame-0 site index x*Ly+y
  std::array<std::vector<int>, 4> A;    // rotated copies of every tensor
};

// ---- CTMRG (ctmrg.cu)
void env_init(EnvImpl &e, const double *A_dev, cudaStream_t s);
// One CTMRG iteration on the tape: reads sv.env, replaces it by the new ids.
void ctmrg_iteration(Tape &t, const Cell &c, int chi, StateVars &sv);
// Leaves for the env buffer and the tensors (+ their rotated copies).
StateVars state_leaves(Tape &t, const EnvImpl &e, const double *A_dev);
// Forward iterations to convergence.  Returns iterations; *err the final change.
int ctmrg_run(EnvImpl &e, const double *A_dev, double tol, int maxit, Prec prec, double *err,
              cudaStream_t s);
// Normalised corner spectra of the env into e.spectra (device).
void corner_spectra(EnvImpl &e, cudaStream_t s);
// Largest spectral change between two spectra buffers; with count_dev, the
// device int is read into *count_host by the same host wait.
double spectra_change(const double *a, const double *b, int nmat, int chi, cudaStream_t s,
                      const int *count_dev = nullptr, int *count_host = nullptr);
// Sign gauge: signs per tensor leg such that ref ~ sign . cand elementwise.
// Returns device buffer of (8 * nsites) x 2 x chi signs (prev, next per tensor).
DBuf solve_signs(const EnvImpl &ref, const std::vector<const double *> &cand, cudaStream_t s,
                 double *residual);

// ---- energy (energy.cu)
struct HamImpl {
  int d = 2;
  double scale = 1.0;
  std::vector<double> h, v, site;  // host copies
  bool has_site = false;
  std::vector<double> d1, d2;      // diagonal (x,y)-(x+1,y+1), anti-diagonal (x+1,y)-(x,y+1)
  bool has_d1 = false, has_d2 = false;
};
struct HamDev {
  DBuf h, v, site, d1, d2;
  HamDev(const HamImpl &H, cudaStream_t s);
};
// energy per site on the tape (scalar variable id)
int energy_on_tape(Tape &t, const Cell &c, int chi, const StateVars &sv, const HamImpl &H,
                   const HamDev &hd);

// ---- metric and GMRES (precond.cu)
// M[(u l d r), (u' l' d' r')] of every site, symmetrised and normalised
void local_metrics(const EnvImpl &e, const double *A_dev, DBuf &M, cudaStream_t s);
double precondition_all(const EnvImpl &e, const double *A_dev, const double *g, double delta,
                        int krylov, int restarts, double *out, cudaStream_t s);
// generic restarted GMRES on device vectors (x0 = 0, CGS2 Arnoldi, Givens);
// returns the relative residual estimate
using MatVec = std::function<void(const double *x, double *y)>;
double gmres_dev(int64_t n, const MatVec &mv, const double *b, double *x, int krylov, int restarts,
                 double rtol, cudaStream_t s, int *matvecs);

// ---- optimiser (optimize.cu)
class LbfgsRun {
 public:
  LbfgsRun(const Cell &c, const HamImpl &H, const ipeps_opts &o, cudaStream_t s);
  ~LbfgsRun();
  LbfgsRun(const LbfgsRun &) = delete;
  LbfgsRun &operator=(const LbfgsRun &) = delete;
  ipeps_iter_info start(const double *A_dev);  // evaluates the starting point (copied)
  bool step(ipeps_iter_info *info);            // one iteration; false when the run has ended
  bool finished() const;
  int iteration() const;
  double energy() const;
  void copy_tensor(double *A_dev) const;       // current tensors (stream-ordered)

 private:
  struct Impl;
  std::unique_ptr<Impl> impl_;
};
ipeps_status optimize_impl(const Cell &c, double *A_dev, const HamImpl &H, const ipeps_opts &o,
                           ipeps_iter_cb cb, void *user, cudaStream_t s);

// ---- gradient (adjoint.cu)
double energy_only(const Cell &c, const double *A_dev, EnvImpl &e, const HamImpl &H, cudaStream_t s);
double energy_grad(const Cell &c, const double *A_dev, EnvImpl &e, const HamImpl &H, double *grad,
                   cudaStream_t s, double *adj_resid, int *adj_mv, double *fp_resid);

}  // namespace ipeps

// the opaque handles of the C ABI
struct ipeps_env_s {
  ipeps::EnvImpl impl;
};
struct ipeps_ham_s {
  ipeps::HamImpl impl;
};
