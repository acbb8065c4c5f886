// Directional CTMRG on the device (Sec. III.A: the environment that the
// energy is contracted with).
//
// One iteration is four left moves, each in a frame of the unit cell rotated
// counter-clockwise by 0, 90, 180 and 270 degrees (the rotation relabels the
// boundary tensors and rotates the legs of A; nothing is copied for the
// environment).  A left move, for every column x and every cut between rows
// y and y+1 (all columns at once):
//   enlarged corners Q_ul, Q_ur, Q_lr, Q_ll of the 2x2 patch at (x, y);
//   halves R1 = Q_ul Q_ur, R2 = Q_lr Q_ll and the opened ring M = R2 R1;
//   truncated SVD M ~ U S V^T (top chi, FP64);
//   projectors P_up = R2^T U S^-1/2 (upper side) and P_dn = R1 V S^-1/2;
//   absorption C1 <- P_up^T (C1 T1), T4 <- P_up^T (T4 A A) P_dn,
//   C4 <- (T3 C4) P_dn, each divided by its Frobenius norm.
// The environment is stored zero padded to chi from the start (init bond
// D^2): padded directions carry zero singular values and are cut, which is
// the same fixed point as growing chi.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <queue>
#include <tuple>

#include "common.h"
#include "engine.h"
#include "ipeps_impl.h"
#include "kernels.h"

namespace ipeps {

double sv_cutoff(Prec prec) {
  // the split mode's projector SVD sees an FP64 four-corner product
  static const double c64 = [] {
    const char *e = std::getenv("IPEPS_SV_CUTOFF_FP64");
    return e ? std::atof(e) : kSvCutoff;
  }();
  static const double c3 = [] {
    const char *e = std::getenv("IPEPS_SV_CUTOFF_TF32X3");
    return e ? std::atof(e) : 1e-7;
  }();
  return prec == Prec::TF32X3_ALL ? c3 : c64;
}

namespace {
int rot_name(int n) { return n < 4 ? (n + 1) % 4 : 4 + (n - 4 + 1) % 4; }

__global__ void embed_kernel(const double *src, int64_t a, int64_t mid, int64_t b, double *dst,
                             int64_t chi) {
  int64_t total = chi * mid * chi;
  int64_t ac = a < chi ? a : chi, bc = b < chi ? b : chi;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t j = e % chi, m = (e / chi) % mid, i = e / (chi * mid);
    dst[e] = (i < ac && j < bc) ? src[(i * mid + m) * b + j] : 0.0;
  }
}
}  // namespace

void Frame::resolve(int n, int x, int y, int *n0, int *x0, int *y0) const {
  int nn = n, xx = x, yy = y;
  for (int k = r - 1; k >= 0; --k) {
    int Lxk = (k % 2 == 0) ? Lx0 : Ly0;
    int nx = ((-yy) % Lxk + Lxk) % Lxk, ny = xx;
    nn = (n >= 0) ? rot_name(nn) : nn;
    xx = nx;
    yy = ny;
  }
  *n0 = nn;
  *x0 = xx;
  *y0 = yy;
}

// --------------------------------------------------------------------- init
void env_init(EnvImpl &e, const double *A_dev, cudaStream_t s) {
  const Cell &c = e.cell;
  const int D = c.D, d = c.d;
  const int64_t D2 = int64_t(D) * D;
  fill(e.buf.p, e.total(), 0.0, s);
  auto Aptr = [&](int x, int y) {
    x = ((x % c.Lx) + c.Lx) % c.Lx;
    y = ((y % c.Ly) + c.Ly) % c.Ly;
    return Ten{const_cast<double *>(A_dev) + (int64_t(x) * c.Ly + y) * c.tsize(), {d, D, D, D, D}};
  };
  struct Spec { int n, dx, dy; const char *la, *lb, *lc; bool corner; };
  // each boundary tensor is the neighbouring double-layer tensor with its
  // outward legs traced ket against bra
  const Spec specs[8] = {
      {C1, -1, -1, "suldr", "sulek", "derk", true},   {T1, 0, -1, "suldr", "sumek", "lmderk", false},
      {C2, 1, -1, "suldr", "sumer", "lmde", true},    {T2, 1, 0, "suldr", "svmer", "uvlmde", false},
      {C3, 1, 1, "suldr", "svmdr", "uvlm", true},     {T3, 0, 1, "suldr", "svmdk", "rkuvlm", false},
      {C4, -1, 1, "suldr", "svldk", "rkuv", true},    {T4, -1, 0, "suldr", "svlek", "derkuv", false}};
  for (int x = 0; x < c.Lx; ++x)
    for (int y = 0; y < c.Ly; ++y)
      for (const Spec &sp : specs) {
        Ten a = Aptr(x + sp.dx, y + sp.dy);
        std::vector<int64_t> od(std::string(sp.lc).size(), D);
        DBuf tmp(size_t(prod(od)), s);
        contract(a, sp.la, a, sp.lb, Ten{tmp.p, od}, sp.lc, s);
        int64_t mid = sp.corner ? 1 : D2;
        embed_kernel<<<256, 256, 0, s>>>(tmp.p, D2, mid, D2, e.ptr(sp.n, x, y), e.chi);
        count_launch();
        check_launch("env embed");
        int64_t n = sp.corner ? e.csize() : e.esize();
        DBuf nr(1, s);
        nrm2(n, e.ptr(sp.n, x, y), nr.p, s);
        div_by_scalar(n, e.ptr(sp.n, x, y), nr.p, s);
      }
}

// ------------------------------------------------------------- tape states
StateVars state_leaves(Tape &t, const EnvImpl &e, const double *A_dev) {
  const Cell &c = e.cell;
  StateVars sv;
  for (int n = 0; n < 8; ++n) {
    sv.env[n].resize(c.nsites());
    for (int x = 0; x < c.Lx; ++x)
      for (int y = 0; y < c.Ly; ++y) sv.env[n][x * c.Ly + y] = t.leaf(e.ptr(n, x, y), e.dims(n));
  }
  for (int q = 0; q < 4; ++q) sv.A[q].resize(c.nsites());
  for (int i = 0; i < c.nsites(); ++i) {
    sv.A[0][i] = t.leaf(const_cast<double *>(A_dev) + i * c.tsize(), {c.d, c.D, c.D, c.D, c.D});
    for (int q = 1; q < 4; ++q) sv.A[q][i] = t_permute(t, sv.A[q - 1][i], {0, 4, 1, 2, 3});
  }
  return sv;
}

namespace {

int corner_ul(Tape &t, int c1, int t1, int t4, int a) {
  int X1 = t_contract(t, c1, "ab", t1, "bcde", "acde");       // [C1.p, u, u', T1.n]
  int X2 = t_contract(t, t4, "fgha", X1, "acde", "fghcde");   // [T4.p, l, l', u, u', T1.n]
  int X3 = t_contract(t, X2, "fghcde", a, "scgjk", "fhdesjk"); // ket A on (u, l)
  int X4 = t_contract(t, X3, "fhdesjk", a, "sdhmn", "fjmekn"); // bra A on (s, u', l')
  t.release(X1);
  t.release(X2);
  t.release(X3);
  const auto &d = t.val(X4).d;
  return t_reshape(t, X4, {d[0] * d[1] * d[2], d[3] * d[4] * d[5]});
}

void left_move(Tape &t, const Cell &c, int chi, StateVars &sv, int r) {
  Frame f{c.Lx, c.Ly, r};
  const int Lx = f.Lx(), Ly = f.Ly();
  auto E = [&](int n, int x, int y) {
    x = ((x % Lx) + Lx) % Lx;
    y = ((y % Ly) + Ly) % Ly;
    int n0, x0, y0;
    f.resolve(n, x, y, &n0, &x0, &y0);
    return sv.env[n0][x0 * c.Ly + y0];
  };
  auto Av = [&](int q, int x, int y) {
    x = ((x % Lx) + Lx) % Lx;
    y = ((y % Ly) + Ly) % Ly;
    int x0, y0;
    f.resolve_site(x, y, &x0, &y0);
    return sv.A[(r + q) % 4][x0 * c.Ly + y0];
  };
  std::vector<int> Pup(Lx * Ly), Pdn(Lx * Ly);
  for (int x = 0; x < Lx; ++x)
    for (int y = 0; y < Ly; ++y) {
      int Qul = corner_ul(t, E(C1, x, y), E(T1, x, y), E(T4, x, y), Av(0, x, y));
      int Qur = corner_ul(t, E(C2, x + 1, y), E(T2, x + 1, y), E(T1, x + 1, y), Av(1, x + 1, y));
      int Qlr = corner_ul(t, E(C3, x + 1, y + 1), E(T3, x + 1, y + 1), E(T2, x + 1, y + 1),
                          Av(2, x + 1, y + 1));
      int Qll = corner_ul(t, E(C4, x, y + 1), E(T4, x, y + 1), E(T3, x, y + 1), Av(3, x, y + 1));
      int R1 = t_contract(t, Qul, "ab", Qur, "bc", "ac");
      int R2 = t_contract(t, Qlr, "ab", Qll, "bc", "ac");
      for (int q : {Qul, Qur, Qlr, Qll}) t.release(q);
      // the four-corner product squares the dynamic range of the half systems:
      // its small singular directions decide the projectors and sit below the
      // 3xTF32 noise floor of |R2||R1|, so the split mode forms it (and the
      // projector products) in FP64
      const Prec keep = t.prec;
      if (keep != Prec::TF32X3_ALL) t.prec = Prec::FP64;
      int M = t_contract(t, R2, "ab", R1, "bc", "ac");
      int N = int(t.val(M).d[0]);
      int U, S, V;
      t.vkey = (r * 64 + x) * 64 + y;
      t_svd(t, M, std::min(chi, N), &U, &S, &V);
      t.release(M);
      int fs = t_inv_sqrt_cut(t, S, sv_cutoff(keep));
      Pup[x * Ly + y] = t_scale_cols(t, t_contract(t, R2, "ba", U, "bk", "ak"), fs);
      Pdn[x * Ly + y] = t_scale_cols(t, t_contract(t, R1, "ab", V, "bk", "ak"), fs);
      t.prec = keep;
      t.release(R1);
      t.release(R2);
    }
  // absorb column x into the left boundary of column x+1 (all columns)
  std::vector<std::tuple<int, int, int, int>> upd;  // (name, x, y, var) in frame r
  for (int x = 0; x < Lx; ++x)
    for (int y = 0; y < Ly; ++y) {
      const int ym = ((y - 1) % Ly + Ly) % Ly;
      int X = t_contract(t, E(C1, x, y), "ab", E(T1, x, y), "bcde", "acde");
      const auto &dx = t.val(X).d;
      X = t_reshape(t, X, {dx[0] * dx[1] * dx[2], dx[3]});
      int c1 = t_contract(t, Pup[x * Ly + ym], "ak", X, "an", "kn");
      // T4' = Pup^T (T4 A Abar) Pdn with the projectors applied first, so no
      // intermediate exceeds chi^2 D^4 d entries: Pup rows are (p, d, d'),
      // Pdn rows are (n, u, u')
      const int et4 = E(T4, x, y);
      const auto dt = t.val(et4).d;  // [p, D, D, n]
      const int pu = Pup[x * Ly + y], pd = Pdn[x * Ly + ym];
      const int pu4 = t_reshape(t, pu, {dt[0], dt[1], dt[2], t.val(pu).d[1]});
      const int pd4 = t_reshape(t, pd, {dt[3], dt[1], dt[2], t.val(pd).d[1]});
      int W1 = t_contract(t, pu4, "pdek", et4, "plqn", "deklqn");
      int W2 = t_contract(t, W1, "deklqn", Av(0, x, y), "suldr", "ekqnsur");  // ket A on (l, d)
      t.release(W1);
      int W3 = t_contract(t, W2, "ekqnsur", Av(0, x, y), "svqeg", "knurvg");  // bra A on (s, l', d')
      t.release(W2);
      int t4 = t_contract(t, W3, "knurvg", pd4, "nuvm", "krgm");
      t.release(W3);
      int Z = t_contract(t, E(T3, x, y), "pden", E(C4, x, y), "nm", "pmde");
      const auto &dz = t.val(Z).d;
      Z = t_reshape(t, Z, {dz[0], dz[1] * dz[2] * dz[3]});
      int c4 = t_contract(t, Z, "pa", Pdn[x * Ly + y], "ak", "pk");
      upd.emplace_back(C1, x + 1, y, t_normalize(t, c1));
      upd.emplace_back(T4, x + 1, y, t_normalize(t, t4));
      upd.emplace_back(C4, x + 1, y, t_normalize(t, c4));
    }
  for (auto &u : upd) {
    int n, x, y, v;
    std::tie(n, x, y, v) = u;
    x = x % Lx;
    int n0, x0, y0;
    f.resolve(n, x, y, &n0, &x0, &y0);
    sv.env[n0][x0 * c.Ly + y0] = v;
  }
}
}  // namespace

void ctmrg_iteration(Tape &t, const Cell &c, int chi, StateVars &sv) {
  for (int r = 0; r < 4; ++r) left_move(t, c, chi, sv, r);
}

// --------------------------------------------------------------- spectra
namespace {
__global__ void gather_corners(const double *buf, int64_t site_size, int64_t csize, int nsites,
                               double *out) {
  int64_t total = int64_t(4) * nsites * csize;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t mat = e / csize, w = e % csize;
    int n = int(mat / nsites), site = int(mat % nsites);
    out[e] = buf[site * site_size + n * csize + w];
  }
}

// column norms of each chi x chi column-major matrix, sorted descending and
// normalised to unit 2-norm
__global__ void spectra_kernel(const double *G, int chi, double *out) {
  extern __shared__ double sv[];
  const double *Gm = G + int64_t(blockIdx.x) * chi * chi;
  for (int j = threadIdx.x; j < chi; j += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < chi; ++i) a += Gm[int64_t(j) * chi + i] * Gm[int64_t(j) * chi + i];
    sv[j] = sqrt(a);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < chi; ++i) {
      double v = sv[i];
      int k = i - 1;
      while (k >= 0 && sv[k] < v) { sv[k + 1] = sv[k]; --k; }
      sv[k + 1] = v;
    }
    double nrm = 0.0;
    for (int i = 0; i < chi; ++i) nrm += sv[i] * sv[i];
    nrm = sqrt(nrm);
    // non-finite input must not look converged: propagate it
    for (int i = 0; i < chi; ++i) sv[i] = (nrm > 0 || !isfinite(nrm)) ? sv[i] / nrm : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < chi; j += blockDim.x) out[int64_t(blockIdx.x) * chi + j] = sv[j];
}

__global__ void spectra_diff_kernel(const double *a, const double *b, int chi, double *out) {
  __shared__ double sh[256];
  const double *x = a + int64_t(blockIdx.x) * chi, *y = b + int64_t(blockIdx.x) * chi;
  double acc = 0.0;
  for (int i = threadIdx.x; i < chi; i += blockDim.x) acc += (x[i] - y[i]) * (x[i] - y[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(sh[0]);
}
}  // namespace

void corner_spectra(EnvImpl &e, cudaStream_t s) {
  const int nmat = 4 * e.cell.nsites();
  if (!e.spectra.p) e.spectra = DBuf(size_t(nmat) * e.chi, s);
  DBuf G(size_t(nmat) * e.csize(), s);
  gather_corners<<<256, 256, 0, s>>>(e.buf.p, e.site_size(), e.csize(), e.cell.nsites(), G.p);
  count_launch();
  double tol = std::max(1e-14, 10.0 * std::sqrt(double(e.chi)) * 2.220446049250313e-16);
  jacobi_svd_colmajor(G.p, e.chi, e.chi, nullptr, s, tol, 60, nmat);
  spectra_kernel<<<nmat, 128, e.chi * sizeof(double), s>>>(G.p, e.chi, e.spectra.p);
  count_launch();
  check_launch("corner_spectra");
  e.have_spectra = true;
}

double spectra_change(const double *a, const double *b, int nmat, int chi, cudaStream_t s, const int *count_dev,
                      int *count_host) {
  DBuf d(size_t(nmat), s);
  spectra_diff_kernel<<<nmat, 256, 0, s>>>(a, b, chi, d.p);
  count_launch();
  check_launch("spectra_diff");
  std::vector<double> h(nmat);
  IPEPS_CUDA(cudaMemcpyAsync(h.data(), d.p, nmat * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (count_dev) IPEPS_CUDA(cudaMemcpyAsync(count_host, count_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  IPEPS_CUDA(stream_sync(s));
  return *std::max_element(h.begin(), h.end());
}

// ------------------------------------------------------------------- run
int ctmrg_run(EnvImpl &e, const double *A_dev, double tol, int maxit, Prec prec, double *err,
              cudaStream_t s) {
  const Cell &c = e.cell;
  const int nmat = 4 * c.nsites();
  if (!e.have_spectra) corner_spectra(e, s);
  DBuf prev(size_t(nmat) * e.chi, s);
  DBuf bad_buf(1, s);
  int *bad_dev = reinterpret_cast<int *>(bad_buf.p);
  double change = INFINITY;
  // split precision: 3xTF32 iterations while the change is above the split
  // floor and still improving, then (TF32X3) FP64 iterations down to tol
  Prec phase = prec;
  double best = INFINITY;
  int since_best = 0;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    const Prec prec = phase;
    IPEPS_CUDA(cudaMemcpyAsync(prev.p, e.spectra.p, nmat * e.chi * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    {
      Tape t(s);
      t.record = false;
      t.prec = prec;
      t.vcache = &e.svd_cache;
      StateVars sv = state_leaves(t, e, A_dev);
      ctmrg_iteration(t, c, e.chi, sv);
      // align the sign gauge of every chi bond with the previous iteration, so
      // that the environment (and the warm starts of the projector SVDs)
      // converge elementwise
      std::vector<const double *> cand(8 * c.nsites());
      for (int n = 0; n < 8; ++n)
        for (int i = 0; i < c.nsites(); ++i) cand[n * c.nsites() + i] = t.vp(sv.env[n][i]);
      double res = 0.0;
      DBuf sig = solve_signs(e, cand, s, &res);
      const int64_t D2 = int64_t(c.D) * c.D;
      for (int n = 0; n < 8; ++n)
        for (int i = 0; i < c.nsites(); ++i) {
          int k = n * c.nsites() + i;
          leg_signs(t.vp(sv.env[n][i]), e.chi, n < 4 ? 1 : D2, e.chi, sig.p + int64_t(2 * k) * e.chi,
                    sig.p + int64_t(2 * k + 1) * e.chi, s);
        }
      // new tensors into a staging buffer, then over the old ones
      DBuf nb(size_t(e.total()), s);
      for (int n = 0; n < 8; ++n)
        for (int i = 0; i < c.nsites(); ++i) {
          int x = i / c.Ly, y = i % c.Ly;
          int64_t sz = (n < 4) ? e.csize() : e.esize();
          IPEPS_CUDA(cudaMemcpyAsync(nb.p + e.offset(n, x, y), t.vp(sv.env[n][i]), sz * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
        }
      std::swap(e.buf, nb);
      // non-finite entries are counted on the device and read with the spectra change below
      count_nonfinite(e.total(), e.buf.p, bad_dev, s);
      if (std::getenv("IPEPS_DEBUG_NAN")) {
        int *cnt = static_cast<int *>(dev_alloc(sizeof(int), s));
        for (int n = 0; n < 8; ++n)
          for (int i = 0; i < c.nsites(); ++i) {
            int x = i / c.Ly, y = i % c.Ly, bad = 0;
            count_nonfinite(n < 4 ? e.csize() : e.esize(), e.ptr(n, x, y), cnt, s);
            IPEPS_CUDA(cudaMemcpyAsync(&bad, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
            IPEPS_CUDA(stream_sync(s));
            if (bad) std::fprintf(stderr, "[ipeps] ctmrg it %d: tensor %d site %d has %d non-finite entries\n", it, n, i, bad);
          }
        dev_free(cnt, s);
      }
    }
    corner_spectra(e, s);
    int bad = 0;
    change = spectra_change(prev.p, e.spectra.p, nmat, e.chi, s, bad_dev, &bad);
    if (bad) throw Error(IPEPS_ERR_NONFINITE, "CTMRG produced non-finite environment tensors");
    if (!std::isfinite(change)) throw Error(IPEPS_ERR_NONFINITE, "CTMRG produced non-finite values");
    if (change < tol && it >= 2) break;
    if (change < 0.7 * best) { best = change; since_best = 0; }
    else ++since_best;
    if (phase == Prec::TF32X3 && (change < kSplitSwitch || since_best >= 10)) phase = Prec::FP64;
    // BF16x3 iterations likewise hand over to FP64-grade tensor-core iterations
    if (phase == Prec::BF16X3 && (change < kSplitSwitch || since_best >= 10)) phase = Prec::FP64_TC;
    if (phase == Prec::TF32X3_ALL && since_best >= 10) break;  // at the noise floor
  }
  e.prec = phase;
  if (it > maxit) it = maxit;
  if (err) *err = change;
  return it;
}

// ------------------------------------------------------------------- gauge
namespace {
__global__ void overlap_kernel(const double *ref, const double *cand, int64_t chi, int64_t mid,
                               double *W) {
  // one block per row i; W[i, j] = sum_m ref[i, m, j] cand[i, m, j]
  int64_t i = blockIdx.x;
  for (int64_t j = threadIdx.x; j < chi; j += blockDim.x) {
    double a = 0.0;
    for (int64_t m = 0; m < mid; ++m) {
      int64_t o = (i * mid + m) * chi + j;
      a += ref[o] * cand[o];
    }
    W[i * chi + j] = a;
  }
}

// (prev bond, next bond) of every boundary tensor: a bond is (side, a, b)
std::pair<std::tuple<int, int, int>, std::tuple<int, int, int>> bond_of(int n, int x, int y, int Lx,
                                                                        int Ly) {
  const int xp = (x + 1) % Lx, yp = (y + 1) % Ly;
  enum { L = 0, T = 1, R = 2, B = 3 };
  switch (n) {
    case C1: return {{L, x, y}, {T, x, y}};
    case T1: return {{T, x, y}, {T, xp, y}};
    case C2: return {{T, xp, y}, {R, x, y}};
    case T2: return {{R, x, y}, {R, x, yp}};
    case C3: return {{R, x, yp}, {B, xp, y}};
    case T3: return {{B, xp, y}, {B, x, y}};
    case C4: return {{B, x, y}, {L, x, yp}};
    default: return {{L, x, yp}, {L, x, y}};  // T4
  }
}
}  // namespace

DBuf solve_signs(const EnvImpl &ref, const std::vector<const double *> &cand, cudaStream_t s,
                 double *residual) {
  const Cell &c = ref.cell;
  const int chi = ref.chi, ns = c.nsites();
  const int64_t D2 = int64_t(c.D) * c.D;
  std::vector<std::vector<double>> W(8 * ns);
  {
    DBuf Wd(size_t(8) * ns * chi * chi, s);
    for (int n = 0; n < 8; ++n)
      for (int i = 0; i < ns; ++i) {
        int x = i / c.Ly, y = i % c.Ly;
        overlap_kernel<<<chi, 128, 0, s>>>(ref.ptr(n, x, y), cand[n * ns + i], chi, n < 4 ? 1 : D2,
                                           Wd.p + int64_t(n * ns + i) * chi * chi);
        count_launch();
      }
    check_launch("overlap");
    std::vector<double> h(size_t(8) * ns * chi * chi);
    IPEPS_CUDA(cudaMemcpyAsync(h.data(), Wd.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    IPEPS_CUDA(stream_sync(s));
    for (int k = 0; k < 8 * ns; ++k)
      W[k].assign(h.begin() + int64_t(k) * chi * chi, h.begin() + int64_t(k + 1) * chi * chi);
  }
  // nodes (bond, index); maximum-weight spanning forest of the sign constraints
  std::map<std::tuple<int, int, int>, int> bid;
  std::vector<std::pair<int, int>> tb(8 * ns);
  for (int n = 0; n < 8; ++n)
    for (int i = 0; i < ns; ++i) {
      auto b = bond_of(n, i / c.Ly, i % c.Ly, c.Lx, c.Ly);
      for (auto key : {b.first, b.second})
        if (!bid.count(key)) {
          int id = int(bid.size());
          bid[key] = id;
        }
      tb[n * ns + i] = {bid[b.first], bid[b.second]};
    }
  const int nb = int(bid.size());
  struct Edge { double w; int to; double s; };
  std::vector<std::vector<Edge>> adj(size_t(nb) * chi);
  std::vector<double> best(size_t(nb) * chi, 0.0);
  for (int k = 0; k < 8 * ns; ++k) {
    int bp = tb[k].first, bn = tb[k].second;
    for (int i = 0; i < chi; ++i)
      for (int j = 0; j < chi; ++j) {
        double w = W[k][i * chi + j];
        if (w == 0.0 || (bp == bn && i == j)) continue;
        int a = bp * chi + i, b = bn * chi + j;
        double sg = w > 0 ? 1.0 : -1.0;
        adj[a].push_back({std::fabs(w), b, sg});
        adj[b].push_back({std::fabs(w), a, sg});
        best[a] = std::max(best[a], std::fabs(w));
        best[b] = std::max(best[b], std::fabs(w));
      }
  }
  std::vector<double> val(size_t(nb) * chi, 0.0);
  std::vector<int> order(size_t(nb) * chi);
  for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return best[a] > best[b]; });
  using QE = std::tuple<double, int, double, int>;  // weight, node, sign, from
  for (int root : order) {
    if (val[root] != 0.0) continue;
    val[root] = 1.0;
    std::priority_queue<QE> pq;
    for (auto &e : adj[root]) pq.emplace(e.w, e.to, e.s, root);
    while (!pq.empty()) {
      auto [w, nd, sg, from] = pq.top();
      pq.pop();
      if (val[nd] != 0.0) continue;
      val[nd] = sg * val[from];
      for (auto &e : adj[nd])
        if (val[e.to] == 0.0) pq.emplace(e.w, e.to, e.s, nd);
    }
  }
  // per tensor (prev signs, next signs)
  std::vector<double> hs(size_t(8) * ns * 2 * chi);
  double res = 0.0;
  for (int k = 0; k < 8 * ns; ++k) {
    int bp = tb[k].first, bn = tb[k].second;
    for (int i = 0; i < chi; ++i) {
      hs[(size_t(k) * 2) * chi + i] = val[bp * chi + i];
      hs[(size_t(k) * 2 + 1) * chi + i] = val[bn * chi + i];
    }
    // |ref|^2 - 2 <ref, s.cand> + |cand|^2 = 2 - 2 sum_ij s_i s_j W_ij for unit tensors
    double ov = 0.0;
    for (int i = 0; i < chi; ++i)
      for (int j = 0; j < chi; ++j) ov += val[bp * chi + i] * val[bn * chi + j] * W[k][i * chi + j];
    res = std::max(res, std::sqrt(std::max(0.0, 2.0 - 2.0 * ov)));
  }
  if (residual) *residual = res;
  // pageable source: the call returns once hs is staged, so hs may go out of scope
  DBuf out(hs.size(), s);
  IPEPS_CUDA(cudaMemcpyAsync(out.p, hs.data(), hs.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  return out;
}

}  // namespace ipeps
