// Energy per site from the environment (Eq. equ:energy): nearest-neighbour
// two-site density matrices of the 2 x 3 patches (horizontal bonds; vertical
// bonds are the horizontal bonds of the picture rotated by 90 degrees) and
// the single-site density matrix of the 3 x 3 patch, each normalised by its
// own trace.  Next-nearest-neighbour (J1-J2) terms use the two diagonal pairs
// of the 2 x 2 plaquette: the ring of its four enlarged corners (the ring the
// projectors are cut from) with the physical legs of the pair left open.
// Every step is recorded on the tape so that dE/dA and dE/denv come from the
// same pass.
#include "common.h"
#include "engine.h"
#include "ipeps_impl.h"

namespace ipeps {

HamDev::HamDev(const HamImpl &H, cudaStream_t s)
    : h(H.h.size(), s), v(H.v.size(), s), site(H.has_site ? H.site.size() : 0, s),
      d1(H.has_d1 ? H.d1.size() : 0, s), d2(H.has_d2 ? H.d2.size() : 0, s) {
  if (H.has_d1)
    IPEPS_CUDA(cudaMemcpyAsync(d1.p, H.d1.data(), H.d1.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  if (H.has_d2)
    IPEPS_CUDA(cudaMemcpyAsync(d2.p, H.d2.data(), H.d2.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  IPEPS_CUDA(cudaMemcpyAsync(h.p, H.h.data(), H.h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  IPEPS_CUDA(cudaMemcpyAsync(v.p, H.v.data(), H.v.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  if (H.has_site)
    IPEPS_CUDA(cudaMemcpyAsync(site.p, H.site.data(), H.site.size() * sizeof(double),
                               cudaMemcpyHostToDevice, s));
}

namespace {

struct Patch {
  Tape &t;
  const Cell &c;
  const StateVars &sv;
  Frame f;
  int E(int n, int x, int y) const {
    const int Lx = f.Lx(), Ly = f.Ly();
    x = ((x % Lx) + Lx) % Lx;
    y = ((y % Ly) + Ly) % Ly;
    int n0, x0, y0;
    f.resolve(n, x, y, &n0, &x0, &y0);
    return sv.env[n0][x0 * c.Ly + y0];
  }
  int A(int x, int y, int q = 0) const {
    const int Lx = f.Lx(), Ly = f.Ly();
    x = ((x % Lx) + Lx) % Lx;
    y = ((y % Ly) + Ly) % Ly;
    int x0, y0;
    f.resolve_site(x, y, &x0, &y0);
    return sv.A[(f.r + q) % 4][x0 * c.Ly + y0];
  }
  // upper-left enlarged corner C1 T1 T4 A Abar as [(T4.p, d, d'), (T1.n, r, r')],
  // or with the site's ket and bra physical legs open as [.., .., s, s']
  int corner(int c1, int t1, int t4, int a, bool open) const {
    int X1 = t_contract(t, c1, "ab", t1, "bcde", "acde");        // [C1.p, u, u', T1.n]
    int X2 = t_contract(t, t4, "fgha", X1, "acde", "fghcde");    // [T4.p, l, l', u, u', T1.n]
    int X3 = t_contract(t, X2, "fghcde", a, "scgjk", "fhdesjk"); // ket A on (u, l)
    if (!open) {
      int X4 = t_contract(t, X3, "fhdesjk", a, "sdhmn", "fjmekn");
      const auto &d = t.val(X4).d;
      return t_reshape(t, X4, {d[0] * d[1] * d[2], d[3] * d[4] * d[5]});
    }
    int X4 = t_contract(t, X3, "fhdesjk", a, "tdhmn", "fjmeknst");
    const auto &d = t.val(X4).d;
    return t_reshape(t, X4, {d[0] * d[1] * d[2], d[3] * d[4] * d[5], d[6], d[7]});
  }
  // rho[s1, s1', s2, s2'] of the plaquette with upper-left site (x, y):
  // which = 1 pairs (x, y) with (x+1, y+1), which = 2 pairs (x+1, y) with (x, y+1)
  int rho_diag(int x, int y, int which) const {
    const bool o1 = which == 1;
    int Qul = corner(E(C1, x, y), E(T1, x, y), E(T4, x, y), A(x, y, 0), o1);
    int Qur = corner(E(C2, x + 1, y), E(T2, x + 1, y), E(T1, x + 1, y), A(x + 1, y, 1), !o1);
    int Qlr = corner(E(C3, x + 1, y + 1), E(T3, x + 1, y + 1), E(T2, x + 1, y + 1), A(x + 1, y + 1, 2), o1);
    int Qll = corner(E(C4, x, y + 1), E(T4, x, y + 1), E(T3, x, y + 1), A(x, y + 1, 3), !o1);
    int R, Y;
    if (o1) {
      R = t_contract(t, Qul, "abst", Qur, "bc", "acst");
      Y = t_contract(t, Qlr, "ceuv", Qll, "ea", "cauv");
    } else {
      R = t_contract(t, Qul, "ab", Qur, "bcst", "acst");
      Y = t_contract(t, Qlr, "ce", Qll, "eauv", "cauv");
    }
    return t_contract(t, R, "acst", Y, "cauv", "stuv");
  }
  // left half of the patch of (x, y) with physical legs open: L[c, r, r', e, s, s']
  int left(int x, int y) const {
    int Lt = t_contract(t, E(C1, x, y), "ab", E(T1, x, y), "buvc", "auvc");
    int Lb = t_contract(t, E(T3, x, y), "edfh", E(C4, x, y), "hg", "edfg");
    int X = t_contract(t, Lt, "auvc", E(T4, x, y), "glma", "cuvlmg");
    X = t_contract(t, X, "cuvlmg", Lb, "edfg", "cuvlmdfe");
    X = t_contract(t, X, "cuvlmdfe", A(x, y), "suldr", "cvmfesr");
    return t_contract(t, X, "cvmfesr", A(x, y), "tvmfw", "crwest");
  }
  // right half of the patch of (x, y): R[c, l, l', e, s, s']
  int right(int x, int y) const {
    int Rt = t_contract(t, E(T1, x, y), "cuvh", E(C2, x, y), "hi", "cuvi");
    int Rb = t_contract(t, E(C3, x, y), "jk", E(T3, x, y), "kdfe", "jdfe");
    int X = t_contract(t, Rt, "cuvi", E(T2, x, y), "irwj", "cuvrwj");
    X = t_contract(t, X, "cuvrwj", Rb, "jdfe", "cuvrwdfe");
    X = t_contract(t, X, "cuvrwdfe", A(x, y), "suldr", "cvwfesl");
    return t_contract(t, X, "cvwfesl", A(x, y), "tvmfw", "clmest");
  }
};

}  // namespace

int energy_on_tape(Tape &t, const Cell &c, int chi, const StateVars &sv, const HamImpl &H,
                   const HamDev &hd) {
  (void)chi;
  std::vector<int> terms;
  Patch p0{t, c, sv, Frame{c.Lx, c.Ly, 0}};
  Patch p1{t, c, sv, Frame{c.Lx, c.Ly, 1}};
  for (int x = 0; x < c.Lx; ++x)
    for (int y = 0; y < c.Ly; ++y) {
      // horizontal bond (x, y)-(x+1, y)
      int L = p0.left(x, y);
      int R = p0.right(x + 1, y);
      int rho = t_contract(t, L, "cxyest", R, "cxyeuv", "stuv");
      terms.push_back(t_rho_ratio(t, rho, hd.h.p, c.d, true));
      // on-site term from the 3 x 3 patch
      if (H.has_site) {
        int RC = t_contract(t, p0.E(C2, x, y), "ci", p0.E(T2, x, y), "irwj", "crwj");
        RC = t_contract(t, RC, "crwj", p0.E(C3, x, y), "je", "crwe");
        int r1 = t_contract(t, L, "crwest", RC, "crwe", "st");
        terms.push_back(t_rho_ratio(t, r1, hd.site.p, c.d, false));
      }
      // vertical bond (x, y)-(x, y+1): in the rotated frame site (x, y) sits at
      // (y, -x mod Lx) and its lower neighbour is its right neighbour
      int xr = y, yr = ((-x) % c.Lx + c.Lx) % c.Lx;
      int Lv = p1.left(xr, yr);
      int Rv = p1.right(xr + 1, yr);
      int rv = t_contract(t, Lv, "cxyest", Rv, "cxyeuv", "stuv");
      terms.push_back(t_rho_ratio(t, rv, hd.v.p, c.d, true));
      // next-nearest neighbours across the plaquette with upper-left site (x, y)
      if (H.has_d1) terms.push_back(t_rho_ratio(t, p0.rho_diag(x, y, 1), hd.d1.p, c.d, true));
      if (H.has_d2) terms.push_back(t_rho_ratio(t, p0.rho_diag(x, y, 2), hd.d2.p, c.d, true));
    }
  return t_sum_scalars(t, terms, H.scale / double(c.nsites()));
}

}  // namespace ipeps
