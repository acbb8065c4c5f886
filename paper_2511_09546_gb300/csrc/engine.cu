// Contraction engine and reverse-mode tape (see engine.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <chrono>
#include <cstdio>
#include <typeinfo>
#include <cstdlib>

#include "common.h"
#include "engine.h"
#include "kernels.h"

namespace ipeps {

// ------------------------------------------------------------------ contract
// The tensor-core path pads M and N to 128 and K to 32 and adds a pack pass;
// below a few million multiply-adds, or when padding would waste more than
// half of the tile, the FP64 kernels are faster and exact.
bool tc_worthwhile(int64_t m, int64_t n, int64_t k) {
  if (m < 64 || n < 64 || k < 32) return false;
  const double mp = double((m + 127) / 128 * 128), np = double((n + 127) / 128 * 128);
  const double kp = double((k + 31) / 32 * 32);
  return double(m) * n * k >= double(1 << 24) && double(m) * n * k >= 0.5 * mp * np * kp;
}

void contract(const Ten &A, const std::string &la, const Ten &B, const std::string &lb, const Ten &C,
              const std::string &lc, cudaStream_t s, double alpha, double beta, Prec prec) {
  IPEPS_REQUIRE(la.size() == A.d.size() && lb.size() == B.d.size() && lc.size() == C.d.size(),
                "contract: label/rank mismatch " + la + "," + lb + "->" + lc);
  std::map<char, int64_t> dim;
  auto note = [&](const std::string &l, const Ten &T) {
    for (size_t i = 0; i < l.size(); ++i) {
      auto it = dim.find(l[i]);
      if (it == dim.end()) dim[l[i]] = T.d[i];
      else IPEPS_REQUIRE(it->second == T.d[i], std::string("contract: size mismatch on ") + l[i]);
    }
  };
  note(la, A); note(lb, B); note(lc, C);
  std::string K, FA, FB;
  for (char c : la) {
    bool inb = lb.find(c) != std::string::npos, inc = lc.find(c) != std::string::npos;
    IPEPS_REQUIRE(inb != inc, std::string("contract: label ") + c + " must be in exactly one of B, C");
    (inb ? K : FA) += c;
  }
  for (char c : lb) {
    bool ina = la.find(c) != std::string::npos, inc = lc.find(c) != std::string::npos;
    IPEPS_REQUIRE(ina != inc, std::string("contract: label ") + c + " must be in exactly one of A, C");
    if (inc) FB += c;
  }
  IPEPS_REQUIRE(FA.size() + FB.size() == lc.size(), "contract: output labels");
  auto dprod = [&](const std::string &l) {
    int64_t n = 1;
    for (char c : l) n *= dim[c];
    return n;
  };
  auto dims_of = [&](const std::string &l) {
    std::vector<int64_t> v;
    for (char c : l) v.push_back(dim[c]);
    return v;
  };
  auto perm_to = [&](const std::string &from, const std::string &to) {
    std::vector<int> p;
    for (char c : to) p.push_back(int(from.find(c)));
    return p;
  };
  const int64_t m = dprod(FA), n = dprod(FB), k = dprod(K);
  if (m == 0 || n == 0) return;

  bool ta = false, tb = false;
  const double *Ap = A.p, *Bp = B.p;
  DBuf Ab, Bb, Cb;
  int64_t lda, ldb;
  if (la == FA + K) { lda = k; }
  else if (la == K + FA) { ta = true; lda = m; }
  else {
    Ab = DBuf(size_t(m * k), s);
    permute(A.p, A.d, perm_to(la, FA + K), Ab.p, s);
    Ap = Ab.p; lda = k;
  }
  if (lb == K + FB) { ldb = n; }
  else if (lb == FB + K) { tb = true; ldb = k; }
  else {
    Bb = DBuf(size_t(k * n), s);
    permute(B.p, B.d, perm_to(lb, K + FB), Bb.p, s);
    Bp = Bb.p; ldb = n;
  }
  const bool direct = (lc == FA + FB);
  double *Cp = C.p;
  if (!direct) {
    Cb = DBuf(size_t(m * n), s);
    Cp = Cb.p;
  }
  double ga = direct ? alpha : 1.0, gb = direct ? beta : 0.0;
  if ((prec == Prec::TF32X3 || prec == Prec::TF32X3_ALL) && tc_worthwhile(m, n, k))
    gemm_tf32x3(ta, tb, m, n, k, ga, Ap, lda, Bp, ldb, gb, Cp, n, s);
  else if (prec == Prec::BF16X3 && oz_worthwhile(m, n, k))
    gemm_oz(2, ta, tb, m, n, k, ga, Ap, lda, Bp, ldb, gb, Cp, n, s);
  else if (prec == Prec::FP64_TC && oz_worthwhile(m, n, k))
    gemm_oz(8, ta, tb, m, n, k, ga, Ap, lda, Bp, ldb, gb, Cp, n, s);
  else
    gemm_f64(ta, tb, m, n, k, ga, Ap, lda, Bp, ldb, gb, Cp, n, s);
  if (!direct) permute(Cp, dims_of(FA + FB), perm_to(FA + FB, lc), C.p, s, alpha, beta);
}

// ---------------------------------------------------------------------- tape
int Tape::leaf(double *p, const std::vector<int64_t> &d) {
  Var v;
  v.val.p = p;
  v.val.d = d;
  vars.push_back(std::move(v));
  return int(vars.size()) - 1;
}

int Tape::make(const std::vector<int64_t> &d) {
  Var v;
  v.own = DBuf(size_t(prod(d)), s);
  v.val.p = v.own.p;
  v.val.d = d;
  vars.push_back(std::move(v));
  return int(vars.size()) - 1;
}

double *Tape::grad(int id, bool create) {
  while (vars[id].alias >= 0) id = vars[id].alias;
  Var &v = vars[id];
  if (!v.grad.p && create) {
    v.grad = DBuf(size_t(v.val.size()), s);
    fill(v.grad.p, v.val.size(), 0.0, s);
  }
  return v.grad.p;
}

void Tape::zero_grads() {
  for (auto &v : vars)
    if (v.grad.p) fill(v.grad.p, v.val.size(), 0.0, s);
}

void Tape::backward() {
  static const bool dbg = std::getenv("IPEPS_DEBUG_NAN") != nullptr;
  int idx = int(nodes.size());
  for (auto it = nodes.rbegin(); it != nodes.rend(); ++it) {
    --idx;
    auto t0 = std::chrono::steady_clock::now();
    (*it)->backward(*this);
    if (dbg) {
      // report the first node whose adjoint produced a non-finite cotangent
      int *cnt = static_cast<int *>(dev_alloc(sizeof(int), s));
      int bad = 0;
      for (size_t v = 0; v < vars.size() && !bad; ++v) {
        if (!vars[v].grad.p) continue;
        count_nonfinite(vars[v].val.size(), vars[v].grad.p, cnt, s);
        IPEPS_CUDA(cudaMemcpyAsync(&bad, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        IPEPS_CUDA(stream_sync(s));
        if (bad) std::fprintf(stderr, "[ipeps] non-finite cotangent after node %d (%s), var %zu\n", idx,
                              typeid(**it).name(), v);
      }
      dev_free(cnt, s);
      double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (ms > 50.0) std::fprintf(stderr, "[ipeps] node %d (%s) backward %.1f ms\n", idx, typeid(**it).name(), ms);
      if (bad) throw Error(IPEPS_ERR_NONFINITE, "non-finite cotangent in the adjoint");
    }
  }
}

void Tape::clear() {
  nodes.clear();
  vars.clear();
}

void Tape::release(int id) {
  if (record) return;
  while (vars[id].alias >= 0) id = vars[id].alias;
  vars[id].own.release();
}

namespace {

Ten gten(Tape &t, int id, double *g) { return Ten{g, t.val(id).d}; }

struct ContractNode : Node {
  int a, b, c;
  std::string la, lb, lc;
  void backward(Tape &t) override {
    double *gc = t.grad(c, false);
    if (!gc) return;
    Ten GC = gten(t, c, gc);
    contract(GC, lc, t.val(b), lb, gten(t, a, t.grad(a)), la, t.s, 1.0, 1.0, t.prec);
    contract(t.val(a), la, GC, lc, gten(t, b, t.grad(b)), lb, t.s, 1.0, 1.0, t.prec);
  }
};

struct PermuteNode : Node {
  int a, y;
  std::vector<int> perm;
  void backward(Tape &t) override {
    double *gy = t.grad(y, false);
    if (!gy) return;
    std::vector<int> inv(perm.size());
    for (size_t i = 0; i < perm.size(); ++i) inv[perm[i]] = int(i);
    permute(gy, t.val(y).d, inv, t.grad(a), t.s, 1.0, 1.0);
  }
};

struct ScaleColsNode : Node {
  int X, f, Y;
  int64_t m, n;
  void backward(Tape &t) override {
    double *gy = t.grad(Y, false);
    if (!gy) return;
    scale_cols(m, n, gy, t.vp(f), t.grad(X), t.s, 1.0);
    DBuf tmp(size_t(n), t.s);
    coldot(m, n, gy, t.vp(X), tmp.p, t.s);
    axpy(n, 1.0, tmp.p, t.grad(f), t.s);
  }
};

__global__ void inv_sqrt_cut_fwd(const double *S, double *F, int n, double cutoff) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double s = S[i];
    F[i] = (s > cutoff * S[0]) ? 1.0 / sqrt(s) : 0.0;
  }
}
__global__ void inv_sqrt_cut_bwd(const double *S, const double *gF, double *gS, int n, double cutoff) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double s = S[i];
    if (s > cutoff * S[0]) gS[i] += gF[i] * (-0.5) / (s * sqrt(s));
  }
}

struct InvSqrtNode : Node {
  int S, F;
  double cutoff;
  void backward(Tape &t) override {
    double *gF = t.grad(F, false);
    if (!gF) return;
    int n = int(t.val(S).size());
    inv_sqrt_cut_bwd<<<(n + 255) / 256, 256, 0, t.s>>>(t.vp(S), gF, t.grad(S), n, cutoff);
    count_launch();
    check_launch("inv_sqrt_cut_bwd");
  }
};

__global__ void normalize_bwd(int64_t n, const double *y, const double *gy, const double *ydotg,
                              const double *nrm, double *gx) {
  double a = *ydotg, inv = 1.0 / (*nrm);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    gx[i] += (gy[i] - y[i] * a) * inv;
}

struct NormalizeNode : Node {
  int x, y;
  DBuf nrm;
  void backward(Tape &t) override {
    double *gy = t.grad(y, false);
    if (!gy) return;
    int64_t n = t.val(y).size();
    DBuf d(1, t.s);
    dot(n, t.vp(y), gy, d.p, t.s);
    normalize_bwd<<<512, 256, 0, t.s>>>(n, t.vp(y), gy, d.p, nrm.p, t.grad(x));
    count_launch();
    check_launch("normalize_bwd");
  }
};

struct SignsNode : Node {
  int x, y;
  int64_t a, mid, b;
  DBuf sp, sn;
  void backward(Tape &t) override {
    double *gy = t.grad(y, false);
    if (!gy) return;
    int64_t n = a * mid * b;
    DBuf tmp(size_t(n), t.s);
    IPEPS_CUDA(cudaMemcpyAsync(tmp.p, gy, n * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
    leg_signs(tmp.p, a, mid, b, sp.p, sn.p, t.s);
    axpy(n, 1.0, tmp.p, t.grad(x), t.s);
  }
};

// inner matrix of the SVD adjoint, split into top (k x N) and bottom ((N-k) x k)
__global__ void svd_inner_kernel(const double *A1, const double *B1, const double *S, const double *gS,
                                 int64_t N, int64_t k, double *top, double *bot) {
  int64_t total = k * N + (N - k) * k;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i, j;
    if (e < k * N) { i = e / N; j = e % N; }
    else { int64_t f = e - k * N; i = k + f / k; j = f % k; }
    double v = 0.0;
    if (i == j) {
      v = gS ? gS[i] : 0.0;
    } else {
      double si = S[i], sj = S[j];
      double diff = sj * sj - si * si;
      if (diff != 0.0) {
        double a = (j < k ? A1[i * k + j] : 0.0) - (i < k ? A1[j * k + i] : 0.0);
        double b = (j < k ? B1[i * k + j] : 0.0) - (i < k ? B1[j * k + i] : 0.0);
        v = (a * sj + si * b) / diff;
      }
    }
    if (e < k * N) top[e] = v;
    else bot[e - k * N] = v;
  }
}

struct SVDNode : Node {
  int M, U, S, V;
  int64_t N, k;
  DBuf Uf, Sf, Vf;  // complete bases, row-major N x N, and all N singular values
  void backward(Tape &t) override {
    double *gU = t.grad(U, false), *gS = t.grad(S, false), *gV = t.grad(V, false);
    if (!gU && !gS && !gV) return;
    cudaStream_t s = t.s;
    DBuf A1(size_t(N * k), s), B1(size_t(N * k), s);
    if (gU) gemm_f64(true, false, N, k, N, 1.0, Uf.p, N, gU, k, 0.0, A1.p, k, s);
    else fill(A1.p, N * k, 0.0, s);
    if (gV) gemm_f64(true, false, N, k, N, 1.0, Vf.p, N, gV, k, 0.0, B1.p, k, s);
    else fill(B1.p, N * k, 0.0, s);
    DBuf top(size_t(k * N), s), bot(size_t((N - k) * k + 1), s);
    svd_inner_kernel<<<512, 256, 0, s>>>(A1.p, B1.p, Sf.p, gS, N, k, top.p, bot.p);
    count_launch();
    check_launch("svd_inner");
    double *gM = t.grad(M);
    // gM += U[:, :k] (top V^T)
    DBuf T1(size_t(k * N), s);
    gemm_f64(false, true, k, N, N, 1.0, top.p, N, Vf.p, N, 0.0, T1.p, N, s);
    gemm_f64(false, false, N, N, k, 1.0, Uf.p, N, T1.p, N, 1.0, gM, N, s);
    if (N > k) {
      // gM += (U[:, k:] bot) V[:, :k]^T
      DBuf T2(size_t(N * k), s);
      gemm_f64(false, false, N, k, N - k, 1.0, Uf.p + k, N, bot.p, k, 0.0, T2.p, k, s);
      gemm_f64(false, true, N, N, k, 1.0, T2.p, k, Vf.p, N, 1.0, gM, N, s);
    }
  }
};

__global__ void rho_ratio_fwd(const double *rho, const double *h, int d, int two_site, double *num,
                              double *den, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double nu = 0.0, de = 0.0;
  if (two_site) {
    int dd = d * d;
    for (int k1 = 0; k1 < d; ++k1)
      for (int b1 = 0; b1 < d; ++b1)
        for (int k2 = 0; k2 < d; ++k2)
          for (int b2 = 0; b2 < d; ++b2) {
            double r = rho[((k1 * d + b1) * d + k2) * d + b2];
            nu += r * h[(b1 * d + b2) * dd + (k1 * d + k2)];
            if (k1 == b1 && k2 == b2) de += r;
          }
  } else {
    for (int k = 0; k < d; ++k)
      for (int b = 0; b < d; ++b) {
        double r = rho[k * d + b];
        nu += r * h[b * d + k];
        if (k == b) de += r;
      }
  }
  *num = nu;
  *den = de;
  *out = nu / de;
}

__global__ void rho_ratio_bwd(const double *h, int d, int two_site, const double *den,
                              const double *out, const double *gout, double *grho) {
  double g = *gout / *den, e = *out;
  if (two_site) {
    int dd = d * d, n = dd * dd;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int b2 = idx % d, k2 = (idx / d) % d, b1 = (idx / dd) % d, k1 = idx / (dd * d);
      double v = h[(b1 * d + b2) * dd + (k1 * d + k2)] - ((k1 == b1 && k2 == b2) ? e : 0.0);
      grho[idx] += g * v;
    }
  } else {
    for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
      int b = idx % d, k = idx / d;
      grho[idx] += g * (h[b * d + k] - (k == b ? e : 0.0));
    }
  }
}

struct RhoRatioNode : Node {
  int rho, out, d;
  bool two;
  const double *h;
  DBuf num, den;
  void backward(Tape &t) override {
    double *go = t.grad(out, false);
    if (!go) return;
    if (std::getenv("IPEPS_DEBUG_NAN")) {
      double hv[4];
      IPEPS_CUDA(cudaMemcpyAsync(hv, num.p, 8, cudaMemcpyDeviceToHost, t.s));
      IPEPS_CUDA(cudaMemcpyAsync(hv + 1, den.p, 8, cudaMemcpyDeviceToHost, t.s));
      IPEPS_CUDA(cudaMemcpyAsync(hv + 2, t.vp(out), 8, cudaMemcpyDeviceToHost, t.s));
      IPEPS_CUDA(cudaMemcpyAsync(hv + 3, go, 8, cudaMemcpyDeviceToHost, t.s));
      IPEPS_CUDA(stream_sync(t.s));
      std::fprintf(stderr, "[ipeps] rho_ratio num %.6e den %.6e out %.6e gout %.6e d %d two %d\n", hv[0], hv[1],
                   hv[2], hv[3], d, int(two));
    }
    rho_ratio_bwd<<<1, 256, 0, t.s>>>(h, d, two ? 1 : 0, den.p, t.vp(out), go, t.grad(rho));
    count_launch();
    check_launch("rho_ratio_bwd");
  }
};

__global__ void add_scaled_scalar(double *dst, const double *src, double scale) {
  if (threadIdx.x == 0 && blockIdx.x == 0) dst[0] += scale * src[0];
}

struct SumNode : Node {
  std::vector<int> xs;
  int out;
  double scale;
  void backward(Tape &t) override {
    double *go = t.grad(out, false);
    if (!go) return;
    for (int x : xs) {
      add_scaled_scalar<<<1, 32, 0, t.s>>>(t.grad(x), go, scale);
      count_launch();
    }
    check_launch("sum_bwd");
  }
};

// gather the sorted factors of a Jacobi SVD of M^T (see svd_full)
__global__ void svd_gather_kernel(const double *Gc, const double *Vg, const double *sig, const int *perm,
                                  int64_t N, double *U, double *V) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < N * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = e / N, jj = e % N;
    int64_t j = perm[jj];
    double u = Vg[j * N + i];
    U[e] = u;
    double sv = sig[j];
    // zero singular value: the left null vector is a coordinate vector of a
    // padded index, which is also a right null vector (padding is symmetric)
    V[e] = sv > 0.0 ? Gc[j * N + i] / sv : u;
  }
}

__global__ void colnorm_contig(const double *G, int64_t m, double *out) {
  int64_t j = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    double v = G[j * m + i];
    acc += v * v;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sqrt(sh[0]);
}

// flip column j of U and V (row-major N x ncols, j < k) so that the entry of U
// with the largest magnitude is positive
// uniform [-1, 1) from a counter hash (splitmix64 finaliser) of (seed, index)
__global__ void random_fill_kernel(double *p, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    uint64_t z = seed + uint64_t(i) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    p[i] = double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

__global__ void svd_sign_kernel(double *U, double *V, int64_t N, int64_t ncols) {
  int64_t j = blockIdx.x;
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  double best = -1.0;
  int64_t arg = 0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    double a = fabs(U[i * ncols + j]);
    if (a > best) { best = a; arg = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = bv[threadIdx.x + s];
      int64_t oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  double sg = U[bi[0] * ncols + j] < 0.0 ? -1.0 : 1.0;
  if (sg < 0.0)
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
      U[i * ncols + j] = -U[i * ncols + j];
      V[i * ncols + j] = -V[i * ncols + j];
    }
}

__global__ void copy_cols_kernel(const double *src, int64_t N, int64_t ldsrc, int64_t k, double *dst) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < N * k;
       e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = src[(e / k) * ldsrc + e % k];
}

}  // namespace

void svd_full(const double *M, int64_t N, double *U, double *S, double *V, cudaStream_t s) {
  // One-sided Jacobi on the columns of G = M^T (the row-major M read column-major):
  // G Vg = Gc (orthogonal columns)  =>  M = Vg diag(sig) (Gc / sig)^T.
  DBuf G(size_t(N * N), s), Vg(size_t(N * N), s), sig(size_t(N), s);
  IPEPS_CUDA(cudaMemcpyAsync(G.p, M, N * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double tol = std::max(1e-14, 10.0 * std::sqrt(double(N)) * 2.220446049250313e-16);
  jacobi_svd_colmajor(G.p, N, N, Vg.p, s, tol, 60, 1);
  colnorm_contig<<<unsigned(N), 256, 0, s>>>(G.p, N, sig.p);
  count_launch();
  std::vector<double> hs(N);
  IPEPS_CUDA(cudaMemcpyAsync(hs.data(), sig.p, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  IPEPS_CUDA(stream_sync(s));
  std::vector<int> perm(N);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return hs[a] > hs[b]; });
  std::vector<double> sorted(N);
  for (int64_t i = 0; i < N; ++i) sorted[i] = hs[perm[i]];
  int *dperm = static_cast<int *>(dev_alloc(N * sizeof(int), s));
  IPEPS_CUDA(cudaMemcpyAsync(dperm, perm.data(), N * sizeof(int), cudaMemcpyHostToDevice, s));
  IPEPS_CUDA(cudaMemcpyAsync(S, sorted.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  svd_gather_kernel<<<512, 256, 0, s>>>(G.p, Vg.p, sig.p, dperm, N, U, V);
  count_launch();
  check_launch("svd_gather");
  IPEPS_CUDA(stream_sync(s));  // host vectors above go out of scope
  dev_free(dperm, s);
}

// ------------------------------------------------------------- primitives
int t_contract(Tape &t, int a, const std::string &la, int b, const std::string &lb,
               const std::string &lc) {
  std::map<char, int64_t> dim;
  for (size_t i = 0; i < la.size(); ++i) dim[la[i]] = t.val(a).d[i];
  for (size_t i = 0; i < lb.size(); ++i) dim[lb[i]] = t.val(b).d[i];
  std::vector<int64_t> dc;
  for (char c : lc) dc.push_back(dim.at(c));
  int c = t.make(dc);
  contract(t.val(a), la, t.val(b), lb, t.val(c), lc, t.s, 1.0, 0.0, t.prec);
  auto *n = new ContractNode;
  n->a = a; n->b = b; n->c = c; n->la = la; n->lb = lb; n->lc = lc;
  t.push(n);
  return c;
}

int t_reshape(Tape &t, int a, const std::vector<int64_t> &d) {
  IPEPS_REQUIRE(prod(d) == t.val(a).size(), "reshape: size mismatch");
  Var v;
  v.val.p = t.val(a).p;
  v.val.d = d;
  v.alias = a;
  t.vars.push_back(std::move(v));
  return int(t.vars.size()) - 1;
}

int t_permute(Tape &t, int a, const std::vector<int> &perm) {
  std::vector<int64_t> d;
  for (int p : perm) d.push_back(t.val(a).d[p]);
  int y = t.make(d);
  permute(t.vp(a), t.val(a).d, perm, t.vp(y), t.s);
  auto *n = new PermuteNode;
  n->a = a; n->y = y; n->perm = perm;
  t.push(n);
  return y;
}

int t_scale_cols(Tape &t, int X, int f) {
  int64_t n = t.val(f).size();
  int64_t m = t.val(X).size() / n;
  int Y = t.make(t.val(X).d);
  scale_cols(m, n, t.vp(X), t.vp(f), t.vp(Y), t.s);
  auto *nd = new ScaleColsNode;
  nd->X = X; nd->f = f; nd->Y = Y; nd->m = m; nd->n = n;
  t.push(nd);
  return Y;
}

int t_inv_sqrt_cut(Tape &t, int S, double cutoff) {
  int n = int(t.val(S).size());
  int F = t.make({int64_t(n)});
  inv_sqrt_cut_fwd<<<(n + 255) / 256, 256, 0, t.s>>>(t.vp(S), t.vp(F), n, cutoff);
  count_launch();
  check_launch("inv_sqrt_cut_fwd");
  auto *nd = new InvSqrtNode;
  nd->S = S; nd->F = F; nd->cutoff = cutoff;
  t.push(nd);
  return F;
}

int t_normalize(Tape &t, int x) {
  int64_t n = t.val(x).size();
  int y = t.make(t.val(x).d);
  auto *nd = new NormalizeNode;
  nd->nrm = DBuf(1, t.s);
  nrm2(n, t.vp(x), nd->nrm.p, t.s);
  IPEPS_CUDA(cudaMemcpyAsync(t.vp(y), t.vp(x), n * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
  div_by_scalar(n, t.vp(y), nd->nrm.p, t.s);
  nd->x = x; nd->y = y;
  t.push(nd);
  return y;
}

int t_signs(Tape &t, int x, const double *sp, const double *sn) {
  const auto &d = t.val(x).d;
  int64_t a = d.front(), b = d.back();
  int64_t mid = t.val(x).size() / (a * b);
  int y = t.make(d);
  IPEPS_CUDA(cudaMemcpyAsync(t.vp(y), t.vp(x), t.val(x).size() * sizeof(double),
                             cudaMemcpyDeviceToDevice, t.s));
  leg_signs(t.vp(y), a, mid, b, sp, sn, t.s);
  auto *nd = new SignsNode;
  nd->x = x; nd->y = y; nd->a = a; nd->mid = mid; nd->b = b;
  nd->sp = DBuf(size_t(a), t.s);
  nd->sn = DBuf(size_t(b), t.s);
  IPEPS_CUDA(cudaMemcpyAsync(nd->sp.p, sp, a * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
  IPEPS_CUDA(cudaMemcpyAsync(nd->sn.p, sn, b * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
  t.push(nd);
  return y;
}

void t_svd(Tape &t, int M, int k, int *U, int *S, int *V) {
  const auto &d = t.val(M).d;
  IPEPS_REQUIRE(d.size() == 2 && d[0] == d[1], "t_svd: square matrix expected");
  int64_t N = d[0];
  IPEPS_REQUIRE(k >= 1 && k <= N, "t_svd: bad rank");
  int64_t kb = std::min<int64_t>(N, ((k + std::max(16, k / 4)) + 1) / 2 * 2);
  if (kb % 2) --kb;
  if (t.vcache && kb >= k && kb < N && N > 256) {
    // truncated SVD: warm-started subspace iteration over a kb-block; a cold
    // start (or a rank-deficient block) takes the full Jacobi SVD once and
    // seeds the warm start from it
    DBuf &vc = (*t.vcache)[t.vkey];
    const size_t csz = size_t(N * kb + kb);
    bool warm = vc.p != nullptr && vc.n == csz;
    if (!warm && N > 1024) {
      // cold start of a large cut: randomised range finder (random block, unit
      // scales) instead of the full Jacobi SVD of an N x N matrix
      vc = DBuf(csz, t.s);
      random_fill_kernel<<<512, 256, 0, t.s>>>(vc.p, N * kb, 0x9E3779B97F4A7C15ull + uint64_t(t.vkey));
      fill(vc.p + N * kb, kb, 1.0, t.s);
      count_launch();
      warm = true;
    }
    DBuf Ub(size_t(N * kb), t.s), Sb(size_t(kb), t.s), Vb(size_t(N * kb), t.s);
    int its = 0;
    bool ok = warm && svd_subspace(t.vp(M), N, k, int(kb), vc.p, Ub.p, Sb.p, Vb.p, t.s, &its,
                                   t.prec == Prec::TF32X3_ALL);
    t.svd_iters += its;
    if (!ok) {
      if (std::getenv("IPEPS_DEBUG"))
        std::fprintf(stderr, "[ipeps] t_svd key %d N %lld: full SVD (%s)\n", t.vkey, (long long)N,
                     warm ? "block failed" : "cold");
      DBuf Uf(size_t(N * N), t.s), Sf(size_t(N), t.s), Vf(size_t(N * N), t.s);
      svd_full(t.vp(M), N, Uf.p, Sf.p, Vf.p, t.s);
      copy_cols_kernel<<<256, 256, 0, t.s>>>(Uf.p, N, N, kb, Ub.p);
      copy_cols_kernel<<<256, 256, 0, t.s>>>(Vf.p, N, N, kb, Vb.p);
      count_launch(2);
      IPEPS_CUDA(cudaMemcpyAsync(Sb.p, Sf.p, kb * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
      if (!warm) vc = DBuf(csz, t.s);
      IPEPS_CUDA(cudaMemcpyAsync(vc.p, Vb.p, N * kb * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
      IPEPS_CUDA(cudaMemcpyAsync(vc.p + N * kb, Sb.p, kb * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
      IPEPS_CUDA(stream_sync(t.s));
    }
    svd_sign_kernel<<<unsigned(k), 256, 0, t.s>>>(Ub.p, Vb.p, N, kb);
    *U = t.make({N, int64_t(k)});
    *V = t.make({N, int64_t(k)});
    *S = t.make({int64_t(k)});
    copy_cols_kernel<<<256, 256, 0, t.s>>>(Ub.p, N, kb, k, t.vp(*U));
    copy_cols_kernel<<<256, 256, 0, t.s>>>(Vb.p, N, kb, k, t.vp(*V));
    count_launch(3);
    check_launch("t_svd block");
    IPEPS_CUDA(cudaMemcpyAsync(t.vp(*S), Sb.p, k * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
    if (t.record) push_trunc_svd_node(t, M, *U, *S, *V, N, k, int(kb), std::move(Ub), std::move(Sb), std::move(Vb));
    return;
  }
  auto *nd = new SVDNode;
  nd->N = N; nd->k = k; nd->M = M;
  nd->Uf = DBuf(size_t(N * N), t.s);
  nd->Vf = DBuf(size_t(N * N), t.s);
  nd->Sf = DBuf(size_t(N), t.s);
  svd_full(t.vp(M), N, nd->Uf.p, nd->Sf.p, nd->Vf.p, t.s);
  svd_sign_kernel<<<unsigned(k), 256, 0, t.s>>>(nd->Uf.p, nd->Vf.p, N, N);
  count_launch();
  *U = t.make({N, int64_t(k)});
  *V = t.make({N, int64_t(k)});
  *S = t.make({int64_t(k)});
  copy_cols_kernel<<<256, 256, 0, t.s>>>(nd->Uf.p, N, N, k, t.vp(*U));
  copy_cols_kernel<<<256, 256, 0, t.s>>>(nd->Vf.p, N, N, k, t.vp(*V));
  count_launch(2);
  check_launch("t_svd");
  IPEPS_CUDA(cudaMemcpyAsync(t.vp(*S), nd->Sf.p, k * sizeof(double), cudaMemcpyDeviceToDevice, t.s));
  nd->U = *U; nd->S = *S; nd->V = *V;
  t.push(nd);
}

int t_rho_ratio(Tape &t, int rho, const double *h_dev, int d, bool two_site) {
  int out = t.make({1});
  auto *nd = new RhoRatioNode;
  nd->num = DBuf(1, t.s);
  nd->den = DBuf(1, t.s);
  rho_ratio_fwd<<<1, 32, 0, t.s>>>(t.vp(rho), h_dev, d, two_site ? 1 : 0, nd->num.p, nd->den.p,
                                   t.vp(out));
  count_launch();
  check_launch("rho_ratio_fwd");
  nd->rho = rho; nd->out = out; nd->d = d; nd->two = two_site; nd->h = h_dev;
  t.push(nd);
  return out;
}

int t_sum_scalars(Tape &t, const std::vector<int> &xs, double scale) {
  int out = t.make({1});
  fill(t.vp(out), 1, 0.0, t.s);
  for (int x : xs) axpy(1, scale, t.vp(x), t.vp(out), t.s);
  auto *nd = new SumNode;
  nd->xs = xs; nd->out = out; nd->scale = scale;
  t.push(nd);
  return out;
}

}  // namespace ipeps
