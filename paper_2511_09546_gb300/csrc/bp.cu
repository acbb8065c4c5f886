// Mean-field (chi = 1) metric preconditioner (Sec. III.B: the local metric of
// Eq. equ:local_metric with environment bond dimension 1, the environment
// belief propagation gives; App. A compares it with the local metric).
//
// A message is a D x D matrix m[ket, bra] on one bond and direction.  Site s
// sends through leg lam the contraction of A_s, A_s (physical legs joined)
// and the messages arriving on its other three legs; every message of a sweep
// is computed from the previous sweep's, symmetrised and divided by its trace,
// starting from identity / D, until no entry changes by more than tol.  The
// message arriving on leg u of site (x, y) is the one (x, y-1) sends down
// (y grows downwards), on l the one (x-1, y) sends right, on d the one
// (x, y+1) sends up, on r the one (x+1, y) sends left.
//
// The metric of site s is N = 1_d (x) c m_u (x) m_l (x) m_d (x) m_r on
// A[p, u, l, d, r] with c <A|N/c|A> = 1, and (N + delta I)^-1 is applied
// exactly in the eigenbases of the four incoming messages: transform the
// vector leg by leg, divide by c lam_u lam_l lam_d lam_r + delta, transform
// back.  Every contraction is a single-leg mode product or a single-leg Gram
// matrix (D <= 32, d D^4 elements), written as its own kernel; the symmetric
// eigenproblems are one warp each (cyclic Jacobi).  All reductions run in a
// fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "bp.h"
#include "common.h"
#include "kernels.h"
#include "profile.h"

namespace ipeps {

namespace {

constexpr int kEigMaxSweeps = 60;

// message k = (x * Ly + y) * 4 + leg sent, legs u = 0, l = 1, d = 2, r = 3
int msg_index(const Cell &c, int x, int y, int leg) { return (x * c.Ly + y) * 4 + leg; }

// the message arriving at (x, y) on `leg`: sent by the neighbour on that side
// through the opposite leg
int incoming_index(const Cell &c, int x, int y, int leg) {
  static const int dx[4] = {0, -1, 0, 1}, dy[4] = {-1, 0, 1, 0}, opp[4] = {2, 3, 0, 1};
  const int nx = ((x + dx[leg]) % c.Lx + c.Lx) % c.Lx;
  const int ny = ((y + dy[leg]) % c.Ly + c.Ly) % c.Ly;
  return msg_index(c, nx, ny, opp[leg]);
}

// A[p, u, l, d, r] viewed as [outer, D, inner] around leg `leg`
void mode_dims(const Cell &c, int leg, int64_t *outer, int64_t *inner) {
  int64_t o = c.d, i = 1;
  for (int k = 0; k < leg; ++k) o *= c.D;
  for (int k = leg + 1; k < 4; ++k) i *= c.D;
  *outer = o;
  *inner = i;
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

__global__ void bp_init_kernel(double *m, int D, int nmsg) {
  const int64_t n = int64_t(nmsg) * D * D;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e % (int64_t(D) * D);
    m[e] = (r / D == r % D) ? 1.0 / D : 0.0;
  }
}

// y[o, a, i] = sum_u M[u, a] x[o, u, i]  (trans = 0)  or  sum_u M[a, u] x[o, u, i]  (trans = 1)
__global__ void mode_product_kernel(const double *__restrict__ x, double *__restrict__ y,
                                    const double *__restrict__ M, int D, int64_t outer, int64_t inner,
                                    int trans) {
  const int64_t n = outer * D * inner;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e % inner, t = e / inner;
    const int a = int(t % D);
    const int64_t o = t / D;
    const double *xp = x + o * D * inner + i;
    double acc = 0.0;
    for (int u = 0; u < D; ++u) acc = fma(trans ? M[a * D + u] : M[u * D + a], xp[u * inner], acc);
    y[e] = acc;
  }
}

// out[a, b] = sum_{o, i} X[o, a, i] Y[o, b, i]; one block of 128 threads per (a, b)
__global__ void __launch_bounds__(128) mode_gram_kernel(const double *__restrict__ X, const double *__restrict__ Y,
                                                        int D, int64_t outer, int64_t inner, double *out) {
  __shared__ double red[128];
  const int a = blockIdx.x / D, b = blockIdx.x % D;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < outer * inner; t += blockDim.x) {
    const int64_t o = t / inner, i = t % inner;
    acc = fma(X[(o * D + a) * inner + i], Y[(o * D + b) * inner + i], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 64; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// symmetrise each new message, divide by its trace; change[k] = max |new - old|
// (NaN when the trace is not positive or an entry is not finite)
__global__ void __launch_bounds__(64) bp_normalise_kernel(double *nw, const double *old, int D, double *change) {
  __shared__ double red[64];
  __shared__ double tr;
  double *m = nw + int64_t(blockIdx.x) * D * D;
  const double *o = old + int64_t(blockIdx.x) * D * D;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int i = e / D, j = e % D;
    if (i < j) {
      const double s = 0.5 * (m[i * D + j] + m[j * D + i]);
      m[i * D + j] = s;
      m[j * D + i] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < D; ++i) t += m[i * D + i];
    tr = t;
  }
  __syncthreads();
  const double t = tr;
  double c = 0.0;
  bool bad = !(t > 0.0) || !isfinite(t);
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const double v = m[e] / t;
    m[e] = v;
    if (!isfinite(v)) bad = true;
    c = fmax(c, fabs(v - o[e]));
  }
  red[threadIdx.x] = bad ? INFINITY : c;
  __syncthreads();
  for (int h = 32; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) change[blockIdx.x] = isinf(red[0]) ? NAN : red[0];
}

// M = V diag(lam) V^T for each symmetric D x D matrix (D <= 32), one warp per
// matrix: cyclic Jacobi rotations (p < q in row order), the 2 x 2 symmetric
// Schur rotation zeroing a_pq, until the off-diagonal part is below 1e-16 of
// the Frobenius norm.  V row-major, V[k * D + j] = component k of eigenvector j.
__global__ void __launch_bounds__(32) sym_eig_kernel(const double *__restrict__ Min, int D,
                                                     double *__restrict__ Vout, double *__restrict__ lam) {
  __shared__ double a[32][33], v[32][33];
  const int k = threadIdx.x;
  const double *M = Min + int64_t(blockIdx.x) * D * D;
  if (k < D)
    for (int j = 0; j < D; ++j) {
      a[k][j] = M[k * D + j];
      v[k][j] = (k == j) ? 1.0 : 0.0;
    }
  __syncwarp();
  for (int sweep = 0; sweep < kEigMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    if (k < D)
      for (int j = 0; j < D; ++j) {
        const double e = a[k][j] * a[k][j];
        tot += e;
        if (j != k) off += e;
      }
    for (int h = 16; h > 0; h >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, h);
      tot += __shfl_xor_sync(0xffffffffu, tot, h);
    }
    // lanes may differ in the last bit: take lane 0's sums so the stop is uniform
    off = __shfl_sync(0xffffffffu, off, 0);
    tot = __shfl_sync(0xffffffffu, tot, 0);
    if (!(off > 1e-32 * tot)) break;  // also ends on a zero or non-finite matrix
    for (int p = 0; p < D - 1; ++p)
      for (int q = p + 1; q < D; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;  // same value in every lane: uniform branch
        const double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        __syncwarp();
        if (k < D) {  // columns: A J and V J
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
        __syncwarp();
        if (k < D) {  // rows: J^T (A J)
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        __syncwarp();
        if (k == 0) {
          a[p][q] = 0.0;
          a[q][p] = 0.0;
        }
        __syncwarp();
      }
  }
  __syncwarp();
  if (k < D) {
    lam[int64_t(blockIdx.x) * D + k] = a[k][k];
    for (int j = 0; j < D; ++j) Vout[int64_t(blockIdx.x) * D * D + k * D + j] = v[k][j];
  }
}

// Lambda[p, a, b, c, e] = lu[a] ll[b] ld[c] lr[e];
// mode 0: y = x Lambda;  mode 1: y = x / (Lambda / *nrm + delta)
// (x and y may be the same array: each element is read once, then written)
__global__ void bp_weight_kernel(const double *x, double *y, int64_t n, int D,
                                 const double *lu, const double *ll, const double *ld, const double *lr,
                                 const double *nrm, double delta, int mode) {
  const double inv = mode ? 1.0 / *nrm : 0.0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    int64_t t = e;
    const int ie = int(t % D); t /= D;
    const int ic = int(t % D); t /= D;
    const int ib = int(t % D); t /= D;
    const int ia = int(t % D);
    const double L = lu[ia] * ll[ib] * ld[ic] * lr[ie];
    y[e] = mode ? x[e] / (L * inv + delta) : x[e] * L;
  }
}

void mode_product(const Cell &c, int leg, const double *x, double *y, const double *M, int trans,
                  cudaStream_t s) {
  int64_t outer, inner;
  mode_dims(c, leg, &outer, &inner);
  mode_product_kernel<<<grid_for(c.tsize()), 256, 0, s>>>(x, y, M, c.D, outer, inner, trans);
  count_launch();
}

// out = the tensor x with every leg transformed by its matrix (trans as in
// mode_product_kernel); t1, t2: scratch of one tensor each
void transform_legs(const Cell &c, const double *x, double *out, const double *const Ms[4], int trans,
                    double *t1, double *t2, cudaStream_t s) {
  mode_product(c, 0, x, t1, Ms[0], trans, s);
  mode_product(c, 1, t1, t2, Ms[1], trans, s);
  mode_product(c, 2, t2, t1, Ms[2], trans, s);
  mode_product(c, 3, t1, out, Ms[3], trans, s);
}

}  // namespace

void bp_metric(const Cell &c, const double *A, double tol, int maxit, BpMetric &m, cudaStream_t s) {
  IPEPS_REQUIRE(c.D >= 1 && c.D <= 32, "bp: bond dimension must be in 1..32");
  IPEPS_REQUIRE(maxit >= 1, "bp: maxit must be >= 1");
  const int D = c.D, ns = c.nsites(), nmsg = 4 * ns;
  const int64_t D2 = int64_t(D) * D, n = c.tsize();
  m.cell = c;
  DBuf cur(size_t(nmsg * D2), s), nxt(size_t(nmsg * D2), s), X(size_t(n), s), Y(size_t(n), s),
      chg(size_t(nmsg), s);
  bp_init_kernel<<<grid_for(nmsg * D2), 256, 0, s>>>(cur.p, D, nmsg);
  count_launch();
  std::vector<double> hc(static_cast<size_t>(nmsg));
  double change = INFINITY;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    {
      ProfScope prof("bp_sweep", s, 0.0, 0.0);
      for (int x = 0; x < c.Lx; ++x)
        for (int y = 0; y < c.Ly; ++y) {
          const double *As = A + int64_t(x * c.Ly + y) * n;
          for (int lam = 0; lam < 4; ++lam) {
            const double *src = As;
            double *bufs[2] = {X.p, Y.p};
            int w = 0;
            for (int mu = 0; mu < 4; ++mu) {
              if (mu == lam) continue;
              mode_product(c, mu, src, bufs[w], cur.p + incoming_index(c, x, y, mu) * D2, 0, s);
              src = bufs[w];
              w ^= 1;
            }
            int64_t outer, inner;
            mode_dims(c, lam, &outer, &inner);
            mode_gram_kernel<<<unsigned(D2), 128, 0, s>>>(src, As, D, outer, inner,
                                                          nxt.p + msg_index(c, x, y, lam) * D2);
            count_launch();
          }
        }
      bp_normalise_kernel<<<nmsg, 64, 0, s>>>(nxt.p, cur.p, D, chg.p);
      count_launch();
      check_launch("bp sweep");
    }
    IPEPS_CUDA(cudaMemcpyAsync(hc.data(), chg.p, nmsg * sizeof(double), cudaMemcpyDeviceToHost, s));
    IPEPS_CUDA(stream_sync(s));
    change = 0.0;
    for (double v : hc) {
      if (!std::isfinite(v)) throw Error(IPEPS_ERR_NONFINITE, "bp: a message has a non-positive trace or non-finite entries");
      change = std::max(change, v);
    }
    std::swap(cur, nxt);
    if (change <= tol) break;
  }
  m.sweeps = it > maxit ? maxit : it;
  m.change = change;
  m.msgs = std::move(cur);
  m.V = DBuf(size_t(nmsg * D2), s);
  m.lam = DBuf(size_t(nmsg) * D, s);
  sym_eig_kernel<<<nmsg, 32, 0, s>>>(m.msgs.p, D, m.V.p, m.lam.p);
  count_launch();
  // c_s = 1 / <A_s| 1 (x) m_u (x) m_l (x) m_d (x) m_r |A_s>, from A in the eigenbases
  m.nrm = DBuf(size_t(ns), s);
  for (int x = 0; x < c.Lx; ++x)
    for (int y = 0; y < c.Ly; ++y) {
      const int site = x * c.Ly + y;
      const double *Vs[4];
      const double *ls[4];
      for (int leg = 0; leg < 4; ++leg) {
        const int k = incoming_index(c, x, y, leg);
        Vs[leg] = m.V.p + k * D2;
        ls[leg] = m.lam.p + int64_t(k) * D;
      }
      DBuf At(size_t(n), s);
      transform_legs(c, A + int64_t(site) * n, At.p, Vs, 0, X.p, Y.p, s);
      bp_weight_kernel<<<grid_for(n), 256, 0, s>>>(At.p, X.p, n, D, ls[0], ls[1], ls[2], ls[3], nullptr, 0.0, 0);
      count_launch();
      dot(n, At.p, X.p, m.nrm.p + site, s);
    }
  check_launch("bp metric");
}

void bp_apply(const BpMetric &m, const double *g, double delta, double *out, cudaStream_t s) {
  const Cell &c = m.cell;
  const int D = c.D;
  const int64_t D2 = int64_t(D) * D, n = c.tsize();
  DBuf X(size_t(n), s), Y(size_t(n), s), Z(size_t(n), s);
  for (int x = 0; x < c.Lx; ++x)
    for (int y = 0; y < c.Ly; ++y) {
      const int site = x * c.Ly + y;
      const double *Vs[4];
      const double *ls[4];
      for (int leg = 0; leg < 4; ++leg) {
        const int k = incoming_index(c, x, y, leg);
        Vs[leg] = m.V.p + k * D2;
        ls[leg] = m.lam.p + int64_t(k) * D;
      }
      transform_legs(c, g + int64_t(site) * n, Z.p, Vs, 0, X.p, Y.p, s);
      bp_weight_kernel<<<grid_for(n), 256, 0, s>>>(Z.p, Z.p, n, D, ls[0], ls[1], ls[2], ls[3],
                                                   m.nrm.p + site, delta, 1);
      count_launch();
      transform_legs(c, Z.p, out + int64_t(site) * n, Vs, 1, X.p, Y.p, s);
    }
  check_launch("bp apply");
}

}  // namespace ipeps
