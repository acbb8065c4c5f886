// One-sided block Jacobi SVD in FP64 (projector truncation, Sec. III.A CTMRG;
// corner spectra for the convergence test).
//
// The m x n matrix is held column-major.  Its columns are grouped in blocks of
// 16; one CTA orthogonalises a pair of blocks: it accumulates the 32 x 32 Gram
// matrix of the pair over row chunks staged in shared memory, diagonalises it
// with a cyclic two-sided Jacobi sweep in shared memory (parallel rotation
// sets), and applies the resulting 32 x 32 rotation to the 32 columns and to
// the matching columns of V.  A round-robin tournament gives nb/2 independent
// block pairs per launch (one launch per step, nb-1 steps per sweep); the
// sweep loop ends when no pair has a cosine above tol.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.h"
#include "kernels.h"
#include "profile.h"

namespace ipeps {

namespace {
constexpr int W = 16;        // block width
constexpr int PW = 2 * W;    // pair width
constexpr int RCH = 64;      // rows per staged chunk

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  // valid for non-negative doubles: their bit patterns order like the values
  atomicMax(reinterpret_cast<unsigned long long *>(addr), __double_as_longlong(v));
}

__device__ __forceinline__ int tourney(int i, int r, int nb) {
  // position i of round r in the round-robin schedule of nb players
  if (i == 0) return 0;
  return ((i - 1 + r) % (nb - 1)) + 1;
}

__global__ void __launch_bounds__(256) jacobi_pair_kernel(double *__restrict__ G, int64_t m,
                                                          double *__restrict__ V, int64_t nv,
                                                          int nb, int step, double tol,
                                                          double *offmax) {
  __shared__ double Gm[PW][PW + 1];
  __shared__ double Z[PW][PW + 1];
  __shared__ double chunk[RCH][PW + 1];
  __shared__ double cs[PW / 2], sn[PW / 2];
  __shared__ int pp[PW / 2], qq[PW / 2];
  __shared__ double red[256];
  __shared__ int skip;

  const int k = blockIdx.x;
  G += int64_t(blockIdx.y) * m * (int64_t(nb) * W);
  if (V) V += int64_t(blockIdx.y) * nv * nv;
  const int bi = tourney(k, step, nb), bj = tourney(nb - 1 - k, step, nb);
  const int tid = threadIdx.x;
  auto gcol = [&](int c) -> int64_t { return c < W ? int64_t(bi) * W + c : int64_t(bj) * W + (c - W); };

  // ---- Gram of the 32 columns
  double acc[4] = {0, 0, 0, 0};
  for (int64_t r0 = 0; r0 < m; r0 += RCH) {
    for (int e = tid; e < RCH * PW; e += 256) {
      int c = e / RCH, r = e % RCH;
      chunk[r][c] = (r0 + r < m) ? G[gcol(c) * m + r0 + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int e = tid + 256 * t;
      int p = e / PW, q = e % PW;
      double a = 0.0;
      for (int r = 0; r < RCH; ++r) a = fma(chunk[r][p], chunk[r][q], a);
      acc[t] += a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int e = tid + 256 * t;
    Gm[e / PW][e % PW] = acc[t];
  }
  __syncthreads();

  // ---- largest cosine between two columns of the pair
  double off = 0.0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int e = tid + 256 * t;
    int p = e / PW, q = e % PW;
    if (p < q) {
      double d = Gm[p][p] * Gm[q][q];
      if (d > 0.0) off = fmax(off, fabs(Gm[p][q]) / sqrt(d));
    }
  }
  red[tid] = off;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
    __syncthreads();
  }
  if (tid == 0) {
    atomic_max_nonneg(offmax, red[0]);
    skip = red[0] <= tol;
  }
  __syncthreads();
  if (skip) return;

  // ---- diagonalise the Gram matrix: Z^T Gm Z = diag
  for (int e = tid; e < PW * PW; e += 256) Z[e / PW][e % PW] = (e / PW == e % PW) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 12; ++sweep) {
    for (int round = 0; round < PW - 1; ++round) {
      if (tid < PW / 2) {
        int p = tourney(tid, round, PW), q = tourney(PW - 1 - tid, round, PW);
        if (p > q) { int t = p; p = q; q = t; }
        double a = Gm[p][p], b = Gm[q][q], g = Gm[p][q];
        double c = 1.0, s = 0.0;
        if (g != 0.0 && fabs(g) > 1e-17 * sqrt(fabs(a * b))) {
          double tau = (b - a) / (2.0 * g);
          double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        cs[tid] = c; sn[tid] = s; pp[tid] = p; qq[tid] = q;
      }
      __syncthreads();
      // columns of Gm and Z
      for (int e = tid; e < (PW / 2) * PW; e += 256) {
        int pr = e / PW, i = e % PW;
        int p = pp[pr], q = qq[pr];
        double c = cs[pr], s = sn[pr];
        double gp = Gm[i][p], gq = Gm[i][q];
        Gm[i][p] = c * gp - s * gq;
        Gm[i][q] = s * gp + c * gq;
        double zp = Z[i][p], zq = Z[i][q];
        Z[i][p] = c * zp - s * zq;
        Z[i][q] = s * zp + c * zq;
      }
      __syncthreads();
      // rows of Gm
      for (int e = tid; e < (PW / 2) * PW; e += 256) {
        int pr = e / PW, j = e % PW;
        int p = pp[pr], q = qq[pr];
        double c = cs[pr], s = sn[pr];
        double gp = Gm[p][j], gq = Gm[q][j];
        Gm[p][j] = c * gp - s * gq;
        Gm[q][j] = s * gp + c * gq;
      }
      __syncthreads();
    }
    // stop when the Gram matrix is diagonal to rounding
    double o = 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int e = tid + 256 * t;
      int p = e / PW, q = e % PW;
      if (p < q) {
        double d = Gm[p][p] * Gm[q][q];
        if (d > 0.0) o = fmax(o, fabs(Gm[p][q]) / sqrt(d));
      }
    }
    red[tid] = o;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
      __syncthreads();
    }
    bool done = red[0] < 1e-16;
    __syncthreads();
    if (done) break;
  }

  // ---- apply Z to the 32 columns of G and of V
  for (int pass = 0; pass < (V ? 2 : 1); ++pass) {
    double *X = pass == 0 ? G : V;
    int64_t rows = pass == 0 ? m : nv;
    for (int64_t r0 = 0; r0 < rows; r0 += RCH) {
      for (int e = tid; e < RCH * PW; e += 256) {
        int c = e / RCH, r = e % RCH;
        chunk[r][c] = (r0 + r < rows) ? X[gcol(c) * rows + r0 + r] : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < RCH * PW; e += 256) {
        int c = e / RCH, r = e % RCH;
        if (r0 + r < rows) {
          double v = 0.0;
#pragma unroll 8
          for (int p = 0; p < PW; ++p) v = fma(chunk[r][p], Z[p][c], v);
          X[gcol(c) * rows + r0 + r] = v;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void eye_kernel(double *V, int64_t n, int64_t batch) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n * n * batch;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t e = i % (n * n);
    V[i] = (e / n == e % n) ? 1.0 : 0.0;
  }
}

// dst[b][c][r] (m x npad per matrix) from src[b][c][r] (m x n), zero padded
__global__ void pad_copy_kernel(const double *__restrict__ src, int64_t m, int64_t n,
                                double *__restrict__ dst, int64_t npad, int64_t batch) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m * npad * batch;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t b = i / (m * npad), e = i % (m * npad);
    int64_t c = e / m, r = e % m;
    dst[i] = c < n ? src[b * m * n + c * m + r] : 0.0;
  }
}

// dst[b] (rows x cols, ld rows) from src[b] (ld x ..), first rows/cols
__global__ void crop_kernel(const double *__restrict__ src, int64_t ld, int64_t sstride, int64_t rows,
                            int64_t cols, double *__restrict__ dst, int64_t batch) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows * cols * batch;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t b = i / (rows * cols), e = i % (rows * cols);
    int64_t c = e / rows, r = e % rows;
    dst[i] = src[b * sstride + c * ld + r];
  }
}
}  // namespace

int jacobi_svd_colmajor(double *G, int64_t m, int64_t n, double *V, cudaStream_t s, double tol,
                        int max_sweeps, int batch) {
  IPEPS_REQUIRE(m >= 1 && n >= 1 && batch >= 1 && batch <= 65535, "jacobi_svd: bad sizes");
  int64_t npad = ((n + PW - 1) / PW) * PW;
  int nb = int(npad / W);
  DBuf Gp(size_t(m * npad * batch), s), off(1, s);
  DBuf Vp(V ? size_t(npad * npad * batch) : 0, s);
  pad_copy_kernel<<<512, 256, 0, s>>>(G, m, n, Gp.p, npad, batch);
  count_launch();
  if (V) {
    eye_kernel<<<512, 256, 0, s>>>(Vp.p, npad, batch);
    count_launch();
  }
  check_launch("jacobi init");
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    IPEPS_CUDA(cudaMemsetAsync(off.p, 0, sizeof(double), s));
    dim3 grd(unsigned(nb / 2), unsigned(batch));
    // algorithmic work counted per pair step: the 32 x 32 Gram matrices of all
    // nb/2 pairs (2 m 32^2 flops each, done even for pairs that are already
    // orthogonal); rotations and the inner eigensolve are not counted, so the
    // rate derived from it is a lower bound
    const double gram_flops = 2.0 * double(m) * PW * PW * (nb / 2) * batch;
    for (int step = 0; step < nb - 1; ++step) {
      ProfScope prof("jacobi_pair", s, gram_flops, 0.0);
      jacobi_pair_kernel<<<grd, 256, 0, s>>>(Gp.p, m, V ? Vp.p : nullptr, npad, nb, step, tol, off.p);
      count_launch();
    }
    check_launch("jacobi_pair");
    double h = 0.0;
    IPEPS_CUDA(cudaMemcpyAsync(&h, off.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    IPEPS_CUDA(stream_sync(s));
    if (!(h > tol)) break;
  }
  // copy back the first n columns (padded columns never mix with real ones)
  crop_kernel<<<512, 256, 0, s>>>(Gp.p, m, m * npad, m, n, G, batch);
  count_launch();
  if (V) {
    crop_kernel<<<512, 256, 0, s>>>(Vp.p, npad, npad * npad, n, n, V, batch);
    count_launch();
  }
  check_launch("jacobi crop");
  return sweep + 1;
}

}  // namespace ipeps
