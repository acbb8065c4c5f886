// Device kernels of libipeps (FP64 data movement, BLAS-1, reductions, GEMM, SVD).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace ipeps {

constexpr int kMaxDims = 8;

// dst = permute(src): dst has dims[perm[0]], ..., dims[perm[nd-1]];
// dst[j0..] = src[i] with i_{perm[k]} = j_k.  alpha scales, beta accumulates
// into dst (dst = alpha * permuted + beta * dst).
void permute(const double *src, const std::vector<int64_t> &dims, const std::vector<int> &perm,
             double *dst, cudaStream_t s, double alpha = 1.0, double beta = 0.0);

void fill(double *x, int64_t n, double v, cudaStream_t s);
void axpy(int64_t n, double a, const double *x, double *y, cudaStream_t s);            // y += a x
void axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s);  // y = a x + b y
void scal(int64_t n, double a, double *x, cudaStream_t s);
// device-scalar variants: y += (*num / *den) * sign * x
void axpy_ratio(int64_t n, const double *num, const double *den, double sign, const double *x,
                double *y, cudaStream_t s);
// out[0] = x.y (deterministic two-pass reduction into a device scalar)
void dot(int64_t n, const double *x, const double *y, double *out, cudaStream_t s);
void nrm2(int64_t n, const double *x, double *out, cudaStream_t s);
// batched column dots: out[j] = sum_i X[i, j] Y[i, j] for row-major (m x n)
void coldot(int64_t m, int64_t n, const double *X, const double *Y, double *out, cudaStream_t s);
// Y[i, j] = X[i, j] * f[j]  (row-major m x n); beta accumulates
void scale_cols(int64_t m, int64_t n, const double *X, const double *f, double *Y,
                cudaStream_t s, double beta = 0.0);
// x /= *nrm (device scalar)
void div_by_scalar(int64_t n, double *x, const double *nrm, cudaStream_t s);
// t[i, ..., j] *= sp[i] * sn[j] for t viewed as (a x mid x b)
void leg_signs(double *t, int64_t a, int64_t mid, int64_t b, const double *sp, const double *sn,
               cudaStream_t s);
// number of non-finite entries -> device int
void count_nonfinite(int64_t n, const double *x, int *out, cudaStream_t s);

// C = alpha op(A) op(B) + beta C, row-major, batched with element strides.
// op(A) is M x K: A is M x K (lda >= K) or, with ta, K x M (lda >= M).
void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
              int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
              cudaStream_t s, int64_t batch = 1, int64_t sA = 0, int64_t sB = 0, int64_t sC = 0);

// gemm_f64 without any device allocation: split-K partial sums in a static
// device array (see ipeps_gemm_noalloc)
void gemm_f64_noalloc(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                      int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                      cudaStream_t s);

// One-sided block Jacobi SVD of `batch` column-major m x n matrices G (ld = m,
// matrix stride m*n): on return G holds U S (orthogonal columns) and, if V is
// not null, V (n x n column-major per matrix, stride n*n) the accumulated
// rotations, so that G_in V = G_out.  Returns the sweeps used.
int jacobi_svd_colmajor(double *G, int64_t m, int64_t n, double *V, cudaStream_t s,
                        double tol = 1e-14, int max_sweeps = 40, int batch = 1);

}  // namespace ipeps
