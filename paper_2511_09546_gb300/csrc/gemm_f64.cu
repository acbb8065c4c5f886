// FP64 GEMM on the CUDA cores (DFMA).  GB300's FP64 rate is about 2 DFMA per
// clock per SM, so a 64x64 register-blocked tile is compute bound at every
// shape the CTMRG produces; the kernel favours simplicity and exact FP64.
#include <cuda_runtime.h>

#include "common.h"
#include "kernels.h"

namespace ipeps {

namespace {
constexpr int BM = 64, BN = 64, BK = 8;

__global__ void __launch_bounds__(256) dgemm_kernel(bool ta, bool tb, int64_t M, int64_t N, int64_t K,
                                                    double alpha, const double *__restrict__ A,
                                                    int64_t lda, const double *__restrict__ B,
                                                    int64_t ldb, double beta, double *__restrict__ C,
                                                    int64_t ldc, int64_t sA, int64_t sB, int64_t sC) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int64_t bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  double acc[4][4] = {};
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (!ta) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = ta ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int nn, kk;
      if (!tb) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = tb ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double v = alpha * acc[i][j];
      double *c = C + gm * ldc + gn;
      *c = (beta == 0.0) ? v : v + beta * (*c);
    }
  }
}
}  // namespace

void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
              int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
              cudaStream_t s, int64_t batch, int64_t sA, int64_t sB, int64_t sC) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta C
    for (int64_t b = 0; b < batch; ++b) {
      if (ldc == N) {
        if (beta == 0.0) fill(C + b * sC, M * N, 0.0, s);
        else scal(M * N, beta, C + b * sC, s);
      } else {
        IPEPS_REQUIRE(false, "gemm_f64: K == 0 with padded ldc");
      }
    }
    return;
  }
  IPEPS_REQUIRE((N + BN - 1) / BN <= 2147483647 && (M + BM - 1) / BM <= 65535 && batch <= 65535,
                "gemm_f64: grid too large");
  dim3 grd(unsigned((N + BN - 1) / BN), unsigned((M + BM - 1) / BM), unsigned(batch));
  dgemm_kernel<<<grd, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC);
  count_launch();
  check_launch("dgemm");
}

}  // namespace ipeps
