// FP64 GEMM on the CUDA cores (DFMA).  GB300's FP64 rate is about 2 DFMA per
// clock per SM, so a 64x64 register-blocked tile is compute bound at every
// shape the CTMRG produces; the kernel favours simplicity and exact FP64, and
// the dispatcher's job is to keep every SM's FP64 pipe busy (split K whenever
// there are fewer output tiles than SMs).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "common.h"
#include "engine.h"
#include "kernels.h"
#include "profile.h"

namespace ipeps {

namespace {
constexpr int BM = 64, BN = 64, BK = 8;

// C tile of TM x TN per CTA of 256 threads (16 x 16, each (TM/16) x (TN/16)
// outputs), K staged in slices of BK through shared memory.  TM = TN = 64 in
// general; 32 x 32 tiles quadruple the CTA count of small outputs, whose 64 x 64
// tiles leave most SMs idle (the FP64 pipe of each occupied SM is the limit).
template <int TM, int TN>
__global__ void __launch_bounds__(256) dgemm_kernel(bool ta, bool tb, int64_t M, int64_t N, int64_t K,
                                                    double alpha, const double *__restrict__ A,
                                                    int64_t lda, const double *__restrict__ B,
                                                    int64_t ldb, double beta, double *__restrict__ C,
                                                    int64_t ldc, int64_t sA, int64_t sB, int64_t sC,
                                                    int64_t kchunk) {
  static_assert(TM % 16 == 0 && TN % 16 == 0 && TM <= 64 && TN <= 64, "dgemm tile");
  constexpr int RM = TM / 16, RN = TN / 16;
  __shared__ double As[BK][TM + 1];
  __shared__ double Bs[BK][TN + 1];
  // batched: blockIdx.z selects the matrix; split-K (kchunk > 0): blockIdx.z
  // selects a K range and C is the slice's partial-sum buffer
  const int64_t bz = blockIdx.z;
  int64_t kbeg = 0, kend = K;
  if (kchunk > 0) {
    kbeg = bz * kchunk;
    kend = kbeg + kchunk < K ? kbeg + kchunk : K;
    C += bz * sC;
  } else {
    A += bz * sA;
    B += bz * sB;
    C += bz * sC;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = int64_t(blockIdx.y) * TM, n0 = int64_t(blockIdx.x) * TN;
  double acc[RM][RN] = {};
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = threadIdx.x; e < TM * BK; e += 256) {
      int mm, kk;
      if (!ta) { mm = e / BK; kk = e % BK; } else { kk = e / TM; mm = e % TM; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < kend) v = ta ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < TN * BK; e += 256) {
      int nn, kk;
      if (!tb) { kk = e / TN; nn = e % TN; } else { nn = e / BK; kk = e % BK; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < kend) v = tb ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[RM], b[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double v = alpha * acc[i][j];
      double *c = C + gm * ldc + gn;
      *c = (beta == 0.0) ? v : v + beta * (*c);
    }
  }
}
// Small output (M N <= 1024), long K: block (z, y) takes K slice z and the 8
// outputs 8 y .. 8 y + 7, one per warp, lanes stride over k; partial sums go
// to W[z] (reduced below).
__global__ void __launch_bounds__(256) multidot_kernel(bool ta, bool tb, int64_t M, int64_t N, int64_t K,
                                                       double alpha, const double *__restrict__ A, int64_t lda,
                                                       const double *__restrict__ B, int64_t ldb,
                                                       double *__restrict__ W, int64_t kchunk) {
  const int64_t z = blockIdx.x;
  const int64_t kbeg = z * kchunk, kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const int64_t o = int64_t(blockIdx.y) * 8 + warp;
    if (o >= M * N) return;
    const int64_t m = o / N, n = o % N;
    double acc = 0.0;
    for (int64_t k = kbeg + lane; k < kend; k += 32) {
      double a = ta ? A[k * lda + m] : A[m * lda + k];
      double b = tb ? B[n * ldb + k] : B[k * ldb + n];
      acc = fma(a, b, acc);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) W[z * M * N + o] = alpha * acc;
  }
}

// One thread per output element (one of M, N small, K moderate): no tile waste.
__global__ void perout_kernel(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                              const double *__restrict__ A, int64_t lda, const double *__restrict__ B,
                              int64_t ldb, double beta, double *__restrict__ C, int64_t ldc) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < M * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t m, n;
    if (N <= M) { m = e / N; n = e % N; } else { n = e / M; m = e % M; }
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double a = ta ? A[k * lda + m] : A[m * lda + k];
      double b = tb ? B[n * ldb + k] : B[k * ldb + n];
      acc = fma(a, b, acc);
    }
    double *c = C + m * ldc + n;
    *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * (*c);
  }
}

// C[i, j] = sum_z W[z][i, j] + beta C[i, j] (fixed order: deterministic)
__global__ void splitk_reduce(const double *__restrict__ W, int S, int64_t M, int64_t N, double beta,
                              double *__restrict__ C, int64_t ldc) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < M * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < S; ++z) acc += W[z * M * N + e];
    double *c = C + (e / N) * ldc + e % N;
    *c = (beta == 0.0) ? acc : acc + beta * (*c);
  }
}

int num_sms() { return device_sm_count(); }
}  // namespace

Prec &fp64_policy() {
  static thread_local Prec p = Prec::FP64;
  return p;
}

// The slice GEMM packs both operands (4 launches) and pads M to 128, N to 64
// and K to 64; below about 2^23 multiply-adds the DFMA kernels finish first.
double &oz_threshold() {
  static thread_local double t = double(1 << 23);
  return t;
}

bool oz_worthwhile(int64_t m, int64_t n, int64_t k) {
  return m >= 16 && n >= 8 && k >= 16 && double(m) * n * k >= oz_threshold();
}

void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
              int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
              cudaStream_t s, int64_t batch, int64_t sA, int64_t sB, int64_t sC) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (fp64_policy() == Prec::FP64_TC && K > 0 && oz_worthwhile(M, N, K)) {
    for (int64_t b = 0; b < batch; ++b)
      gemm_oz(8, ta, tb, M, N, K, alpha, A + b * sA, lda, B + b * sB, ldb, beta, C + b * sC, ldc, s);
    return;
  }
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
  ProfScope prof(shape_class("dgemm", M, N, K * batch), s, 2.0 * M * N * K * batch,
                 8.0 * batch * (M * K + K * N + M * N * (beta == 0.0 ? 1.0 : 2.0)));
  const int sms = num_sms();
  if (batch == 1 && M * N <= 1024 && K >= 256) {
    const int64_t groups = (M * N + 7) / 8;
    int64_t S = std::max<int64_t>(1, std::min<int64_t>((4 * sms + groups - 1) / groups, (K + 127) / 128));
    int64_t kchunk = (K + S - 1) / S;
    S = (K + kchunk - 1) / kchunk;
    double *W = static_cast<double *>(dev_alloc(size_t(S) * M * N * sizeof(double), s));
    multidot_kernel<<<dim3(unsigned(S), unsigned((M * N + 7) / 8)), 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B,
                                                                                   ldb, W, kchunk);
    int rg = int(std::min<int64_t>((M * N + 255) / 256, 4 * sms));
    splitk_reduce<<<rg, 256, 0, s>>>(W, int(S), M, N, beta, C, ldc);
    count_launch(2);
    check_launch("dgemm multidot");
    dev_free(W, s);
    return;
  }
  if (batch == 1 && std::min(M, N) <= 8 && K <= 512) {
    int rg = int(std::min<int64_t>((M * N + 255) / 256, 16 * sms));
    perout_kernel<<<rg, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    count_launch();
    check_launch("dgemm perout");
    return;
  }
  // Tile plan.  The FP64 pipe of each occupied SM (~4 DFMA per ns) is the
  // limit, so the time is about (CTA waves) x (DFMA per CTA) / rate, plus a
  // reduce launch and its reads when K is split.  Candidates: 64 x 64 tiles,
  // and 32 x 32 tiles when the 64 x 64 ones leave SMs idle; each with K
  // unsplit, or split (batch 1) into the slices (of at least BK) that fill one
  // wave.  The cheapest wins; ties keep the larger tile and fewer slices.
  struct Plan { int tile; int64_t ctas, S, kchunk; double ns; };
  auto cost = [&](int T, int64_t S, int64_t kchunk) {
    Plan p{T, ((N + T - 1) / T) * ((M + T - 1) / T) * batch, S, kchunk, 0.0};
    const int64_t kc = S > 1 ? kchunk : (K + BK - 1) / BK * BK;
    p.ns = double((p.ctas * S + sms - 1) / sms) * T * T * kc / 4.0;
    if (S > 1) p.ns += 2500.0 + double(S) * M * N * 8.0 / 5000.0;
    return p;
  };
  auto split_of = [&](int T, Plan *out) {
    const int64_t ctas = ((N + T - 1) / T) * ((M + T - 1) / T);
    if (batch != 1 || ctas >= sms || K < 2 * BK) return false;
    int64_t S = std::min<int64_t>({sms / ctas, K / BK, int64_t(512)});
    if (S < 2) return false;
    const int64_t kchunk = ((K + S - 1) / S + BK - 1) / BK * BK;
    S = (K + kchunk - 1) / kchunk;
    if (S < 2) return false;
    *out = cost(T, S, kchunk);
    return true;
  };
  constexpr int ST = 32;
  Plan best = cost(BM, 1, 0), cand;
  if (split_of(BM, &cand) && cand.ns < best.ns) best = cand;
  if (((N + BN - 1) / BN) * ((M + BM - 1) / BM) * batch < sms) {
    Plan small = cost(ST, 1, 0);
    if (split_of(ST, &cand) && cand.ns < small.ns) small = cand;
    if (small.ns < 0.95 * best.ns) best = small;
  }
  IPEPS_REQUIRE((M + best.tile - 1) / best.tile <= 65535, "gemm_f64: grid too large");
  const dim3 grd(unsigned((N + best.tile - 1) / best.tile), unsigned((M + best.tile - 1) / best.tile),
                 unsigned(best.S > 1 ? best.S : batch));
  if (best.S > 1) {
    // split K: slice z writes its partial sums to W[z], a second kernel adds them in order
    double *W = static_cast<double *>(dev_alloc(size_t(best.S) * M * N * sizeof(double), s));
    if (best.tile == ST)
      dgemm_kernel<ST, ST><<<grd, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, 0.0, W, N, 0, 0, M * N,
                                                best.kchunk);
    else
      dgemm_kernel<BM, BN><<<grd, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, 0.0, W, N, 0, 0, M * N,
                                                best.kchunk);
    int rg = int(std::min<int64_t>((M * N + 255) / 256, 4 * sms));
    splitk_reduce<<<rg, 256, 0, s>>>(W, int(best.S), M, N, beta, C, ldc);
    count_launch(2);
    check_launch("dgemm splitk");
    dev_free(W, s);
    return;
  }
  if (best.tile == ST)
    dgemm_kernel<ST, ST><<<grd, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC, 0);
  else
    dgemm_kernel<BM, BN><<<grd, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC, 0);
  count_launch();
  check_launch("dgemm");
}

}  // namespace ipeps

// ---------------------------------------------------------------------------
// Allocation-free split-K GEMM (see ipeps_gemm_noalloc in include/ipeps.h).
// The split-K partial sums live in this file-scope device array instead of a
// stream-ordered allocation.  Every slice of it that a call reads is written
// by the same call first, so nothing needs clearing between calls; calls that
// overlap on the GPU share the array and race.
namespace ipeps {
namespace {
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 22;  // 4 Mi doubles = 32 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// device address of g_noalloc_scratch for the current device (host code may
// not use the symbol itself: it is a host-side stand-in, not a device address).
// Looked up once per device index and kept for the life of the process: after
// a cudaDeviceReset (or any reset of the primary context) the cached address
// is stale, so the entry point must not be used past such a reset.
double *noalloc_scratch_ptr() {
  static double *ptrs[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  IPEPS_CUDA(cudaGetDevice(&dev));
  IPEPS_REQUIRE(dev >= 0 && dev < 64, "gemm_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      throw Error(IPEPS_ERR_CUDA, std::string("gemm_noalloc: cudaGetSymbolAddress failed: ") +
                                      cudaGetErrorString(e));
    ptrs[dev] = static_cast<double *>(p);
  }
  return ptrs[dev];
}

__global__ void scale_matrix_kernel(int64_t M, int64_t N, double beta, double *C, int64_t ldc) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < M * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    double *c = C + (e / N) * ldc + e % N;
    *c = (beta == 0.0) ? 0.0 : beta * (*c);
  }
}
}  // namespace

void gemm_f64_noalloc(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                      int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                      cudaStream_t s) {
  IPEPS_REQUIRE(M >= 0 && N >= 0 && K >= 0, "gemm_noalloc: negative size");
  if (M == 0 || N == 0) return;
  IPEPS_REQUIRE(M * N <= kNoAllocScratchDoubles,
                "gemm_noalloc: M*N = " + std::to_string(M * N) + " exceeds the scratch of " +
                    std::to_string(kNoAllocScratchDoubles) + " doubles (32 MiB)");
  const int sms = num_sms();
  ProfScope prof("dgemm", s, 2.0 * M * N * K, 8.0 * (M * K + K * N + M * N * (beta == 0.0 ? 1.0 : 2.0)));
  if (K == 0) {
    scale_matrix_kernel<<<int(std::min<int64_t>((M * N + 255) / 256, 4 * sms)), 256, 0, s>>>(M, N, beta, C, ldc);
    count_launch();
    check_launch("gemm_noalloc scale");
    return;
  }
  double *W = noalloc_scratch_ptr();
  const int64_t tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  const int64_t fit = kNoAllocScratchDoubles / (M * N);  // slices that fit in the scratch
  if (M * N <= 1024 && K >= 256) {
    int64_t S = std::min<int64_t>({int64_t(4) * sms, (K + 255) / 256, fit});
    int64_t kchunk = (K + S - 1) / S;
    S = (K + kchunk - 1) / kchunk;
    multidot_kernel<<<dim3(unsigned(S), unsigned((M * N + 7) / 8)), 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B,
                                                                                   ldb, W, kchunk);
    splitk_reduce<<<int(std::min<int64_t>((M * N + 255) / 256, 4 * sms)), 256, 0, s>>>(W, int(S), M, N, beta, C, ldc);
    count_launch(2);
    check_launch("gemm_noalloc multidot");
    return;
  }
  int64_t S = std::max<int64_t>(1, std::min<int64_t>({(2 * sms + tiles - 1) / tiles, (K + 511) / 512, fit, int64_t(512)}));
  int64_t kchunk = ((K + S - 1) / S + BK - 1) / BK * BK;
  S = (K + kchunk - 1) / kchunk;
  IPEPS_REQUIRE((M + BM - 1) / BM <= 65535, "gemm_noalloc: grid too large");
  dim3 grd(unsigned((N + BN - 1) / BN), unsigned((M + BM - 1) / BM), unsigned(S));
  dgemm_kernel<BM, BN><<<grd, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, 0.0, W, N, 0, 0, M * N, kchunk);
  splitk_reduce<<<int(std::min<int64_t>((M * N + 255) / 256, 4 * sms)), 256, 0, s>>>(W, int(S), M, N, beta, C, ldc);
  count_launch(2);
  check_launch("gemm_noalloc splitk");
}
}  // namespace ipeps
