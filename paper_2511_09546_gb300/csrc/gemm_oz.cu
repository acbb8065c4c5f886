// FP64-accurate (and reduced-precision) GEMM on the BF16 tensor cores
// (tcgen05.mma kind::f16, sm_103a) by exponent-aligned integer slicing.
//
// GB300 retires about 1.1 TFLOP/s of FP64 on its CUDA cores, three orders of
// magnitude below its BF16 tensor rate.  This kernel computes C = alpha op(A)
// op(B) + beta C for FP64 operands from products of small integers, which the
// tensor cores form and sum exactly:
//
//   Row i of op(A) is scaled by 2^-E_i with 2^E_i > max_k |a_ik| and written as
//   S digits of 7 bits, a_ik = 2^(E_i - 7) sum_p a~_ikp with a~_ikp = d_p 2^(-7p),
//   d_0 in [-128, 128] and d_p in [-64, 64] for p >= 1 (each digit the rounded
//   remainder of the previous ones; FP64 arithmetic, exact).  Columns of op(B)
//   likewise (exponent F_j).  Every digit is an integer of at most 8 bits times
//   a power of two, hence exact in BF16.
//
//   a_ik b_kj = 2^(E_i + F_j - 14) sum_{p,q} a~_ikp b~_kjq; the pair (p, q)
//   carries the scale 2^(-7 (p + q)), so pairs of one "level" L = p + q share an
//   accumulator.  Pairs with L >= S are dropped (they lie below 2^(-7 S) of the
//   leading term).
//
//   Exactness: a level-L sum over a chunk of 512 K elements is an integer
//   multiple of 2^(-7L) below 2^24 of that unit for L <= 4 (at most
//   (L + 3) 2^12 per element), so the FP32 tensor-core accumulation of levels
//   0 .. 4 is exact whatever order the hardware adds in.  After each chunk the
//   flush warps turn those sums into integers and add them into one 64-bit
//   fixed-point accumulator per output (least significant bit at level 4).
//   Levels 5 and beyond share one FP32 accumulator over all of K: their
//   rounding, 2^-24 of a quantity 2^-35 below the leading term, is far below
//   FP64 rounding.  The result is (acc 2^-28 + tail) 2^(E_i + F_j - 14).
//
// With S = 8 (36 BF16 products per term) the error bound is that of an FP64
// GEMM taken relative to max_k |a_ik| max_k |b_kj| instead of sum_k |a_ik b_kj|;
// with S = 2 (3 products: the BF16x3 scheme) it is about 2^-15 of the same.
//
// Roles (one CTA per 128 x BN output tile and K range, 10 or 18 warps):
//   * flush warps 0 .. 4 BN/32 - 1: warp w owns TMEM lanes 32 (w % 4) .. +31
//     (output rows) and columns 32 (w / 4) .. +31 of every accumulator;
//   * lane 0 of the producer warp streams K slices of 32 elements, all S digits
//     of A and of B per slice, with TMA (64-byte swizzle) into a ring of stages;
//     the producer warp also owns the TMEM allocation;
//   * lane 0 of the MMA warp issues, per 16-element K step, one tcgen05.mma
//     (M = 128, N = BN, K = 16) per pair into its level's accumulator, releases
//     stages with tcgen05.commit and signals each finished chunk.
// Every mbarrier wait is bounded: on expiry the kernel raises the error word,
// skips the write of C, drains its own copies (bounded), frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "common.h"
#include "engine.h"
#include "kernels.h"
#include "profile.h"
#include "tc_ptx.h"

namespace ipeps {

namespace {
using namespace ptx;

constexpr int OBM = 128;             // rows per tile (TMEM lanes)
constexpr int OBK = 32;              // K elements per slice: 64 bytes of BF16 per row
constexpr int OCHUNK = 16;           // K slices per exactly summed chunk (512 elements)
constexpr int OLEX = 5;              // levels summed exactly (0 .. 4)
constexpr int OBETA = 7;             // bits per digit
constexpr int ORING = 200 * 1024;    // shared-memory ring
constexpr int OGROUP_M = 8;

template <int S> __host__ __device__ constexpr int lex() { return S < OLEX ? S : OLEX; }
template <int S> __host__ __device__ constexpr bool has_tail() { return S > OLEX; }
template <int S, int BN> __host__ __device__ constexpr int nacc() { return lex<S>() + (has_tail<S>() ? 1 : 0); }
template <int S, int BN> __host__ __device__ constexpr uint32_t tmem_cols() {
  return nacc<S, BN>() * BN <= 32 ? 32u
         : nacc<S, BN>() * BN <= 64 ? 64u
         : nacc<S, BN>() * BN <= 128 ? 128u
         : nacc<S, BN>() * BN <= 256 ? 256u
                                     : 512u;
}
template <int BN> __host__ __device__ constexpr int oflush_warps() { return 4 * (BN / 32); }
template <int BN> __host__ __device__ constexpr int othreads() { return 32 * (oflush_warps<BN>() + 2); }
template <int S, int BN> __host__ __device__ constexpr int stage_bytes() { return S * (OBM + BN) * OBK * 2; }
template <int S, int BN> __host__ __device__ constexpr int ostages() {
  return ORING / stage_bytes<S, BN>() < 8 ? ORING / stage_bytes<S, BN>() : 8;
}

// A~ in slice kt, digit p: rows m0.., columns p Kp + kt OBK (the packed operand is
// rows x S Kp with digit p in columns p Kp .. p Kp + Kp - 1)
template <int S, int BN>
__global__ void __launch_bounds__(othreads<BN>(), 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const int *__restrict__ ea, const int *__restrict__ eb, int64_t M, int64_t N, int Kp,
                   int nk, int kper, double alpha, double beta, double *__restrict__ C, int64_t ldc,
                   int64_t zstride, int *err) {
  static_assert(tmem_cols<S, BN>() <= 512, "accumulators exceed tensor memory");
  constexpr uint32_t A_TILE = OBM * OBK * 2, B_TILE = BN * OBK * 2;
  constexpr int STAGES = ostages<S, BN>();
  constexpr int FLUSH_WARPS = oflush_warps<BN>(), PRODUCER_WARP = FLUSH_WARPS, MMA_WARP = FLUSH_WARPS + 1;
  constexpr int LEX = lex<S>();
  static_assert(STAGES >= 2, "ring too small");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], acc_full, acc_empty;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mt, ntile;
  {
    const int nt = gridDim.x, mtiles = gridDim.y;
    const int id = blockIdx.y * nt + blockIdx.x, per = OGROUP_M * nt;
    const int first = (id / per) * OGROUP_M, rows = min(OGROUP_M, mtiles - first);
    mt = first + (id % per) % rows;
    ntile = (id % per) / rows;
  }
  const int m0 = mt * OBM, n0 = ntile * BN;
  // K range of this CTA (split K over blockIdx.z): slices [k_beg, k_end)
  const int k_beg = blockIdx.z * kper, k_end = min(nk, k_beg + kper);
  const int nks = k_end - k_beg;
  const int nchunks = (nks + OCHUNK - 1) / OCHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, FLUSH_WARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == PRODUCER_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols<S, BN>())
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  int issued = 0;
  if (warp == PRODUCER_WARP) {
    if (lane == 0) {
      for (int i = 0; i < nks; ++i) {
        const int s = i % STAGES, kt = k_beg + i;
        if (!mbar_wait(&empty[s], ((i / STAGES) & 1) ^ 1, err)) break;
        uint8_t *st = base + size_t(s) * stage_bytes<S, BN>();
        mbar_expect_tx(&full[s], uint32_t(stage_bytes<S, BN>()));
#pragma unroll
        for (int p = 0; p < S; ++p) {
          tma_load_2d(st + p * A_TILE, &mapA, &full[s], p * Kp + kt * OBK, m0);
          tma_load_2d(st + S * A_TILE + p * B_TILE, &mapB, &full[s], p * Kp + kt * OBK, n0);
        }
        issued = i + 1;
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      // kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both K-major
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) |
                                 (uint32_t(OBM >> 4) << 24);
      bool ok = true, tail_started = false;
      int i = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        ok = mbar_wait(&acc_empty, (c & 1) ^ 1, err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t started = 0;  // exact levels written in this chunk
        const int i_end = min(nks, i + OCHUNK);
        for (; i < i_end; ++i) {
          const int s = i % STAGES;
          ok = mbar_wait(&full[s], (i / STAGES) & 1, err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(base + size_t(s) * stage_bytes<S, BN>());
#pragma unroll
          for (int ks = 0; ks < OBK / 16; ++ks) {  // 16 BF16 = 32 bytes per MMA: +2 in the address field
#pragma unroll
            for (int p = 0; p < S; ++p) {
              const uint64_t ad = smem_desc_sw64(st + p * A_TILE) + 2 * ks;
#pragma unroll
              for (int q = 0; q + p < S; ++q) {
                const int L = p + q;
                const uint64_t bd = smem_desc_sw64(st + S * A_TILE + q * B_TILE) + 2 * ks;
                uint32_t acc;
                if (L < LEX) {
                  acc = (started >> L) & 1u;
                  started |= 1u << L;
                  mma_bf16(tmem + uint32_t(L * BN), ad, bd, idesc, acc);
                } else {
                  acc = tail_started ? 1u : 0u;
                  tail_started = true;
                  mma_bf16(tmem + uint32_t(LEX * BN), ad, bd, idesc, acc);
                }
              }
            }
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full);
      }
    }
  } else {
    // ---- flush warps: exact level sums (TMEM, FP32 integers) -> 64-bit fixed point
    const uint32_t lanes = uint32_t((warp & 3) * 32) << 16, cw = uint32_t((warp >> 2) * 32);
    long long acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = __all_sync(0xffffffffu, mbar_wait(&acc_full, c & 1, err) ? 1 : 0) != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int L = 0; L < LEX; ++L) {
        uint32_t v0[16], v1[16];
        tmem_ld16_issue(tmem + lanes + uint32_t(L * BN) + cw, v0);
        tmem_ld16_issue(tmem + lanes + uint32_t(L * BN) + cw + 16, v1);
        tmem_ld_wait(v0);
        tmem_ld_wait(v1);
        // the level sum is an exact integer multiple of 2^(-7L) below 2^24 of it
        const float up = __int_as_float((127 + OBETA * L) << 23);  // 2^(7L)
        const long long w = 1ll << (OBETA * (LEX - 1 - L));
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          acc[j] += (long long)__float2int_rn(__uint_as_float(v0[j]) * up) * w;
          acc[16 + j] += (long long)__float2int_rn(__uint_as_float(v1[j]) * up) * w;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty);
    }
    if (ok && nchunks > 0) {
      float tail[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) tail[j] = 0.0f;
      if (has_tail<S>()) {
        uint32_t v0[16], v1[16];
        tmem_ld16_issue(tmem + lanes + uint32_t(LEX * BN) + cw, v0);
        tmem_ld16_issue(tmem + lanes + uint32_t(LEX * BN) + cw + 16, v1);
        tmem_ld_wait(v0);
        tmem_ld_wait(v1);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          tail[j] = __uint_as_float(v0[j]);
          tail[16 + j] = __uint_as_float(v1[j]);
        }
      }
      const int64_t row = m0 + (warp & 3) * 32 + lane;
      const int64_t col0 = n0 + (warp >> 2) * 32;
      if (row < M) {
        const int er = ea[row];
        double *crow = C + blockIdx.z * zstride + row * ldc + col0;
        const double fix = ldexp(1.0, -OBETA * (LEX - 1));
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (col0 + j < N) {
            const double t = double(acc[j]) * fix + double(tail[j]);
            const double v = alpha * ldexp(t, er + eb[col0 + j] - 2 * OBETA);
            crow[j] = (beta == 0.0) ? v : v + beta * crow[j];
          }
        }
      }
    }
  }
  if (warp == PRODUCER_WARP && lane == 0 && issued > 0 && *err) {
    for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i)
      mbar_wait(&full[i % STAGES], (i / STAGES) & 1, err, 200000000ll);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == PRODUCER_WARP) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols<S, BN>())
                 : "memory");
  }
}

// exponent E_r with 2^E_r > max_k |op(X)[r, k]| (0 for a zero row), one row of
// op(X) per warp when its elements are contiguous
__global__ void oz_rowexp_contig(const double *__restrict__ X, int64_t ld, int64_t rows, int64_t K, int *ex,
                                 int64_t rows_pad) {
  const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows_pad) return;
  double m = 0.0;
  if (r < rows)
    for (int64_t k = lane; k < K; k += 32) m = fmax(m, fabs(X[r * ld + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int e = 0;
    frexp(m, &e);
    ex[r] = e;
  }
}

// the same when the elements of a row of op(X) are strided (X stored K x rows)
__global__ void oz_rowexp_strided(const double *__restrict__ X, int64_t ld, int64_t rows, int64_t K, int *ex,
                                  int64_t rows_pad) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows_pad) return;
  double m = 0.0;
  if (r < rows)
    for (int64_t k = 0; k < K; ++k) m = fmax(m, fabs(X[k * ld + r]));
  int e = 0;
  frexp(m, &e);
  ex[r] = e;
}

// P[r][p Kp + k] = BF16 digit p of op(X)[r, k] 2^-E_r (zero outside rows x K),
// one 256-thread block per 32 x 32 tile with a shared-memory transpose
template <int S>
__global__ void __launch_bounds__(256) oz_digits_kernel(const double *__restrict__ X, int64_t ld, bool trans,
                                                        int64_t rows, int64_t K, int64_t Kp,
                                                        const int *__restrict__ ex, __nv_bfloat16 *__restrict__ P) {
  __shared__ double T[32][33];  // T[k][r]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k0 = int64_t(blockIdx.x) * 32, r0 = int64_t(blockIdx.y) * 32;
#pragma unroll
  for (int i = 0; i < 32; i += 8) {
    if (trans) {
      const int64_t k = k0 + ty + i, r = r0 + tx;
      T[ty + i][tx] = (k < K && r < rows) ? X[k * ld + r] : 0.0;
    } else {
      const int64_t r = r0 + ty + i, k = k0 + tx;
      T[tx][ty + i] = (k < K && r < rows) ? X[r * ld + k] : 0.0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 32; i += 8) {
    const int r = ty + i;
    const int64_t row = r0 + r;
    double v = ldexp(T[tx][r], -ex[row] + OBETA);  // in (-2^7, 2^7): exact power-of-two scaling
    __nv_bfloat16 *dst = P + row * (S * Kp) + k0 + tx;
#pragma unroll
    for (int p = 0; p < S; ++p) {
      const double d = rint(v);
      v = (v - d) * double(1 << OBETA);  // exact: |v - d| <= 1/2
      dst[p * Kp] = __float2bfloat16_rn(ldexpf(float(d), -OBETA * p));
    }
  }
}

// C = sum_z W[z] + beta C in a fixed order (split K)
__global__ void oz_reduce(const double *__restrict__ W, int Z, int64_t M, int64_t N, double beta, double *C,
                          int64_t ldc) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < M * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < Z; ++z) acc += W[z * M * N + e];
    double *c = C + (e / N) * ldc + e % N;
    *c = (beta == 0.0) ? acc : acc + beta * (*c);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
      throw Error(IPEPS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

CUtensorMap oz_map(const __nv_bfloat16 *P, int64_t rows_pad, int64_t cols, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows_pad)};
  cuuint64_t strides[1] = {cuuint64_t(cols) * 2};
  cuuint32_t box[2] = {cuuint32_t(OBK), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = oz_encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(P), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(IPEPS_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
  return m;
}

int oz_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

template <int S, int BN>
void oz_run(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
            const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s) {
  const int64_t Kp = (K + OBK - 1) / OBK * OBK;
  const int64_t Mp = (M + OBM - 1) / OBM * OBM, Np = (N + BN - 1) / BN * BN;
  IPEPS_REQUIRE(Mp / OBM <= 65535 && S * Kp <= 2147483647 && Kp / OBK <= (int64_t(1) << 24),
                "oz_gemm: problem too large");
  __nv_bfloat16 *Pa = static_cast<__nv_bfloat16 *>(dev_alloc(size_t(Mp) * S * Kp * 2, s));
  __nv_bfloat16 *Pb = static_cast<__nv_bfloat16 *>(dev_alloc(size_t(Np) * S * Kp * 2, s));
  int *ea = static_cast<int *>(dev_alloc(size_t(Mp) * sizeof(int), s));
  int *eb = static_cast<int *>(dev_alloc(size_t(Np) * sizeof(int), s));
  {
    ProfScope prof("oz_pack", s, 0.0, 8.0 * (M * K + K * N) * 2 + 2.0 * S * (Mp + Np) * Kp);
    // op(A)[m, k]: contiguous along k unless ta; op(B) as rows n: element (n, k) is
    // B[k * ldb + n] (strided in k) unless tb
    if (!ta) oz_rowexp_contig<<<unsigned((Mp * 32 + 255) / 256), 256, 0, s>>>(A, lda, M, K, ea, Mp);
    else oz_rowexp_strided<<<unsigned((Mp + 255) / 256), 256, 0, s>>>(A, lda, M, K, ea, Mp);
    if (tb) oz_rowexp_contig<<<unsigned((Np * 32 + 255) / 256), 256, 0, s>>>(B, ldb, N, K, eb, Np);
    else oz_rowexp_strided<<<unsigned((Np + 255) / 256), 256, 0, s>>>(B, ldb, N, K, eb, Np);
    oz_digits_kernel<S><<<dim3(unsigned(Kp / 32), unsigned(Mp / 32)), 256, 0, s>>>(A, lda, ta, M, K, Kp, ea, Pa);
    oz_digits_kernel<S><<<dim3(unsigned(Kp / 32), unsigned(Np / 32)), 256, 0, s>>>(B, ldb, !tb, N, K, Kp, eb, Pb);
    count_launch(4);
    check_launch("oz_pack");
  }
  const CUtensorMap ma = oz_map(Pa, Mp, S * Kp, OBM);
  const CUtensorMap mb = oz_map(Pb, Np, S * Kp, BN);
  // split K when the output tiles leave SMs idle; every split covers whole slices
  const int nk = int(Kp / OBK);
  const int64_t tiles = (Mp / OBM) * (Np / BN);
  int Z = int(std::max<int64_t>(1, std::min<int64_t>(oz_sms() / std::max<int64_t>(1, tiles), nk)));
  const int kper = (nk + Z - 1) / Z;
  Z = (nk + kper - 1) / kper;
  double *W = nullptr;
  if (Z > 1) W = static_cast<double *>(dev_alloc(size_t(Z) * M * N * sizeof(double), s));
  int *err = tc_error_word();
  {
    ProfScope prof(shape_class("oz_gemm", M, N, K), s, 2.0 * M * N * K,
                   2.0 * S * (Mp + Np) * Kp + 8.0 * M * N * (beta == 0.0 ? 1 : 2));
    constexpr size_t smem = size_t(ostages<S, BN>()) * stage_bytes<S, BN>() + 1024;
    static bool attr = false;
    if (!attr) {
      IPEPS_CUDA(cudaFuncSetAttribute(oz_gemm_kernel<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      attr = true;
    }
    dim3 grid(unsigned(Np / BN), unsigned(Mp / OBM), unsigned(Z));
    if (Z > 1)
      oz_gemm_kernel<S, BN><<<grid, othreads<BN>(), smem, s>>>(ma, mb, ea, eb, M, N, int(Kp), nk, kper, alpha, 0.0,
                                                              W, N, M * N, err);
    else
      oz_gemm_kernel<S, BN><<<grid, othreads<BN>(), smem, s>>>(ma, mb, ea, eb, M, N, int(Kp), nk, kper, alpha, beta,
                                                              C, ldc, 0, err);
    count_launch();
    check_launch("oz_gemm");
    if (Z > 1) {
      oz_reduce<<<int(std::min<int64_t>((M * N + 255) / 256, 4 * oz_sms())), 256, 0, s>>>(W, Z, M, N, beta, C, ldc);
      count_launch();
      check_launch("oz_reduce");
    }
  }
  if (W) dev_free(W, s);
  dev_free(Pa, s);
  dev_free(Pb, s);
  dev_free(ea, s);
  dev_free(eb, s);
}

}  // namespace

void gemm_oz(int slices, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);  // C = beta C
    return;
  }
  switch (slices) {
    case 2: oz_run<2, 128>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s); break;
    case 3: oz_run<3, 128>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s); break;
    case 8: oz_run<8, 64>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s); break;
    default: throw Error(IPEPS_ERR_ARG, "oz_gemm: slices must be 2, 3 or 8");
  }
}

}  // namespace ipeps
