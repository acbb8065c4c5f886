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
//   d_0 in [-128, 128] and d_p in [-64, 63] for p >= 1 (the balanced base-128
//   digits of the integer round(a_ik 2^(7S - E_i))).  Columns of op(B)
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
#include <memory>
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

// E with 2^E > x for the largest |x| of a row given by its bit pattern (0 for zero)
__device__ __forceinline__ int oz_exp(unsigned long long bits) {
  int e = 0;
  frexp(__longlong_as_double((long long)bits), &e);
  return e;
}

// A~ in slice kt, digit p: rows m0.., columns p Kp + kt OBK (the packed operand is
// rows x S Kp with digit p in columns p Kp .. p Kp + Kp - 1)
template <int S, int BN>
__global__ void __launch_bounds__(othreads<BN>(), 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const unsigned long long *__restrict__ ma_x, const unsigned long long *__restrict__ mb_x,
                   int64_t M, int64_t N, int Kp,
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
        const int er = oz_exp(ma_x[row]);
        double *crow = C + blockIdx.z * zstride + row * ldc + col0;
        const double fix = ldexp(1.0, -OBETA * (LEX - 1));
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (col0 + j < N) {
            const double t = double(acc[j]) * fix + double(tail[j]);
            const double v = alpha * ldexp(t, er + oz_exp(mb_x[col0 + j]) - 2 * OBETA);
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

// Operand packing.  A row r of op(X) (row r of A, or column r of B) is
// scaled by 2^-E_r with 2^E_r > max_k |op(X)[r, k]|, taken from the largest bit
// pattern of |x| in the row (the IEEE order of non-negative doubles is the
// order of their bit patterns).  Both kernels walk 32 x 64 tiles of op(X) (32
// rows, 64 K elements) read along whichever index is contiguous in memory.

__device__ __forceinline__ double oz_load(const double *__restrict__ X, int64_t ld, bool trans, int64_t rows,
                                          int64_t K, int64_t r, int64_t k) {
  return (r < rows && k < K) ? (trans ? X[k * ld + r] : X[r * ld + k]) : 0.0;
}

// mx[r] = max over the tile's k of the bit pattern of |op(X)[r, k]| (atomic max
// across tiles; mx zeroed beforehand)
__global__ void __launch_bounds__(256) oz_absmax_kernel(const double *__restrict__ X, int64_t ld, bool trans,
                                                        int64_t rows, int64_t K,
                                                        unsigned long long *__restrict__ mx) {
  __shared__ unsigned long long part[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k0 = int64_t(blockIdx.x) * 64, r0 = int64_t(blockIdx.y) * 32;
  if (!trans) {
    // warp ty: rows ty, ty + 8, ..; lanes along k (contiguous)
    for (int i = ty; i < 32; i += 8) {
      const int64_t r = r0 + i;
      unsigned long long m = 0;
      for (int j = tx; j < 64; j += 32)
        m = max(m, (unsigned long long)__double_as_longlong(fabs(oz_load(X, ld, false, rows, K, r, k0 + j))));
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (tx == 0 && r < rows && m) atomicMax(mx + r, m);
    }
  } else {
    // lanes along r (contiguous), warp ty takes k = ty, ty + 8, ..
    unsigned long long m = 0;
    for (int j = ty; j < 64; j += 8)
      m = max(m, (unsigned long long)__double_as_longlong(fabs(oz_load(X, ld, true, rows, K, r0 + tx, k0 + j))));
    part[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
      for (int w = 1; w < 8; ++w) m = max(m, part[w][tx]);
      if (r0 + tx < rows && m) atomicMax(mx + r0 + tx, m);
    }
  }
}

// P[r][p Kp + k] = digit p of op(X)[r, k]: F = round(x 2^(7S - E_r)) (|F| < 2^(7S),
// 64-bit integer), split into balanced base-128 digits from the bottom
// (d_p in [-64, 63] for p >= 1, the top digit d_0 in [-128, 128]), each stored as
// the BF16 value d_p 2^(-7p).  Two consecutive k per thread: 32-bit stores,
// 128 contiguous bytes per warp and digit.
template <int S>
__global__ void __launch_bounds__(256) oz_digits_kernel(const double *__restrict__ X, int64_t ld, bool trans,
                                                        int64_t rows, int64_t K, int64_t Kp,
                                                        const unsigned long long *__restrict__ mx,
                                                        __nv_bfloat16 *__restrict__ P) {
  __shared__ double T[64][33];  // T[k][r]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k0 = int64_t(blockIdx.x) * 64, r0 = int64_t(blockIdx.y) * 32;
  if (trans) {
#pragma unroll
    for (int i = 0; i < 64; i += 8) T[ty + i][tx] = oz_load(X, ld, true, rows, K, r0 + tx, k0 + ty + i);
  } else {
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
      T[tx][ty + i] = oz_load(X, ld, false, rows, K, r0 + ty + i, k0 + tx);
      T[tx + 32][ty + i] = oz_load(X, ld, false, rows, K, r0 + ty + i, k0 + tx + 32);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 32; i += 8) {
    const int r = ty + i;
    const int64_t row = r0 + r;
    const int sh = OBETA * S - oz_exp(mx[row]);
    long long F[2];
    F[0] = llrint(ldexp(T[2 * tx][r], sh));
    F[1] = llrint(ldexp(T[2 * tx + 1][r], sh));
    int d[2][S];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int p = S - 1; p >= 1; --p) {
        const int v = int(((F[h] + 64) & 127) - 64);
        d[h][p] = v;
        F[h] = (F[h] - v) >> OBETA;
      }
      d[h][0] = int(F[h]);
    }
    uint32_t *dst = reinterpret_cast<uint32_t *>(P + row * (S * Kp) + k0) + tx;
#pragma unroll
    for (int p = 0; p < S; ++p) {
      const float sc = __int_as_float((127 - OBETA * p) << 23);  // 2^(-7p)
      const __nv_bfloat16 lo = __float2bfloat16_rn(float(d[0][p]) * sc);
      const __nv_bfloat16 hi = __float2bfloat16_rn(float(d[1][p]) * sc);
      dst[(p * Kp) / 2] = uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
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
  // a driver entry point, the same for every device (thread-safe static
  // initialisation; a throw leaves it for the next call)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
      throw Error(IPEPS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
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

int oz_sms() { return device_sm_count(); }

}  // namespace

// Packed operand: the digits of op(X) (rows x K) as rows_pad x S Kp BF16 and the
// per-row maxima (bit patterns) that fix the row exponents.
struct OzPacked {
  int S = 0;
  int64_t rows = 0, rows_pad = 0, K = 0, Kp = 0;
  __nv_bfloat16 *P = nullptr;
  unsigned long long *mx = nullptr;
  cudaStream_t s = nullptr;
  ~OzPacked() {
    if (P) dev_free(P, s);
    if (mx) dev_free(mx, s);
  }
};

namespace {

template <int S>
std::shared_ptr<OzPacked> oz_pack(const double *X, int64_t ld, bool trans, int64_t rows, int64_t K, int64_t align,
                                  cudaStream_t s) {
  auto out = std::make_shared<OzPacked>();
  out->S = S;
  out->rows = rows;
  out->K = K;
  out->Kp = (K + 63) / 64 * 64;  // whole 64-element pack tiles (two K slices)
  out->rows_pad = (rows + align - 1) / align * align;
  out->s = s;
  IPEPS_REQUIRE(out->rows_pad / 32 <= 65535 && S * out->Kp <= 2147483647 && out->Kp / OBK <= (int64_t(1) << 24),
                "oz_gemm: problem too large");
  out->P = static_cast<__nv_bfloat16 *>(dev_alloc(size_t(out->rows_pad) * S * out->Kp * 2, s));
  out->mx = static_cast<unsigned long long *>(dev_alloc(size_t(out->rows_pad) * 8, s));
  ProfScope prof("oz_pack", s, 0.0, 8.0 * rows * K + 2.0 * S * out->rows_pad * out->Kp);
  IPEPS_CUDA(cudaMemsetAsync(out->mx, 0, size_t(out->rows_pad) * 8, s));
  const dim3 grid(unsigned(out->Kp / 64), unsigned(out->rows_pad / 32));
  oz_absmax_kernel<<<grid, 256, 0, s>>>(X, ld, trans, rows, K, out->mx);
  oz_digits_kernel<S><<<grid, 256, 0, s>>>(X, ld, trans, rows, K, out->Kp, out->mx, out->P);
  count_launch(2);
  check_launch("oz_pack");
  return out;
}

template <int S, int BN>
void oz_multiply(const OzPacked &a, const OzPacked &b, int64_t M, int64_t N, double alpha, double beta, double *C,
                 int64_t ldc, cudaStream_t s) {
  IPEPS_REQUIRE(a.S == S && b.S == S && a.Kp == b.Kp && a.rows_pad % OBM == 0 && b.rows_pad % BN == 0 &&
                    a.rows == M && b.rows == N,
                "oz_gemm: packed operands do not match");
  const int64_t Kp = a.Kp, Mp = a.rows_pad, Np = b.rows_pad, K = a.K;
  const CUtensorMap ma = oz_map(a.P, Mp, S * Kp, OBM);
  const CUtensorMap mb = oz_map(b.P, Np, S * Kp, BN);
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
    static const char *names[9] = {"", "", "oz2_gemm", "oz3_gemm", "", "", "", "", "oz8_gemm"};
    ProfScope prof(shape_class(names[S], M, N, K), s, 2.0 * M * N * K,
                   2.0 * S * (Mp + Np) * Kp + 8.0 * M * N * (beta == 0.0 ? 1 : 2));
    constexpr size_t smem = size_t(ostages<S, BN>()) * stage_bytes<S, BN>() + 1024;
    once_per_device(reinterpret_cast<const void *>(oz_gemm_kernel<S, BN>), []() {
      IPEPS_CUDA(cudaFuncSetAttribute(oz_gemm_kernel<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    });
    dim3 grid(unsigned(Np / BN), unsigned(Mp / OBM), unsigned(Z));
    if (Z > 1)
      oz_gemm_kernel<S, BN><<<grid, othreads<BN>(), smem, s>>>(ma, mb, a.mx, b.mx, M, N, int(Kp), nk, kper, alpha,
                                                              0.0, W, N, M * N, err);
    else
      oz_gemm_kernel<S, BN><<<grid, othreads<BN>(), smem, s>>>(ma, mb, a.mx, b.mx, M, N, int(Kp), nk, kper, alpha,
                                                              beta, C, ldc, 0, err);
    count_launch();
    check_launch("oz_gemm");
    if (Z > 1) {
      oz_reduce<<<int(std::min<int64_t>((M * N + 255) / 256, 4 * oz_sms())), 256, 0, s>>>(W, Z, M, N, beta, C, ldc);
      count_launch();
      check_launch("oz_reduce");
    }
  }
  if (W) dev_free(W, s);
}

template <int S, int BN>
void oz_run(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
            const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s,
            const OzPacked *pa) {
  std::shared_ptr<OzPacked> own;
  if (!pa) {
    own = oz_pack<S>(A, lda, ta, M, K, OBM, s);
    pa = own.get();
  }
  // op(B) as rows n: element (n, k) is B[k * ldb + n] (strided in k) unless tb
  auto pb = oz_pack<S>(B, ldb, !tb, N, K, BN, s);
  oz_multiply<S, BN>(*pa, *pb, M, N, alpha, beta, C, ldc, s);
}

}  // namespace

void gemm_oz(int slices, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s,
             const OzPacked *packed_a) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);  // C = beta C
    return;
  }
  IPEPS_REQUIRE(!packed_a || packed_a->S == slices, "oz_gemm: packed operand has another digit count");
  switch (slices) {
    case 2: oz_run<2, 128>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, packed_a); break;
    case 3: oz_run<3, 128>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, packed_a); break;
    case 8: oz_run<8, 64>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, packed_a); break;
    default: throw Error(IPEPS_ERR_ARG, "oz_gemm: slices must be 2, 3 or 8");
  }
}

std::shared_ptr<OzPacked> pack_left_fp64(bool ta, int64_t M, int64_t K, const double *A, int64_t lda,
                                         cudaStream_t s) {
  if (fp64_policy() != Prec::FP64_TC || M <= 0 || K <= 0) return nullptr;
  return oz_pack<8>(A, lda, ta, M, K, OBM, s);
}

void gemm_f64_packed(const OzPacked *pa, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                     const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                     int64_t ldc, cudaStream_t s) {
  if (pa && K > 0 && M > 0 && N > 0 && oz_worthwhile(M, N, K)) {
    IPEPS_REQUIRE(pa->rows == M && pa->K == K, "gemm_f64_packed: packed operand has another shape");
    gemm_oz(8, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, pa);
  } else {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  }
}

}  // namespace ipeps
