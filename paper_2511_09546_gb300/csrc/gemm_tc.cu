// 3xTF32 GEMM on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// The bulk contractions of the split-precision path: C = alpha op(A) op(B) +
// beta C with FP64 operands and result.  Each operand is split x = hi + lo
// with hi = tf32(x) and lo = tf32(x - hi); the product
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi is one TF32 GEMM over a tripled K:
//   A' = [A_hi | A_hi | A_lo]   (M x 3K, K-major)
//   B' = [B_hi | B_lo | B_hi]   (N x 3K, K-major)
// written by one tiled pack kernel that also absorbs the transposes of op(A),
// op(B).
//
// Accumulation.  The tensor core rounds its FP32 accumulator toward zero
// after every MMA, so one accumulator run over the whole of K carries an error
// that grows linearly in K/8 and is biased; at K = 8192 that error is as large
// as dropping the lo terms altogether.  The kernel therefore accumulates only
// `chunk` K slices in TMEM, then adds the chunk's partial sums into a
// compensated (two-sum) FP32 pair per output held in registers, so the
// truncation bias no longer builds up across chunks.  Two TMEM accumulators
// alternate, so the MMAs of one chunk overlap the flush of the previous one.
//
// Roles (one CTA per 128 x 128 output tile, 10 warps):
//   * warps 0-7 flush and write the result: warp w reads TMEM lanes
//     32 (w % 4) .. +31 (its rows) and columns 64 (w / 4) .. +63;
//   * lane 0 of warp 8 streams 32-wide K slices of A' and B' with TMA (128-byte
//     swizzle) into a ring of shared-memory stages guarded by mbarriers; warp 8
//     also owns the TMEM allocation (two accumulators, 2 x 128 columns);
//   * lane 0 of warp 9 issues tcgen05.mma (M = 128, N = 128, K = 8, four per
//     slice), releases each stage with tcgen05.commit and signals each
//     finished chunk on the accumulator's mbarrier.
// Every mbarrier wait is bounded: on expiry the kernel raises an error word,
// skips the write of C, drains its own copies (again bounded), frees its TMEM
// and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <string>

#include "common.h"
#include "engine.h"
#include "kernels.h"
#include "profile.h"
#include "tc_ptx.h"

namespace ipeps {

namespace {
using namespace ptx;

constexpr int BM = 128;          // rows per tile (TMEM lanes)
constexpr int BKT = 32;          // TF32 elements per K slice = 128 bytes (one swizzle row)
constexpr int RING_BYTES = 204800;  // shared-memory ring: 6 x 32 KB (BN 128), 5 x 40 KB (BN 192)
constexpr int GROUP_M = 8;       // CTA raster: 8 tile rows per group share the B' tiles in L2
constexpr int WCOLS = 64;        // accumulator columns per flush warp
// warps 0 .. 4 BN/64 - 1 flush (lane quarter w % 4, columns 64 (w / 4) ..),
// then one producer warp and one MMA warp
template <int BN> __host__ __device__ constexpr int flush_warps() { return 4 * (BN / WCOLS); }
template <int BN> __host__ __device__ constexpr int threads() { return 32 * (flush_warps<BN>() + 2); }
constexpr int TMEM_COLS = 512;   // BN 256: two accumulators; BN 128: two accumulators, lo, spare

template <int BN, bool COMP>
__global__ void __launch_bounds__(threads<BN>(), 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   int64_t M, int64_t N, int nk, int chunk, double alpha, double beta,
                   double *__restrict__ C, int64_t ldc, int *err) {
  constexpr uint32_t A_BYTES = BM * BKT * 4, B_BYTES = BN * BKT * 4;
  constexpr int STAGES = RING_BYTES / int(A_BYTES + B_BYTES);
  constexpr int FLUSH_WARPS = flush_warps<BN>(), PRODUCER_WARP = FLUSH_WARPS, MMA_WARP = FLUSH_WARPS + 1;
  static_assert(!COMP || 4 * BN <= TMEM_COLS, "the lo halves need TMEM columns 2 BN .. 3 BN");
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned ring of stages: [A stage | B stage] x STAGES
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped raster: consecutive CTAs walk GROUP_M tile rows column by column
  int mt, ntile;
  {
    const int nt = gridDim.x, mtiles = gridDim.y;
    const int id = blockIdx.y * nt + blockIdx.x, per = GROUP_M * nt;
    const int first = (id / per) * GROUP_M, rows = min(GROUP_M, mtiles - first);
    mt = first + (id % per) % rows;
    ntile = (id % per) / rows;
  }
  const int m0 = mt * BM, n0 = ntile * BN;
  const int nchunks = (nk + chunk - 1) / chunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], FLUSH_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == PRODUCER_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(uint32_t(TMEM_COLS))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  int issued = 0;  // K slices whose loads lane 0 of the producer warp started
  if (warp == PRODUCER_WARP) {
    if (lane == 0) {
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES;
        if (!mbar_wait(&empty[s], ((kt / STAGES) & 1) ^ 1, err)) break;
        uint8_t *sa = base + size_t(s) * (A_BYTES + B_BYTES);
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sa, &mapA, &full[s], kt * BKT, m0);
        tma_load_2d(sa + A_BYTES, &mapB, &full[s], kt * BKT, n0);
        issued = kt + 1;
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(BN >> 3) << 17) |
                                 (uint32_t(BM >> 4) << 24);
      bool ok = true;
      int kt = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1, use = c >> 1;
        ok = mbar_wait(&acc_empty[b], (use & 1) ^ 1, err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + uint32_t(b * BN);
        const int k_first = kt, k_end = min(nk, kt + chunk);
        for (; kt < k_end; ++kt) {
          const int s = kt % STAGES;
          ok = mbar_wait(&full[s], (kt / STAGES) & 1, err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          uint8_t *sa = base + size_t(s) * (A_BYTES + B_BYTES);
          const uint64_t ad = smem_desc(smem_u32(sa)), bd = smem_desc(smem_u32(sa + A_BYTES));
#pragma unroll
          for (int ks = 0; ks < BKT / 8; ++ks)  // 8 TF32 = 32 bytes per MMA: +2 in the address field
            mma_tf32(acc, ad + 2 * ks, bd + 2 * ks, idesc, (kt != k_first || ks != 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[b]);
      }
    }
  } else {
    // ---- flush warps: chunk partials (TMEM, FP32) -> running sums hi (registers)
    // and, when COMP, the two-sum error terms lo (TMEM columns 2 BN ..)
    const uint32_t lanes = uint32_t((warp & 3) * 32) << 16, cw = uint32_t((warp >> 2) * WCOLS);
    const uint32_t t_acc = tmem + lanes + cw, t_lo = tmem + lanes + 2 * BN + cw;
    float hi[WCOLS];
#pragma unroll
    for (int j = 0; j < WCOLS; ++j) hi[j] = 0.0f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1, use = c >> 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], use & 1, err) ? 1 : 0) != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int q = 0; q < WCOLS / 16; ++q) {
        uint32_t v[16], l[16];
        tmem_ld16_issue(t_acc + uint32_t(b * BN + q * 16), v);
        if (COMP && c > 0) tmem_ld16_issue(t_lo + uint32_t(q * 16), l);
        tmem_ld_wait(v);
        if (q == WCOLS / 16 - 1) {
          // the accumulator is in registers: hand it back to the MMA warp before the last adds
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (COMP) {
          if (c > 0) tmem_ld_wait(l);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            // two-sum: hi + x = sum + e exactly
            const float x = __uint_as_float(v[j]), hv = hi[q * 16 + j];
            const float sum = hv + x, bv = sum - hv;
            const float e = (hv - (sum - bv)) + (x - bv);
            hi[q * 16 + j] = sum;
            l[j] = __float_as_uint(c > 0 ? __uint_as_float(l[j]) + e : e);
          }
          tmem_st16(t_lo + uint32_t(q * 16), l);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) hi[q * 16 + j] += __uint_as_float(v[j]);
        }
      }
      if (COMP) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    if (ok) {
      const int64_t row = m0 + (warp & 3) * 32 + lane;
      const int64_t col0 = n0 + (warp >> 2) * WCOLS;
#pragma unroll
      for (int q = 0; q < WCOLS / 16; ++q) {
        uint32_t l[16];
        if (COMP) {
          tmem_ld16_issue(t_lo + uint32_t(q * 16), l);
          tmem_ld_wait(l);
        }
        if (row < M) {
          double *crow = C + row * ldc + col0 + q * 16;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (col0 + q * 16 + j < N) {
              const double sum = double(hi[q * 16 + j]) + (COMP ? double(__uint_as_float(l[j])) : 0.0);
              crow[j] = (beta == 0.0) ? alpha * sum : alpha * sum + beta * crow[j];
            }
          }
        }
        // one 16-column group of C traffic at a time: keeps the beta*C loads
        // from being hoisted next to the live running sums
        asm volatile("" ::: "memory");
      }
    }
  }
  // on an error path, let this CTA's copies land before the shared memory goes away
  if (warp == PRODUCER_WARP && lane == 0 && issued > 0 && *err) {
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
      mbar_wait(&full[kt % STAGES], (kt / STAGES) & 1, err, 200000000ll);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == PRODUCER_WARP) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(TMEM_COLS))
                 : "memory");
  }
}

// tf32(x): round-to-nearest to 10 explicit mantissa bits, kept in an FP32 container
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// P[r][seg * Kp + k] for r < rows_pad, k < Kp: segment pattern (hi, hi, lo) for A
// (pattern 0) or (hi, lo, hi) for B (pattern 1); source element (r, k) of op(X)
// is X[k * ld + r] when trans, X[r * ld + k] otherwise; zero outside (rows, K).
// One 256-thread block per 32 x 32 tile: coalesced reads along whichever index
// is contiguous in X, a shared-memory transpose, coalesced writes along k.
__global__ void __launch_bounds__(256) split_pack_kernel(const double *__restrict__ X, int64_t ld, bool trans,
                                                         int64_t rows, int64_t K, int64_t Kp, int pattern,
                                                         float *__restrict__ P) {
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
    const double x = T[tx][r];
    const float hi = to_tf32(float(x));
    const float lo = to_tf32(float(x - double(hi)));
    float *row = P + (r0 + r) * (3 * Kp) + k0 + tx;
    row[0] = hi;
    row[Kp] = (pattern == 0) ? hi : lo;
    row[2 * Kp] = (pattern == 0) ? lo : hi;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

CUtensorMap make_map(const float *P, int64_t rows_pad, int64_t Kt, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {cuuint64_t(Kt), cuuint64_t(rows_pad)};
  cuuint64_t strides[1] = {cuuint64_t(Kt) * 4};
  cuuint32_t box[2] = {cuuint32_t(BKT), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(P), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(IPEPS_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
  return m;
}

template <int BN, bool COMP>
void launch(const CUtensorMap &ma, const CUtensorMap &mb, int64_t M, int64_t N, int64_t Np, int nk, int chunk,
            double alpha, double beta, double *C, int64_t ldc, int *err, cudaStream_t s) {
  constexpr size_t stage = size_t(BM + BN) * BKT * 4;
  constexpr size_t smem = (RING_BYTES / stage) * stage + 1024;
  once_per_device(reinterpret_cast<const void *>(tc_gemm_kernel<BN, COMP>), []() {
    IPEPS_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<BN, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(Np / BN), unsigned((M + BM - 1) / BM));
  cfg.blockDim = dim3(threads<BN>());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  IPEPS_CUDA(cudaLaunchKernelEx(&cfg, tc_gemm_kernel<BN, COMP>, ma, mb, M, N, nk, chunk, alpha, beta,
                                C, ldc, err));
  count_launch();
  check_launch("tc_gemm");
}

bool compensated() {
  // two-sum compensation of the sum over chunks (default on)
  static bool c = [] {
    const char *e = std::getenv("IPEPS_TC_COMP");
    return !(e && std::atoi(e) == 0);
  }();
  return c;
}

int chunk_slices() {
  // K slices (32 TF32 elements of the tripled K) per TMEM accumulation chunk
  static int c = [] {
    const char *e = std::getenv("IPEPS_TC_CHUNK");
    int v = e ? std::atoi(e) : 8;
    return v < 1 ? 1 : v;
  }();
  return c;
}

}  // namespace

void gemm_tf32x3(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                 const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);  // C = beta C
    return;
  }
  IPEPS_REQUIRE((M + BM - 1) / BM <= 65535, "tc_gemm: M too large");
  const int64_t Kp = (K + BKT - 1) / BKT * BKT, Kt = 3 * Kp;
  // wide outputs: 192-column tiles (less shared-memory traffic per MMA),
  // plain FP32 sum over chunks; narrow outputs: 128-column tiles, compensated
  const int bn = N > 128 ? 192 : 128;
  const int64_t Mp = (M + BM - 1) / BM * BM, Np = (N + bn - 1) / bn * bn;
  IPEPS_REQUIRE(Kt / BKT <= 2147483647 && Kp / 32 <= 2147483647, "tc_gemm: K too large");
  float *Ap = static_cast<float *>(dev_alloc(size_t(Mp) * Kt * sizeof(float), s));
  float *Bp = static_cast<float *>(dev_alloc(size_t(Np) * Kt * sizeof(float), s));
  {
    ProfScope prof("tc_pack", s, 0.0, 8.0 * (M * K + K * N) + 12.0 * (Mp + Np) * Kp);
    // op(A)[m, k]: A stored M x K (lda) or, transposed, K x M
    split_pack_kernel<<<dim3(unsigned(Kp / 32), unsigned(Mp / 32)), 256, 0, s>>>(A, lda, ta, M, K, Kp, 0, Ap);
    // op(B)[k, n] as rows n of B': B stored K x N (ldb), i.e. element (n, k) at B[k * ldb + n]
    // (trans view) or, when tb, N x K with element (n, k) at B[n * ldb + k]
    split_pack_kernel<<<dim3(unsigned(Kp / 32), unsigned(Np / 32)), 256, 0, s>>>(B, ldb, !tb, N, K, Kp, 1, Bp);
    count_launch(2);
    check_launch("tc_pack");
  }
  const CUtensorMap ma = make_map(Ap, Mp, Kt, BM);
  const CUtensorMap mb = make_map(Bp, Np, Kt, bn);
  int *err = tc_error_word();
  {
    ProfScope prof(shape_class("tc_gemm", M, N, K), s, 2.0 * M * N * K, 4.0 * (Mp + Np) * Kt + 8.0 * M * N * (beta == 0.0 ? 1 : 2));
    const int nk = int(Kt / BKT), ch = chunk_slices();
    const bool comp = compensated();
    if (bn == 192) launch<192, false>(ma, mb, M, N, Np, nk, ch, alpha, beta, C, ldc, err, s);
    else if (comp) launch<128, true>(ma, mb, M, N, Np, nk, ch, alpha, beta, C, ldc, err, s);
    else launch<128, false>(ma, mb, M, N, Np, nk, ch, alpha, beta, C, ldc, err, s);
  }
  dev_free(Ap, s);
  dev_free(Bp, s);
}

// The error word of the tensor-core kernels: one device int per device,
// raised by a kernel whose bounded mbarrier wait expired.  Launches do not
// synchronise; the C ABI reads the word once per call (tc_check_errors).
int *tc_error_word() {
  static int *w[kMaxDevices] = {};
  static std::mutex mu;
  const int d = current_device();
  std::lock_guard<std::mutex> lk(mu);
  if (!w[d]) {
    int *p = nullptr;
    IPEPS_CUDA(cudaMalloc(&p, sizeof(int)));
    IPEPS_CUDA(cudaMemset(p, 0, sizeof(int)));
    w[d] = p;
  }
  return w[d];
}

void tc_check_errors(cudaStream_t s) {
  int *w = tc_error_word();
  int h = 0;
  IPEPS_CUDA(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, s));
  IPEPS_CUDA(stream_sync(s));
  if (h) {
    IPEPS_CUDA(cudaMemsetAsync(w, 0, sizeof(int), s));
    IPEPS_CUDA(stream_sync(s));
    throw Error(IPEPS_ERR_TIMEOUT, "a tensor-core GEMM's bounded mbarrier wait expired");
  }
}

}  // namespace ipeps
