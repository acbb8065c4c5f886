// FP64 data-movement, BLAS-1 and reduction kernels (HBM bound: grid-stride
// loops over 2 x SM-count blocks, 64-bit indices, deterministic reductions).
#include <cuda_runtime.h>

#include "common.h"
#include "kernels.h"
#include "profile.h"

namespace ipeps {

namespace {

int grid_for(int64_t n, int threads = 256) {
  const int sms = device_sm_count();
  int64_t want = (n + threads - 1) / threads;
  int64_t cap = int64_t(sms) * 8;
  if (want < 1) want = 1;
  return int(want < cap ? want : cap);
}

struct PermParams {
  int nd;
  int64_t out_dims[kMaxDims];
  int64_t in_stride_for_out[kMaxDims];  // stride in src of output axis k
};

__global__ void permute_kernel(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                               PermParams p, double alpha, double beta) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n;
       j += int64_t(gridDim.x) * blockDim.x) {
    int64_t rem = j, off = 0;
    for (int k = p.nd - 1; k >= 0; --k) {
      int64_t ik = rem % p.out_dims[k];
      rem /= p.out_dims[k];
      off += ik * p.in_stride_for_out[k];
    }
    double v = alpha * src[off];
    dst[j] = (beta == 0.0) ? v : v + beta * dst[j];
  }
}

// 2-D tiled transpose for the common case: dst[b, c, a] from src[b, a, c]
// style permutations reduce to batched (rows x cols) -> (cols x rows).
__global__ void transpose_batched_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                         int64_t rows, int64_t cols, int64_t batch, double alpha,
                                         double beta) {
  __shared__ double tile[32][33];
  int64_t b = blockIdx.z;
  const double *S = src + b * rows * cols;
  double *Dd = dst + b * rows * cols;
  int64_t r0 = int64_t(blockIdx.y) * 32, c0 = int64_t(blockIdx.x) * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = S[r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) {
      double v = alpha * tile[threadIdx.x][k];
      int64_t o = c * rows + r;
      Dd[o] = (beta == 0.0) ? v : v + beta * Dd[o];
    }
  }
}

__global__ void fill_kernel(double *x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] = v;
}

__global__ void axpby_kernel(int64_t n, double a, const double *__restrict__ x, double b,
                             double *__restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = (b == 0.0 ? 0.0 : b * y[i]) + a * x[i];
}

__global__ void axpy_ratio_kernel(int64_t n, const double *num, const double *den, double sign,
                                  const double *__restrict__ x, double *__restrict__ y) {
  double a = sign * (*num) / (*den);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] += a * x[i];
}

__global__ void scal_kernel(int64_t n, double a, double *x) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= a;
}

// deterministic reduction: each block writes a partial, one block sums them
template <int T>
__device__ double block_sum(double v) {
  __shared__ double sh[T / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < T / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

__global__ void dot_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                            double *partial) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    acc += x[i] * y[i];
  double r = block_sum<256>(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void sum_partials(const double *partial, int np, double *out, int sqrt_out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  double r = block_sum<256>(acc);
  if (threadIdx.x == 0) out[0] = sqrt_out ? sqrt(r) : r;
}

__global__ void coldot_kernel(int64_t m, int64_t n, const double *__restrict__ X,
                              const double *__restrict__ Y, double *out) {
  // one block per column j; rows strided
  int64_t j = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) acc += X[i * n + j] * Y[i * n + j];
  double r = block_sum<256>(acc);
  if (threadIdx.x == 0) out[j] = r;
}

__global__ void scale_cols_kernel(int64_t m, int64_t n, const double *__restrict__ X,
                                  const double *__restrict__ f, double *__restrict__ Y, double beta) {
  int64_t total = m * n;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    double v = X[i] * f[i % n];
    Y[i] = (beta == 0.0) ? v : v + beta * Y[i];
  }
}

__global__ void div_scalar_kernel(int64_t n, double *x, const double *nrm) {
  double inv = (*nrm != 0.0) ? 1.0 / (*nrm) : 0.0;  // a zero tensor stays zero
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= inv;
}

__global__ void leg_signs_kernel(double *t, int64_t a, int64_t mid, int64_t b, const double *sp,
                                 const double *sn) {
  int64_t total = a * mid * b;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    int64_t ib = i % b;
    int64_t ia = i / (mid * b);
    t[i] *= sp[ia] * sn[ib];
  }
}

__global__ void nonfinite_kernel(int64_t n, const double *x, int *out) {
  int c = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    c += !isfinite(x[i]);
  if (c) atomicAdd(out, c);
}

}  // namespace

void permute(const double *src, const std::vector<int64_t> &dims, const std::vector<int> &perm,
             double *dst, cudaStream_t s, double alpha, double beta) {
  int nd = int(dims.size());
  IPEPS_REQUIRE(nd >= 1 && nd <= kMaxDims && int(perm.size()) == nd, "permute: bad rank");
  int64_t n = prod(dims);
  if (n == 0) return;
  // collapse to a batched 2-D transpose when perm = (0..p-1, q.., p..q-1) with
  // the two moved groups contiguous: src[b, a, c] -> dst[b, c, a]
  {
    int lead = 0;
    while (lead < nd && perm[lead] == lead) ++lead;
    if (lead < nd) {
      // dst axes after lead: must be [k..nd-1, lead..k-1] for some k
      int k = perm[lead];
      bool ok = k > lead;
      for (int i = lead; ok && i < nd; ++i) {
        int expect = (i - lead < nd - k) ? k + (i - lead) : lead + (i - lead - (nd - k));
        ok = perm[i] == expect;
      }
      if (ok) {
        int64_t batch = 1, rows = 1, cols = 1;
        for (int i = 0; i < lead; ++i) batch *= dims[i];
        for (int i = lead; i < k; ++i) rows *= dims[i];
        for (int i = k; i < nd; ++i) cols *= dims[i];
        if (batch <= 65535 && (rows + 31) / 32 <= 65535) {
          ProfScope prof("permute", s, 0.0, 16.0 * n * (beta == 0.0 ? 1.0 : 1.5));
          dim3 blk(32, 8), grd(unsigned((cols + 31) / 32), unsigned((rows + 31) / 32), unsigned(batch));
          transpose_batched_kernel<<<grd, blk, 0, s>>>(src, dst, rows, cols, batch, alpha, beta);
          count_launch();
          check_launch("transpose_batched");
          return;
        }
      }
    } else {
      // identity permutation
      if (beta == 0.0 && alpha == 1.0) {
        if (src != dst) IPEPS_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      } else {
        axpby(n, alpha, src, beta, dst, s);
      }
      return;
    }
  }
  PermParams p;
  p.nd = nd;
  int64_t in_stride[kMaxDims];
  int64_t st = 1;
  for (int i = nd - 1; i >= 0; --i) {
    in_stride[i] = st;
    st *= dims[i];
  }
  for (int k = 0; k < nd; ++k) {
    p.out_dims[k] = dims[perm[k]];
    p.in_stride_for_out[k] = in_stride[perm[k]];
  }
  ProfScope prof("permute", s, 0.0, 16.0 * n * (beta == 0.0 ? 1.0 : 1.5));
  permute_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n, p, alpha, beta);
  count_launch();
  check_launch("permute");
}

void fill(double *x, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return;
  if (v == 0.0) {
    IPEPS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    return;
  }
  fill_kernel<<<grid_for(n), 256, 0, s>>>(x, n, v);
  count_launch();
  check_launch("fill");
}

void axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s) {
  if (n <= 0) return;
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, a, x, b, y);
  count_launch();
  check_launch("axpby");
}

void axpy(int64_t n, double a, const double *x, double *y, cudaStream_t s) { axpby(n, a, x, 1.0, y, s); }

void axpy_ratio(int64_t n, const double *num, const double *den, double sign, const double *x,
                double *y, cudaStream_t s) {
  if (n <= 0) return;
  axpy_ratio_kernel<<<grid_for(n), 256, 0, s>>>(n, num, den, sign, x, y);
  count_launch();
  check_launch("axpy_ratio");
}

void scal(int64_t n, double a, double *x, cudaStream_t s) {
  if (n <= 0) return;
  scal_kernel<<<grid_for(n), 256, 0, s>>>(n, a, x);
  count_launch();
  check_launch("scal");
}

static void reduce2(int64_t n, const double *x, const double *y, double *out, bool sq,
                    cudaStream_t s) {
  int g = grid_for(n);
  if (g > 1024) g = 1024;
  double *partial = static_cast<double *>(dev_alloc(g * sizeof(double), s));
  dot_partial<<<g, 256, 0, s>>>(n, x, y, partial);
  sum_partials<<<1, 256, 0, s>>>(partial, g, out, sq ? 1 : 0);
  count_launch(2);
  check_launch("dot");
  dev_free(partial, s);
}

void dot(int64_t n, const double *x, const double *y, double *out, cudaStream_t s) {
  reduce2(n, x, y, out, false, s);
}
void nrm2(int64_t n, const double *x, double *out, cudaStream_t s) { reduce2(n, x, x, out, true, s); }

void coldot(int64_t m, int64_t n, const double *X, const double *Y, double *out, cudaStream_t s) {
  if (n <= 0) return;
  coldot_kernel<<<unsigned(n), 256, 0, s>>>(m, n, X, Y, out);
  count_launch();
  check_launch("coldot");
}

void scale_cols(int64_t m, int64_t n, const double *X, const double *f, double *Y, cudaStream_t s,
                double beta) {
  if (m * n <= 0) return;
  scale_cols_kernel<<<grid_for(m * n), 256, 0, s>>>(m, n, X, f, Y, beta);
  count_launch();
  check_launch("scale_cols");
}

void div_by_scalar(int64_t n, double *x, const double *nrm, cudaStream_t s) {
  if (n <= 0) return;
  div_scalar_kernel<<<grid_for(n), 256, 0, s>>>(n, x, nrm);
  count_launch();
  check_launch("div_by_scalar");
}

void leg_signs(double *t, int64_t a, int64_t mid, int64_t b, const double *sp, const double *sn,
               cudaStream_t s) {
  int64_t n = a * mid * b;
  if (n <= 0) return;
  leg_signs_kernel<<<grid_for(n), 256, 0, s>>>(t, a, mid, b, sp, sn);
  count_launch();
  check_launch("leg_signs");
}

void count_nonfinite(int64_t n, const double *x, int *out, cudaStream_t s) {
  IPEPS_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
  if (n <= 0) return;
  nonfinite_kernel<<<grid_for(n), 256, 0, s>>>(n, x, out);
  count_launch();
  check_launch("count_nonfinite");
}

}  // namespace ipeps
