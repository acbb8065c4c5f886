// Contraction engine and reverse-mode tape of libipeps.
//
// Every tensor network step of the path is a pairwise contraction written by
// index labels; a contraction lowers to (at most) one permutation per operand
// and one GEMM.  The Tape records the primitive operations of a forward pass
// (contract, permute, reshape, truncated SVD, column scaling, normalisation,
// fixed sign gauges, density-matrix ratios) with their inputs kept resident in
// HBM, and replays their hand-written adjoints in reverse order to form
// vector-Jacobian products.  The same recorded pass can be replayed with many
// cotangents (the fixed-point adjoint solve needs one replay per Krylov step).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.h"
#include "kernels.h"

namespace ipeps {

enum class Prec { FP64 = 0, TF32X3 = 1, TF32X3_ALL = 2, FP64_TC = 3, BF16X3 = 4 };

// Arithmetic of the FP64-grade GEMMs (gemm_f64) issued by this thread: the
// CUDA-core DFMA kernels (Prec::FP64) or, for Prec::FP64_TC, the
// exponent-aligned BF16-slice tensor-core GEMM with 8 digits where the shape
// is large enough.  Set for the duration of a C-ABI call by PolicyScope.
Prec &fp64_policy();
struct PolicyScope {
  Prec old;
  explicit PolicyScope(Prec p) : old(fp64_policy()) { fp64_policy() = p; }
  ~PolicyScope() { fp64_policy() = old; }
  PolicyScope(const PolicyScope &) = delete;
  PolicyScope &operator=(const PolicyScope &) = delete;
};
// FP64-grade products for contractions run in precision p
inline Prec fp64_grade_of(Prec p) { return (p == Prec::FP64_TC || p == Prec::BF16X3) ? Prec::FP64_TC : Prec::FP64; }
// the shape is large enough for the slice GEMM to beat the DFMA kernels:
// M N K at least oz_threshold() (this thread's crossover, 2^23 by default;
// the server's autotuner sets it per problem shape)
bool oz_worthwhile(int64_t m, int64_t n, int64_t k);
double &oz_threshold();
// C = alpha op(A) op(B) + beta C on the BF16 tensor cores with `slices` 7-bit
// digits per operand (2: BF16x3, 3, or 8: FP64-grade); row-major, FP64 in and out
struct OzPacked;
void gemm_oz(int slices, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t s,
             const OzPacked *packed_a = nullptr);
// A left operand that several FP64-grade products share, packed once into
// digits (nullptr when the FP64 policy is the DFMA path); gemm_f64_packed uses
// the packed digits when the shape takes the tensor-core path and A otherwise
std::shared_ptr<OzPacked> pack_left_fp64(bool ta, int64_t M, int64_t K, const double *A, int64_t lda,
                                         cudaStream_t s);
void gemm_f64_packed(const OzPacked *pa, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                     const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                     int64_t ldc, cudaStream_t s);
// error word of the tensor-core kernels and its check (synchronises s)
int *tc_error_word();
void tc_check_errors(cudaStream_t s);

struct Ten {
  double *p = nullptr;
  std::vector<int64_t> d;
  int64_t size() const { return prod(d); }
};

// C(lc) = alpha * A(la) B(lb) + beta * C, labels one char per axis; every
// label of A and of B appears in exactly two of (A, B, C).
void contract(const Ten &A, const std::string &la, const Ten &B, const std::string &lb, const Ten &C,
              const std::string &lc, cudaStream_t s, double alpha = 1.0, double beta = 0.0,
              Prec prec = Prec::FP64);

// 3xTF32 tensor-core GEMM (tcgen05, sm_103a); falls back to an error if the
// device does not support it.  Row-major, C = alpha op(A) op(B) + beta C.
void gemm_tf32x3(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                 int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                 cudaStream_t s);

struct Tape;

struct Node {
  virtual ~Node() = default;
  virtual void backward(Tape &t) = 0;
};

struct Var {
  Ten val;
  DBuf own;         // storage if the tape owns the value
  DBuf grad;        // lazily allocated cotangent
  int alias = -1;   // reshape view of another variable (shares value and cotangent)
};

struct Tape {
  cudaStream_t s;
  Prec prec = Prec::FP64;
  bool record = true;
  std::vector<Var> vars;
  std::vector<std::unique_ptr<Node>> nodes;
  // warm-start blocks of the truncated SVD, keyed per projector cut (forward
  // passes that are not recorded use subspace iteration from these)
  std::map<int, DBuf> *vcache = nullptr;
  int vkey = 0;
  int svd_iters = 0;  // subspace iterations spent (statistics)

  explicit Tape(cudaStream_t st) : s(st) {}
  int leaf(double *p, const std::vector<int64_t> &d);   // external memory, not owned
  int make(const std::vector<int64_t> &d);               // owned, uninitialised
  const Ten &val(int id) const { return vars[id].val; }
  double *vp(int id) const { return vars[id].val.p; }
  // cotangent of id (allocated and zeroed on first use); nullptr if absent and !create
  double *grad(int id, bool create = true);
  void zero_grads();
  void push(Node *n) {
    if (record) nodes.emplace_back(n);
    else delete n;
  }
  void backward();      // replay adjoints (all nodes, reverse order)
  void clear();         // drop nodes and variables
  // forward-only passes: free the storage behind id (and behind the variable a
  // reshape view of it aliases); the caller uses none of them again.  A
  // recording tape keeps every value for the backward pass, so this is a no-op.
  void release(int id);
};

// ---- recorded primitives (return the new variable id)
int t_contract(Tape &t, int a, const std::string &la, int b, const std::string &lb,
               const std::string &lc);
int t_reshape(Tape &t, int a, const std::vector<int64_t> &d);
int t_permute(Tape &t, int a, const std::vector<int> &perm);
// Y = X diag(f), X row-major (m x n) viewed from any shape with last dims product n
int t_scale_cols(Tape &t, int X, int f);
// f = s^-1/2 where s > cutoff * s[0], else 0
int t_inv_sqrt_cut(Tape &t, int S, double cutoff);
// y = x / |x|_F
int t_normalize(Tape &t, int x);
// y = sp[i] sn[j] x[i, ..., j] (constant signs, device vectors)
int t_signs(Tape &t, int x, const double *sp, const double *sn);
// top-k SVD of a square row-major matrix: U (N x k), S (k), V (N x k) with
// the largest-magnitude entry of each column of U positive
void t_svd(Tape &t, int M, int k, int *U, int *S, int *V);
// scalar Tr(rho h) / Tr(rho), rho[k1, b1, k2, b2] (two-site) or rho[k, b]
int t_rho_ratio(Tape &t, int rho, const double *h_dev, int d, bool two_site);
// sum of scalar variables times a constant
int t_sum_scalars(Tape &t, const std::vector<int> &xs, double scale);

// full SVD of a row-major N x N matrix: U, V row-major N x N, S descending
void svd_full(const double *M, int64_t N, double *U, double *S, double *V, cudaStream_t s);
// top-k singular triplets (k even, chi <= k <= N) by subspace iteration warm
// started from cache = [V (N x k) | S (k)], which receives the new block.
// U, V row-major N x k, S descending.  Returns false (nothing written to the
// cache) when the block is numerically rank deficient; callers then use svd_full.
bool svd_subspace(const double *M, int64_t N, int chi, int k, double *cache, double *U, double *S,
                  double *V, cudaStream_t s, int *iters, bool tc = false);
// records the adjoint of the top-chi triplets computed from a kb-block
void push_trunc_svd_node(Tape &t, int M, int U, int S, int V, int64_t N, int chi, int kb, DBuf &&Uk,
                         DBuf &&Sk, DBuf &&Vk);

}  // namespace ipeps
