/*
 * ipeps.h -- C ABI of the GB300 (sm_103a) preconditioned iPEPS hot path.
 *
 * The library computes, for an iPEPS unit cell of real tensors,
 *   - the CTMRG environment run to a fixed point (Sec. III.A of the paper:
 *     the energy is contracted with CTMRG);
 *   - the energy per site, Eq. (equ:energy), and its gradient dE/dA at the
 *     fixed point (Sec. III.A: the gradient of the energy functional);
 *   - the local-metric preconditioner, Eq. (equ:local_metric), regularised by
 *     delta I (Sec. III.B) and inverted with GMRES (Sec. III.C);
 *   - plain and preconditioned L-BFGS with the Hager-Zhang line search
 *     (Sec. II and Sec. IV.A).
 *
 * Conventions shared by every call
 *   - Tensor layout: the unit cell has Lx columns and Ly rows; tensor (x, y)
 *     is stored at offset (x * Ly + y) * d * D^4 doubles, each tensor
 *     row-major with legs (s, u, l, d, r) = (physical, up, left, down, right).
 *   - Pointers named *_dev are device pointers owned by the caller; *_host
 *     and scalar outputs are host pointers.  The library owns ipeps_env,
 *     ipeps_ham and its workspaces (stream-ordered pool allocations).
 *   - Every call is enqueued on `stream` (NULL = the legacy default stream)
 *     and returns after the host scalars it reports are available, i.e. it
 *     synchronises the stream before returning.
 *   - Nothing aborts or traps: errors come back as an ipeps_status and a
 *     thread-local message from ipeps_last_error().  Inputs are FP64; the
 *     precision enum only selects the arithmetic of the bulk contractions.
 *   - No call launches a kernel that waits on another launch.
 *   - Calls run on the calling thread's current CUDA device (device index
 *     below 64).  The allocation pool setting, the tensor-core error word,
 *     kernel attributes and SM counts are kept per device, so one process
 *     may drive several devices from different threads; an ipeps_env or a
 *     server belongs to the device that was current when it was created.
 */
#ifndef IPEPS_H
#define IPEPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IPEPS_OK = 0,
  IPEPS_ERR_ARG = 1,           /* invalid argument (shape, size, NULL pointer) */
  IPEPS_ERR_NOMEM = 2,         /* device allocation failed */
  IPEPS_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  IPEPS_ERR_NONFINITE = 4,     /* NaN or Inf in an input or produced value */
  IPEPS_ERR_NOT_CONVERGED = 5, /* iteration limit reached; best result kept */
  IPEPS_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
  IPEPS_ERR_CANCELLED = 7      /* stopped by the caller's callback */
} ipeps_status;

typedef enum {
  IPEPS_FP64 = 0,       /* every contraction in FP64 */
  IPEPS_TF32X3 = 1,     /* split precision: enlarged corners, half-system products
                           and absorption as 3xTF32 GEMMs on tcgen05 tensor cores
                           (FP32 accumulation in chunks, compensated across them);
                           the four-corner product, the projector products and
                           their truncated SVD, normalisation, the convergence
                           test, the gradient adjoint and the preconditioner stay
                           FP64.  CTMRG runs split-precision iterations until the
                           spectra change < 1e-6 (or stops improving), then FP64
                           iterations until tol: the fixed point, energy and
                           gradient are those of the FP64 path. */
  IPEPS_TF32X3_ALL = 2, /* throughput mode for large chi D^2: every bulk GEMM,
                           the four-corner and projector products included, and
                           the adjoint's GEMMs as 3xTF32; SVD, normalisation and
                           preconditioner FP64; no FP64 phase, so the spectra
                           change stalls near the 3xTF32 noise floor and a tol
                           below it ends in IPEPS_ERR_NOT_CONVERGED */
  IPEPS_FP64_TC = 3,    /* FP64-grade results from the BF16 tensor cores: every
                           GEMM large enough to gain (contractions, SVD and
                           adjoint products, metric) is formed from 8 exponent-
                           aligned 7-bit digits per operand, 36 BF16 products
                           per term summed exactly in FP32 chunks and in 64-bit
                           fixed point (error bound of an FP64 GEMM taken relative
                           to the row and column maxima); small GEMMs, SVD
                           rotations, reductions and GMRES stay FP64 */
  IPEPS_BF16X3 = 4      /* BF16x3 contractions: enlarged corners, half systems and
                           absorption from 2 digits per operand (3 BF16 products
                           per term, about 2^-15 of the row and column maxima);
                           the four-corner and projector products and every other
                           GEMM as IPEPS_FP64_TC.  CTMRG runs BF16x3 iterations
                           until the spectra change < 1e-6 (or stops improving),
                           then IPEPS_FP64_TC iterations to tol; the gradient is
                           that of the IPEPS_FP64_TC fixed point. */
} ipeps_prec;

typedef struct {
  int Lx, Ly; /* unit cell: columns, rows (>= 1) */
  int d;      /* physical dimension (>= 1) */
  int D;      /* virtual bond dimension (>= 1) */
} ipeps_shape;

typedef struct CUstream_st *ipeps_stream_t; /* same type as cudaStream_t */
typedef struct ipeps_env_s *ipeps_env;      /* opaque, device resident */
typedef struct ipeps_ham_s *ipeps_ham;      /* opaque, host resident */

/* ------------------------------------------------------------------ S0 */
/* Dense Hamiltonian terms (host pointers, copied).  h_h: (d*d) x (d*d)
 * operator on the horizontal bond (left site, right site); h_v: same on the
 * vertical bond (upper site, lower site); h_site: d x d on-site term or NULL;
 * scale multiplies the per-tensor energy to give the energy per site.
 * Matrix element op[(b1*d + b2) * d*d + (k1*d + k2)] = <b1 b2|op|k1 k2>.
 * Sec. IV.A Eq. (eq:H_heisenberg); Sec. IV.B. */
ipeps_status ipeps_ham_create(int d, const double *h_h, const double *h_v,
                              const double *h_site, double scale, ipeps_ham *out);
/* Spin-1/2 Heisenberg S.S (J); rotated != 0 applies the sublattice spin flip
 * of Sec. IV.A (second site rotated by i sigma_y), as used with a 1x1 cell. */
ipeps_status ipeps_ham_heisenberg(int rotated, double J, ipeps_ham *out);

/* Next-nearest-neighbour terms (J1-J2 model): h_d1 acts
 * on the diagonal pair (x, y)-(x+1, y+1), h_d2 on the anti-diagonal pair
 * (x+1, y)-(x, y+1) of every 2x2 plaquette, each a host (d*d) x (d*d) row-major
 * matrix in the convention of ipeps_ham_create (copied; NULL removes the
 * term).  Their expectation values come from the ring of the plaquette's four
 * enlarged corners with the pair's physical legs open, each normalised by its
 * own trace, and add to the per-site energy (times the Hamiltonian's scale).
 * For the Heisenberg J1-J2 model both are J2 S.S, unrotated also in the
 * sublattice-rotated 1x1 frame (diagonal neighbours share a sublattice).
 * Errors: IPEPS_ERR_ARG for a NULL Hamiltonian or non-finite entries. */
ipeps_status ipeps_ham_set_nnn(ipeps_ham ham, const double *h_d1, const double *h_d2);
/* Spin-1/2 J1-J2 Heisenberg model: J1 S.S on nearest-neighbour bonds
 * (sublattice-rotated as ipeps_ham_heisenberg when rotated != 0) and J2 S.S
 * on both diagonals of every plaquette (ipeps_ham_set_nnn; unrotated, as
 * diagonal neighbours share a sublattice).  Errors: IPEPS_ERR_ARG for a NULL
 * out or non-finite couplings. */
ipeps_status ipeps_ham_j1j2(int rotated, double J1, double J2, ipeps_ham *out);
/* Spin-1/2 Kitaev model K S^g S^g with two sites (a, b) merged per tensor
 * (d = 4): z link inside the tensor, x link b(x,y)-a(x+1,y), y link
 * b(x,y)-a(x,y+1); energy reported per honeycomb site (scale 1/2). */
ipeps_status ipeps_ham_kitaev(double K, ipeps_ham *out);
void ipeps_ham_destroy(ipeps_ham h);

/* --------------------------------------------------------- S1 .. S6 */
/* CTMRG environment to a fixed point (Sec. III.A).  A_dev: the unit cell
 * (layout above).  chi: environment bond dimension (>= 1).  Iterates until
 * the largest change of the normalised corner singular values is < tol, or
 * maxit iterations.  *inout_env == NULL: cold start, a new environment is
 * created and returned; otherwise it is warm started (it must have the same
 * shape and chi).  iters_out / err_out (host, may be NULL) receive the
 * iteration count and the final change.  Returns IPEPS_ERR_NOT_CONVERGED
 * (environment kept) when maxit is reached. */
ipeps_status ipeps_ctmrg(const ipeps_shape *shape, const double *A_dev, int chi, double tol,
                         int maxit, ipeps_prec prec, ipeps_env *inout_env, int *iters_out,
                         double *err_out, ipeps_stream_t stream);

/* Normalised singular values of the 4*Lx*Ly corners, chi each, written to
 * host memory (4*Lx*Ly*chi doubles, corner order C1..C4, site order x*Ly+y).
 * Gauge invariant; used to compare environments. */
ipeps_status ipeps_env_corner_spectra(ipeps_env env, double *out_host, size_t n,
                                      ipeps_stream_t stream);
void ipeps_env_destroy(ipeps_env env);

/* ------------------------------------------------------------ S7 .. S10 */
/* Energy per site, Eq. (equ:energy), from a converged environment. */
ipeps_status ipeps_energy(const ipeps_shape *shape, const double *A_dev, ipeps_env env,
                          ipeps_ham ham, double *E_out, ipeps_stream_t stream);
/* Energy and its gradient dE/dA at the CTMRG fixed point (Sec. III.A),
 * differentiated implicitly: g = dE/dA|_env + (dF/dA)^T lam with
 * (I - (dF/denv)^T) lam = dE/denv, F one gauge-fixed CTMRG iteration.
 * env must be converged for A_dev.  grad_dev: caller-allocated device
 * buffer with the layout of A.  E_out: host. */
ipeps_status ipeps_energy_grad(const ipeps_shape *shape, const double *A_dev, ipeps_env env,
                               ipeps_ham ham, double *E_out, double *grad_dev,
                               ipeps_stream_t stream);

/* ------------------------------------------------------------ S11, S12 */
/* Preconditioned gradient P^-1 g for every tensor of the cell:
 * P = 1_d (x) M + delta I with M the tensor's single-site environment
 * (Eq. equ:local_metric; Sec. IV.B: one M per tensor), symmetrised and
 * scaled so that <A|1 (x) M|A> = 1; solved by GMRES with Krylov dimension
 * `krylov` and `restarts` outer iterations, x0 = 0 (Sec. III.C uses 30 and
 * 1).  g_dev, out_dev: device, layout of A (out_dev may alias nothing).
 * delta < 0 selects the |g|^2 rule of Sec. III.B: delta = max(|g|^2, 1e-12)
 * with |g| the Euclidean norm of g over the whole cell.
 * resid_out (host, may be NULL): the largest relative residual. */
ipeps_status ipeps_precondition(const ipeps_shape *shape, const double *A_dev, ipeps_env env,
                                const double *g_dev, double delta, int krylov, int restarts,
                                double *out_dev, double *resid_out, ipeps_stream_t stream);

/* Mean-field preconditioned gradient (Sec. III.B: the local metric with the
 * environment's bond dimension set to 1, the environment belief propagation
 * gives; App. A).  Messages: one real D x D matrix m[ket, bra] per bond and
 * direction; site s sends through leg lam the contraction of A_s and A_s
 * (physical legs joined) with the messages arriving on its other three legs,
 * symmetrised and divided by its trace; sweeps update all messages from the
 * previous sweep's, from identity / D, until no entry changes by more than
 * bp_tol or bp_maxit sweeps ran.  The message arriving on leg u of site (x, y)
 * is the one (x, y-1) sends down (y grows downwards), l: (x-1, y) sends
 * right, d: (x, y+1) sends up, r: (x+1, y) sends left.  The metric of a site is
 * N = 1_d (x) c m_u (x) m_l (x) m_d (x) m_r, c such that <A|N|A> = 1, and
 * out = (N + delta I)^-1 g is applied exactly in the eigenbases of the four
 * messages.  No environment is needed.  A_dev, g_dev, out_dev: device, layout
 * of A (out_dev aliases neither); delta < 0 selects delta = max(|g|^2, 1e-12)
 * as in ipeps_precondition.  D <= 32.  sweeps_out / change_out (host, may be
 * NULL): sweeps run and the last largest change; reaching bp_maxit is not an
 * error (the last messages are used).  IPEPS_ERR_NONFINITE if a message
 * loses its positive trace. */
ipeps_status ipeps_precondition_bp(const ipeps_shape *shape, const double *A_dev, const double *g_dev,
                                   double delta, double bp_tol, int bp_maxit, double *out_dev, int *sweeps_out,
                                   double *change_out, ipeps_stream_t stream);

/* ----------------------------------------------------------------- S13 */
typedef struct {
  int chi;              /* environment bond dimension */
  double ctm_tol;       /* CTMRG corner-spectrum tolerance */
  int ctm_maxit;        /* CTMRG iteration limit per evaluation */
  ipeps_prec prec;      /* contraction arithmetic */
  int precondition;     /* 0: plain L-BFGS, 1: local-metric preconditioned,
                           2: mean-field (chi = 1) metric, ipeps_precondition_bp
                              with bp_tol 1e-12, bp_maxit 1000 (D <= 32) */
  int krylov, restarts; /* GMRES (30, 1 in Sec. III.C) */
  int delta_rule;       /* 0: delta = |g|^2, 1: delta = |E_k - E_{k-1}| (Sec. III.B) */
  int history;          /* L-BFGS history m (200 in Sec. IV.A) */
  int maxiter;          /* optimisation iterations */
  double gtol;          /* stop when |g| < gtol */
  double E_target;      /* stop when E <= E_target (use -1e300 to disable) */
} ipeps_opts;

typedef struct {
  int iter;        /* 0 for the starting point */
  double E;        /* energy per site */
  double gnorm;    /* |g| */
  double alpha;    /* accepted step (0 for iter 0) */
  double delta;    /* regularisation used for the step */
  int evals;       /* energy/gradient evaluations of this iteration */
  int ctm_iters;   /* CTMRG iterations of the accepted point */
  double wall_ms;  /* wall time of the iteration */
} ipeps_iter_info;

/* Return nonzero from the callback to stop (status IPEPS_ERR_CANCELLED). */
typedef int (*ipeps_iter_cb)(const ipeps_iter_info *info, void *user);

void ipeps_opts_default(ipeps_opts *opts);
/* Minimise E(A) (Sec. II, Sec. IV.A).  A_dev: in the starting cell, out the
 * final cell.  cb may be NULL. */
ipeps_status ipeps_optimize(const ipeps_shape *shape, double *A_dev, ipeps_ham ham,
                            const ipeps_opts *opts, ipeps_iter_cb cb, void *user,
                            ipeps_stream_t stream);

/* ------------------------------------------------------------ serving */
/* Many independent optimisations on one GPU (no counterpart in the paper,
 * which runs one optimisation at a time, Sec. IV).  A server owns `slots`
 * worker threads; each takes the admitted job whose last L-BFGS iteration is
 * oldest and runs its next iteration (ipeps_optimize's iteration) on the job's
 * own CUDA stream, so iterations of different jobs overlap on the device and
 * jobs that arrive while others run start as soon as a slot and memory are
 * free.  Each job's tensors, environment, L-BFGS history and tapes stay on the
 * device from admission to its end.  Admission by device memory: a queued job
 * is admitted (oldest first) when the sum of ipeps_job_footprint over admitted
 * jobs stays within hbm_budget_bytes (a job larger than the budget runs alone).
 * With autotune != 0 the first job of every (d, D, chi, cell, precision) class
 * times one CTMRG iteration at three settings of the tensor-core crossover
 * (the GEMM size above which the BF16-digit kernel is used) and the class
 * keeps the fastest.  A job's result is independent of the other jobs: every
 * kernel is deterministic and each job has private buffers.  The device is
 * the one current at ipeps_server_create.  All calls are thread safe;
 * messages of failed calls come from ipeps_server_last_error(). */
typedef struct {
  int slots;               /* worker threads (1 .. 64), default 3 */
  size_t hbm_budget_bytes; /* 0: 80% of the free device memory at creation */
  int autotune;            /* per-class tensor-core crossover, default 1 */
} ipeps_server_opts;

typedef struct ipeps_server_s *ipeps_server;

typedef struct {
  ipeps_shape shape;    /* unit cell */
  const double *A_host; /* starting tensors, host, layout above (copied) */
  ipeps_ham ham;        /* Hamiltonian (copied; may be destroyed after submit) */
  ipeps_opts opts;      /* as for ipeps_optimize */
} ipeps_job_desc;

typedef enum {
  IPEPS_JOB_QUEUED = 0,
  IPEPS_JOB_RUNNING = 1,
  IPEPS_JOB_DONE = 2,      /* maxiter, gtol or E_target reached */
  IPEPS_JOB_FAILED = 3,    /* see ipeps_job_result.error */
  IPEPS_JOB_CANCELLED = 4
} ipeps_job_state;

typedef struct {
  int state;              /* ipeps_job_state */
  int iterations;         /* L-BFGS iterations completed */
  double E, gnorm;        /* energy per site and |g| of the current point */
  double queued_ms;       /* submit to admission */
  double run_ms;          /* admission to end (so far, while running) */
  double iter_ms_p50, iter_ms_p99; /* wall time per iteration of this job */
  size_t footprint_bytes; /* admission estimate */
  int error;              /* ipeps_status of a failed job */
} ipeps_job_result;

typedef struct {
  int jobs_done, jobs_running, jobs_queued;
  int64_t iterations;            /* iterations of ended jobs */
  double iter_ms_p50, iter_ms_p99;
  size_t hbm_in_use_bytes, hbm_budget_bytes;
} ipeps_server_stats;

void ipeps_server_opts_default(ipeps_server_opts *opts);
/* Estimated device bytes of one job (environment, recorded tapes with their
 * cotangents, line-search copies); 0 for an invalid shape. */
size_t ipeps_job_footprint(const ipeps_shape *shape, int chi);
ipeps_status ipeps_server_create(const ipeps_server_opts *opts, ipeps_server *out);
/* Queue a job; *job_id identifies it.  Errors: IPEPS_ERR_ARG (shape, options,
 * non-finite A, Hamiltonian of another d). */
ipeps_status ipeps_server_submit(ipeps_server srv, const ipeps_job_desc *desc, uint64_t *job_id);
/* Non-blocking snapshot of a job. */
ipeps_status ipeps_server_poll(ipeps_server srv, uint64_t job_id, ipeps_job_result *res);
/* Block until the job has ended; IPEPS_ERR_TIMEOUT after timeout_s seconds. */
ipeps_status ipeps_server_wait(ipeps_server srv, uint64_t job_id, double timeout_s);
/* Stop a job: a queued job at once, a running one after its current iteration. */
ipeps_status ipeps_server_cancel(ipeps_server srv, uint64_t job_id);
/* Final tensors of an ended job (host, n >= Lx Ly d D^4 doubles). */
ipeps_status ipeps_server_tensor(ipeps_server srv, uint64_t job_id, double *A_host, size_t n);
ipeps_status ipeps_server_get_stats(ipeps_server srv, ipeps_server_stats *stats);
const char *ipeps_server_last_error(void);
/* Waits for the iterations in flight, frees every job and joins the workers. */
void ipeps_server_destroy(ipeps_server srv);

/* ------------------------------------------------------------- GEMM */
/* The contraction engine's GEMM (row-major): C = alpha op(A) op(B) + beta C,
 * op(A) M x K (ta != 0: A stored K x M), op(B) K x N (tb != 0: B stored
 * N x K), device pointers, leading dimensions in elements.  prec selects the
 * FP64 CUDA-core kernels, the 3xTF32 tcgen05 kernel (FP32 accumulate;
 * IPEPS_TF32X3 and IPEPS_TF32X3_ALL alike) or the BF16-digit tcgen05 kernel
 * (IPEPS_FP64_TC: 8 digits, IPEPS_BF16X3: 2 digits).
 * Every contraction of the hot path lowers to this call (after at most one
 * permutation per operand). */
ipeps_status ipeps_gemm(ipeps_prec prec, int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                        const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                        double *C, int64_t ldc, ipeps_stream_t stream);

/* Allocation-free variant of the FP64 path of ipeps_gemm (no counterpart in
 * the paper; an interface addition).  Some callers cannot let a library
 * allocate device memory: a host program whose device memory is already
 * reserved by another allocator (a new allocation could fail mid-run), or a
 * loop that must not take the device-wide synchronisation a cudaFree implies.
 * This call allocates nothing: it splits K over the SMs and keeps the partial
 * sums in a file-scope device array of 4 Mi doubles (32 MiB) that every GPU
 * loading the library holds until exit.  The caller passes A, B and C only.
 * Requires M * N <= 4194304 (returns IPEPS_ERR_ARG with a message
 * otherwise).  The first call on a device looks up that array's device
 * address with that device current and keeps it for the life of the
 * process (not valid across a cudaDeviceReset); make that first call before
 * any stream capture.  Later calls reuse the address.  The array keeps the last call's partial
 * sums, each call writes every slice it reads, and calls that overlap on the
 * GPU (other streams or threads) share the array and race: serialise them.
 * Arguments and result as ipeps_gemm with prec = IPEPS_FP64.  Synchronises
 * the stream before returning. */
ipeps_status ipeps_gemm_noalloc(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                                const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                                double *C, int64_t ldc, ipeps_stream_t stream);

/* ------------------------------------------------------------- misc */
const char *ipeps_last_error(void);
/* Kernel launches issued by this thread since the last reset (for reports). */
uint64_t ipeps_launch_count(int reset);
/* Host waits on a stream (synchronisations) issued by this thread since the
 * last reset (for reports). */
uint64_t ipeps_sync_count(int reset);
/* Live kernel timing: enable != 0 clears the statistics and records a CUDA
 * event pair around every instrumented launch on its stream; 0 stops.
 * ipeps_profile_query fills the launch count, summed duration (ms) and the
 * algorithmic FLOPs and bytes of one kernel class ("dgemm", "tc_gemm",
 * "jacobi_pair", "permute"); returns 0 if that class never ran.
 * ipeps_profile_names lists the classes seen (comma separated). */
void ipeps_profile(int enable);
int ipeps_profile_query(const char *name, uint64_t *count, double *ms, double *flops, double *bytes);
const char *ipeps_profile_names(void);

#ifdef __cplusplus
}
#endif
#endif /* IPEPS_H */
