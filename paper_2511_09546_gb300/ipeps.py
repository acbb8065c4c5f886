"""Python binding of libipeps (argument marshalling only).

Every call goes to the C ABI declared in include/ipeps.h; every step of the
hot path runs in the library's CUDA kernels.  Device buffers are torch CUDA
tensors (float64, contiguous) used as plain memory; the unit cell is a tensor
of shape (Lx, Ly, d, D, D, D, D) with legs (s, u, l, d, r).  The module
raises at import of the library if libipeps.so is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libipeps.so")
_lib = None

FP64, TF32X3, TF32X3_ALL, FP64_TC, BF16X3 = 0, 1, 2, 3, 4
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_NOMEM", 3: "ERR_CUDA", 4: "ERR_NONFINITE",
          5: "ERR_NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_CANCELLED"}


class Shape(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Ly", C.c_int), ("d", C.c_int), ("D", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("chi", C.c_int), ("ctm_tol", C.c_double), ("ctm_maxit", C.c_int), ("prec", C.c_int),
                ("precondition", C.c_int), ("krylov", C.c_int), ("restarts", C.c_int),
                ("delta_rule", C.c_int), ("history", C.c_int), ("maxiter", C.c_int),
                ("gtol", C.c_double), ("E_target", C.c_double)]


class IterInfo(C.Structure):
    _fields_ = [("iter", C.c_int), ("E", C.c_double), ("gnorm", C.c_double), ("alpha", C.c_double),
                ("delta", C.c_double), ("evals", C.c_int), ("ctm_iters", C.c_int), ("wall_ms", C.c_double)]


ITER_CB = C.CFUNCTYPE(C.c_int, C.POINTER(IterInfo), C.c_void_p)


class IpepsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing; build it with __graft_entry__.build()")
        L = C.CDLL(_LIB_PATH)
        vp, i, d, dp = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)
        sp = C.POINTER(Shape)
        L.ipeps_last_error.restype = C.c_char_p
        L.ipeps_launch_count.restype = C.c_uint64
        L.ipeps_launch_count.argtypes = [i]
        L.ipeps_sync_count.restype = C.c_uint64
        L.ipeps_sync_count.argtypes = [i]
        L.ipeps_profile.argtypes = [i]
        L.ipeps_profile_query.argtypes = [C.c_char_p, C.POINTER(C.c_uint64), dp, dp, dp]
        L.ipeps_profile_query.restype = i
        L.ipeps_profile_names.restype = C.c_char_p
        L.ipeps_ham_create.argtypes = [i, dp, dp, dp, d, C.POINTER(vp)]
        L.ipeps_ham_heisenberg.argtypes = [i, d, C.POINTER(vp)]
        L.ipeps_ham_kitaev.argtypes = [d, C.POINTER(vp)]
        L.ipeps_ham_j1j2.argtypes = [i, d, d, C.POINTER(vp)]
        L.ipeps_ham_set_nnn.argtypes = [vp, dp, dp]
        L.ipeps_ham_destroy.argtypes = [vp]
        L.ipeps_ctmrg.argtypes = [sp, vp, i, d, i, i, C.POINTER(vp), C.POINTER(i), dp, vp]
        L.ipeps_env_corner_spectra.argtypes = [vp, dp, C.c_size_t, vp]
        L.ipeps_env_destroy.argtypes = [vp]
        L.ipeps_energy.argtypes = [sp, vp, vp, vp, dp, vp]
        L.ipeps_energy_grad.argtypes = [sp, vp, vp, vp, dp, vp, vp]
        L.ipeps_precondition.argtypes = [sp, vp, vp, vp, d, i, i, vp, dp, vp]
        L.ipeps_precondition_bp.argtypes = [sp, vp, vp, d, d, i, vp, C.POINTER(i), dp, vp]
        L.ipeps_opts_default.argtypes = [C.POINTER(Opts)]
        i64 = C.c_int64
        L.ipeps_gemm.argtypes = [i, i, i, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64, vp]
        L.ipeps_gemm.restype = i
        L.ipeps_gemm_noalloc.argtypes = [i, i, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64, vp]
        L.ipeps_gemm_noalloc.restype = i
        L.ipeps_optimize.argtypes = [sp, vp, vp, C.POINTER(Opts), ITER_CB, vp, vp]
        for name in ("ipeps_ham_create", "ipeps_ham_heisenberg", "ipeps_ham_kitaev", "ipeps_ham_set_nnn",
                     "ipeps_ham_j1j2", "ipeps_ctmrg",
                     "ipeps_env_corner_spectra", "ipeps_energy", "ipeps_energy_grad",
                     "ipeps_precondition", "ipeps_optimize"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def _check(st, allow=()):
    if st != 0 and st not in allow:
        raise IpepsError(st, lib().ipeps_last_error().decode())
    return st


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(x):
    """float64 contiguous CUDA tensor (copies host arrays to the device)."""
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64))
    if not x.is_cuda:
        x = x.to("cuda")
    if x.dtype != torch.float64:
        raise TypeError("float64 tensors expected")
    return x.contiguous()


def _shape(A):
    Lx, Ly, d, D = A.shape[0], A.shape[1], A.shape[2], A.shape[3]
    return Shape(Lx, Ly, d, D)


def cell_tensor(cell):
    """Stack a nested list cell[x][y] of (d, D, D, D, D) arrays into (Lx, Ly, d, D, D, D, D)."""
    return np.stack([np.stack([np.asarray(a, dtype=np.float64) for a in col]) for col in cell])


class Ham:
    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipeps_ham_destroy(self.h)
            self.h = None


def ham_create(d, h, v, site=None, scale=1.0):
    h = np.ascontiguousarray(h, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    dp = C.POINTER(C.c_double)
    sp = None if site is None else np.ascontiguousarray(site, dtype=np.float64)
    out = C.c_void_p()
    _check(lib().ipeps_ham_create(d, h.ctypes.data_as(dp), v.ctypes.data_as(dp),
                                  None if sp is None else sp.ctypes.data_as(dp), scale, C.byref(out)))
    return Ham(out)


def ham_heisenberg(rotated=True, J=1.0):
    out = C.c_void_p()
    _check(lib().ipeps_ham_heisenberg(int(rotated), J, C.byref(out)))
    return Ham(out)


def ham_set_nnn(ham, d1, d2):
    """Next-nearest-neighbour operators ((d*d) x (d*d) arrays or None) on the
    diagonal and anti-diagonal pairs of every plaquette."""
    dp = C.POINTER(C.c_double)
    a = None if d1 is None else np.ascontiguousarray(d1, dtype=np.float64)
    b = None if d2 is None else np.ascontiguousarray(d2, dtype=np.float64)
    _check(lib().ipeps_ham_set_nnn(ham.h, None if a is None else a.ctypes.data_as(dp),
                                   None if b is None else b.ctypes.data_as(dp)))
    return ham


def ham_j1j2(J1=1.0, J2=0.5, rotated=True):
    """J1-J2 Heisenberg model: J1 S.S on nearest neighbours (sublattice-rotated
    when rotated), J2 S.S on both diagonals (never rotated: same sublattice)."""
    out = C.c_void_p()
    _check(lib().ipeps_ham_j1j2(int(rotated), J1, J2, C.byref(out)))
    return Ham(out)


def ham_kitaev(K=-1.0):
    out = C.c_void_p()
    _check(lib().ipeps_ham_kitaev(K, C.byref(out)))
    return Ham(out)


class Env:
    def __init__(self, handle, shape, chi):
        self.h, self.shape, self.chi = handle, shape, chi
        self.version = 0  # advanced by every ctmrg() that updates this environment

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipeps_env_destroy(self.h)
            self.h = None

    def corner_spectra(self):
        n = 4 * self.shape.Lx * self.shape.Ly * self.chi
        out = np.zeros(n)
        _check(lib().ipeps_env_corner_spectra(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), n, _stream()))
        return out.reshape(4, self.shape.Lx * self.shape.Ly, self.chi)


def ctmrg(A, chi, tol=1e-10, maxit=500, prec=FP64, env=None, allow_unconverged=False):
    """CTMRG environment of the cell A.  Returns (env, iterations, final change)."""
    A = _dev(A)
    shape = _shape(A)
    h = C.c_void_p(env.h.value if env is not None else None)
    it = C.c_int()
    err = C.c_double()
    st = lib().ipeps_ctmrg(C.byref(shape), C.c_void_p(A.data_ptr()), chi, tol, maxit, prec, C.byref(h),
                           C.byref(it), C.byref(err), _stream())
    if env is None and h.value:
        env = Env(h, shape, chi)
    elif env is not None:
        env.version += 1
    _check(st, allow=(5,) if allow_unconverged else ())
    return env, it.value, err.value


def energy(A, env, ham):
    A = _dev(A)
    shape = _shape(A)
    E = C.c_double()
    _check(lib().ipeps_energy(C.byref(shape), C.c_void_p(A.data_ptr()), env.h, ham.h, C.byref(E), _stream()))
    return E.value


def energy_grad(A, env, ham):
    """(E, dE/dA) at the CTMRG fixed point; dE/dA has the shape of A."""
    A = _dev(A)
    shape = _shape(A)
    g = torch.empty_like(A)
    E = C.c_double()
    _check(lib().ipeps_energy_grad(C.byref(shape), C.c_void_p(A.data_ptr()), env.h, ham.h, C.byref(E),
                                   C.c_void_p(g.data_ptr()), _stream()))
    return E.value, g


def precondition(A, env, g, delta, krylov=30, restarts=1):
    """P^-1 g with P = 1 (x) M + delta I per tensor.  Returns (x, worst relative residual)."""
    A = _dev(A)
    g = _dev(g)
    shape = _shape(A)
    out = torch.empty_like(g)
    res = C.c_double()
    _check(lib().ipeps_precondition(C.byref(shape), C.c_void_p(A.data_ptr()), env.h, C.c_void_p(g.data_ptr()),
                                    delta, krylov, restarts, C.c_void_p(out.data_ptr()), C.byref(res), _stream()))
    return out, res.value


def precondition_bp(A, g, delta, tol=1e-12, maxit=1000):
    """(N + delta I)^-1 g with N the mean-field (chi = 1) metric of every tensor;
    needs no environment.  Returns (x, sweeps, last largest message change)."""
    A = _dev(A)
    g = _dev(g)
    if g.shape != A.shape:
        raise ValueError("precondition_bp: g must have the shape of A")
    shape = _shape(A)
    out = torch.empty_like(g)
    sweeps = C.c_int()
    change = C.c_double()
    _check(lib().ipeps_precondition_bp(C.byref(shape), C.c_void_p(A.data_ptr()), C.c_void_p(g.data_ptr()),
                                       delta, tol, maxit, C.c_void_p(out.data_ptr()), C.byref(sweeps),
                                       C.byref(change), _stream()))
    return out, sweeps.value, change.value


def default_opts(**kw):
    o = Opts()
    lib().ipeps_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def optimize(A, ham, opts, callback=None):
    """Run L-BFGS in place on a device copy of A.  Returns (A_final, log, status)."""
    A = _dev(A).clone()
    shape = _shape(A)
    log = []

    def _cb(info_p, _user):
        i = info_p.contents
        rec = dict(iter=i.iter, E=i.E, gnorm=i.gnorm, alpha=i.alpha, delta=i.delta, evals=i.evals,
                   ctm_iters=i.ctm_iters, wall_ms=i.wall_ms)
        log.append(rec)
        if callback is not None and callback(rec):
            return 1
        return 0

    cb = ITER_CB(_cb)
    st = lib().ipeps_optimize(C.byref(shape), C.c_void_p(A.data_ptr()), ham.h, C.byref(opts), cb, None, _stream())
    _check(st, allow=(5, 7))
    return A, log, st


def launch_count(reset=False):
    return int(lib().ipeps_launch_count(1 if reset else 0))


def sync_count(reset=False):
    """Host waits on a stream issued by this thread (since the last reset)."""
    return int(lib().ipeps_sync_count(1 if reset else 0))


def profile(enable=True):
    """Enable (and clear) or disable the library's live kernel timing."""
    lib().ipeps_profile(1 if enable else 0)


def profile_stats():
    """{kernel class: dict(count, ms, flops, bytes)} since profile(True)."""
    out = {}
    names = lib().ipeps_profile_names().decode()
    for name in [n for n in names.split(",") if n]:
        cnt = C.c_uint64()
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        if lib().ipeps_profile_query(name.encode(), C.byref(cnt), C.byref(ms), C.byref(fl), C.byref(by)):
            out[name] = dict(count=cnt.value, ms=ms.value, flops=fl.value, bytes=by.value)
    return out


def gemm(A, B, ta=False, tb=False, alpha=1.0, beta=0.0, C=None, prec=FP64):
    """C = alpha op(A) op(B) + beta C with the library's GEMM (2-D float64 CUDA tensors)."""
    A = _dev(A)
    B = _dev(B)
    M, K = (A.shape[1], A.shape[0]) if ta else (A.shape[0], A.shape[1])
    K2, N = (B.shape[1], B.shape[0]) if tb else (B.shape[0], B.shape[1])
    if K != K2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    _check_out(C, M, N, A.device)
    _check(lib().ipeps_gemm(prec, int(ta), int(tb), M, N, K, alpha, C_ptr(A), A.shape[1], C_ptr(B), B.shape[1],
                            beta, C_ptr(C), C.shape[1], _stream()))
    return C


def C_ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_out(C, M, N, device):
    """C must be a contiguous float64 CUDA tensor of shape (M, N) on `device`:
    the library writes M x N doubles at its address with row stride N."""
    if not (isinstance(C, torch.Tensor) and C.is_cuda and C.dtype == torch.float64 and C.is_contiguous()):
        raise TypeError("C must be a contiguous float64 CUDA tensor")
    if tuple(C.shape) != (M, N):
        raise ValueError(f"C has shape {tuple(C.shape)}, expected {(M, N)}")
    if C.device != device:
        raise ValueError("C is on another device than A")


def gemm_noalloc(A, B, C, ta=False, tb=False, alpha=1.0, beta=0.0):
    """C = alpha op(A) op(B) + beta C through the allocation-free FP64 entry point
    (C is written in place; the library allocates no device memory for it)."""
    A = _dev(A)
    B = _dev(B)
    if A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be matrices")
    M, K = (A.shape[1], A.shape[0]) if ta else (A.shape[0], A.shape[1])
    K2, N = (B.shape[1], B.shape[0]) if tb else (B.shape[0], B.shape[1])
    if K != K2:
        raise ValueError("inner dimensions differ")
    if B.device != A.device:
        raise ValueError("A and B are on different devices")
    _check_out(C, M, N, A.device)
    _check(lib().ipeps_gemm_noalloc(int(ta), int(tb), M, N, K, alpha, C_ptr(A), A.shape[1], C_ptr(B),
                                    B.shape[1], beta, C_ptr(C), C.shape[1], _stream()))
    return C


class EnergyFunction(torch.autograd.Function):
    """E(A) as a differentiable function: the forward runs CTMRG to its fixed
    point (warm-started from `state["env"]` when present) and the energy; the
    backward calls ipeps_energy_grad, the fixed-point gradient dE/dA of the
    library, at the forward's environment."""

    @staticmethod
    def forward(ctx, A, ham, chi, tol, maxit, prec, state):
        env, _, _ = ctmrg(A, chi, tol=tol, maxit=maxit, prec=prec, env=state.get("env"))
        state["env"] = env
        E = energy(A, env, ham)
        ctx.save_for_backward(A)
        ctx.env, ctx.version, ctx.ham = env, env.version, ham
        return torch.tensor(E, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, gE):
        (A,) = ctx.saved_tensors
        if ctx.env.version != ctx.version:
            raise RuntimeError("the environment of this energy was advanced by a later ctmrg() before backward")
        _, g = energy_grad(A.detach(), ctx.env, ctx.ham)
        return gE * g, None, None, None, None, None, None


def energy_fn(A, ham, chi, tol=1e-10, maxit=500, prec=FP64, state=None):
    """E(A) per site with autograd support (see EnergyFunction).  A: CUDA float64
    tensor (Lx, Ly, d, D, D, D, D).  state: a dict that keeps the environment
    between calls for warm starts (a fresh dict each call cold-starts)."""
    return EnergyFunction.apply(A, ham, chi, tol, maxit, prec, {} if state is None else state)


# ------------------------------------------------------------------ serving
class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("autotune", C.c_int)]


class JobDesc(C.Structure):
    _fields_ = [("shape", Shape), ("A_host", C.POINTER(C.c_double)), ("ham", C.c_void_p), ("opts", Opts)]


class JobResult(C.Structure):
    _fields_ = [("state", C.c_int), ("iterations", C.c_int), ("E", C.c_double), ("gnorm", C.c_double),
                ("queued_ms", C.c_double), ("run_ms", C.c_double), ("iter_ms_p50", C.c_double),
                ("iter_ms_p99", C.c_double), ("footprint_bytes", C.c_size_t), ("error", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("jobs_done", C.c_int), ("jobs_running", C.c_int), ("jobs_queued", C.c_int),
                ("iterations", C.c_int64), ("iter_ms_p50", C.c_double), ("iter_ms_p99", C.c_double),
                ("hbm_in_use_bytes", C.c_size_t), ("hbm_budget_bytes", C.c_size_t)]


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


def _server_lib():
    L = lib()
    if not getattr(L, "_server_ready", False):
        vp, u64 = C.c_void_p, C.c_uint64
        L.ipeps_server_opts_default.argtypes = [C.POINTER(ServerOpts)]
        L.ipeps_job_footprint.argtypes = [C.POINTER(Shape), C.c_int]
        L.ipeps_job_footprint.restype = C.c_size_t
        L.ipeps_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(vp)]
        L.ipeps_server_submit.argtypes = [vp, C.POINTER(JobDesc), C.POINTER(u64)]
        L.ipeps_server_poll.argtypes = [vp, u64, C.POINTER(JobResult)]
        L.ipeps_server_wait.argtypes = [vp, u64, C.c_double]
        L.ipeps_server_cancel.argtypes = [vp, u64]
        L.ipeps_server_tensor.argtypes = [vp, u64, C.POINTER(C.c_double), C.c_size_t]
        L.ipeps_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.ipeps_server_destroy.argtypes = [vp]
        L.ipeps_server_last_error.restype = C.c_char_p
        for name in ("ipeps_server_create", "ipeps_server_submit", "ipeps_server_poll", "ipeps_server_wait",
                     "ipeps_server_cancel", "ipeps_server_tensor", "ipeps_server_get_stats"):
            getattr(L, name).restype = C.c_int
        L._server_ready = True
    return L


def _scheck(st):
    if st != 0:
        raise IpepsError(st, _server_lib().ipeps_server_last_error().decode())
    return st


def job_footprint(Lx, Ly, d, D, chi):
    """Device bytes the server budgets for one job of this shape."""
    sh = Shape(Lx, Ly, d, D)
    return int(_server_lib().ipeps_job_footprint(C.byref(sh), chi))


class Server:
    """Many optimisation jobs on the current GPU (see ipeps_server_* in include/ipeps.h)."""

    def __init__(self, slots=3, hbm_budget_bytes=0, autotune=True):
        L = _server_lib()
        o = ServerOpts()
        L.ipeps_server_opts_default(C.byref(o))
        o.slots, o.hbm_budget_bytes, o.autotune = slots, int(hbm_budget_bytes), int(bool(autotune))
        self.h = C.c_void_p()
        _scheck(L.ipeps_server_create(C.byref(o), C.byref(self.h)))
        self.shapes = {}

    def submit(self, A, ham, opts):
        """A: host array (Lx, Ly, d, D, D, D, D); ham: Ham; opts: Opts.  Returns a job id."""
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        desc = JobDesc(_shape(A), A.ctypes.data_as(C.POINTER(C.c_double)), ham.h, opts)
        jid = C.c_uint64()
        _scheck(_server_lib().ipeps_server_submit(self.h, C.byref(desc), C.byref(jid)))
        self.shapes[jid.value] = A.shape
        return jid.value

    def poll(self, job):
        r = JobResult()
        _scheck(_server_lib().ipeps_server_poll(self.h, job, C.byref(r)))
        return dict(state=JOB_STATES[r.state], iterations=r.iterations, E=r.E, gnorm=r.gnorm,
                    queued_ms=r.queued_ms, run_ms=r.run_ms, iter_ms_p50=r.iter_ms_p50,
                    iter_ms_p99=r.iter_ms_p99, footprint_bytes=r.footprint_bytes, error=r.error)

    def wait(self, job, timeout=3600.0):
        _scheck(_server_lib().ipeps_server_wait(self.h, job, float(timeout)))
        return self.poll(job)

    def cancel(self, job):
        _scheck(_server_lib().ipeps_server_cancel(self.h, job))

    def tensor(self, job):
        out = np.zeros(self.shapes[job])
        _scheck(_server_lib().ipeps_server_tensor(self.h, job, out.ctypes.data_as(C.POINTER(C.c_double)),
                                                  out.size))
        return out

    def stats(self):
        s = ServerStats()
        _scheck(_server_lib().ipeps_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _server_lib().ipeps_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        if _lib is not None:
            self.close()
