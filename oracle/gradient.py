"""Energy gradient at the CTMRG fixed point (oracle, test infrastructure).

Sec. III.A obtains dE/dA by backward-mode automatic differentiation through
the contraction; Sec. IV.A unrolls the last 20 of (3+20) CTMRG steps.  The
reading fixed for the build differentiates the fixed point itself: with
e* = F(e*, A), where F is one CTMRG iteration followed by the constant sign
gauge sigma that makes e* an elementwise fixed point,

    g = dE/dA|_e + (dF/dA)^T lam,     (I - (dF/de)^T) lam = dE/de|_A.

Every vector-Jacobian product comes from torch's CPU autograd of one F
application (a library primitive; torch's SVD backward is the full thin-SVD
formula, so the truncation to chi is differentiated exactly), and the linear
system is solved by the oracle's GMRES to a relative residual of 1e-13.

Parity pins: central finite differences, <g, A> = 0 (scale invariance),
g = 0 for D=1 product states, and unrolled differentiation of N iterations
converging to the fixed-point gradient as N grows (tests/test_oracle_grad.py).
"""
from __future__ import annotations

import numpy as np
import torch
from torch.func import vjp

from . import ctmrg as C
from .energy import energy
from .gmres import gmres


def _flat_env(Lx, Ly, env):
    return tuple(env[n][x][y] for n in C.NAMES for x in range(Lx) for y in range(Ly))


def _unflat_env(Lx, Ly, flat):
    env = {n: [[None] * Ly for _ in range(Lx)] for n in C.NAMES}
    k = 0
    for n in C.NAMES:
        for x in range(Lx):
            for y in range(Ly):
                env[n][x][y] = flat[k]
                k += 1
    return env


def _flat_A(Lx, Ly, A):
    return tuple(A[x][y] for x in range(Lx) for y in range(Ly))


def _unflat_A(Lx, Ly, flat):
    return [[flat[x * Ly + y] for y in range(Ly)] for x in range(Lx)]


def _vec(ts):
    return np.concatenate([t.detach().numpy().ravel() for t in ts])


def _unvec(v, like):
    out, k = [], 0
    for t in like:
        n = t.numel()
        out.append(torch.as_tensor(v[k:k + n].reshape(t.shape), dtype=C.DT))
        k += n
    return tuple(out)


def energy_and_gradient(cell, ham, chi, tol=1e-12, maxit=2000, env=None, adj_tol=1e-13,
                        adj_maxmv=600, return_info=False):
    """E and dE/dA (list of lists like cell) at the CTMRG fixed point."""
    Lx, Ly = len(cell), len(cell[0])
    env, sig, iters, err, res = C.fixed_point(cell, chi, tol=tol, maxit=maxit, env=env)
    if not err < tol:
        if return_info:
            return float("nan"), None, dict(converged=False, ctm_iters=iters, ctm_err=err, env=env)
        raise RuntimeError("CTMRG did not converge")
    A = C.as_torch_cell(cell)
    e_flat = tuple(t.detach().clone() for t in _flat_env(Lx, Ly, env))
    a_flat = tuple(t.detach().clone() for t in _flat_A(Lx, Ly, A))

    def F(e_in, a_in):
        e = _unflat_env(Lx, Ly, e_in)
        a = _unflat_A(Lx, Ly, a_in)
        e1 = C.ctmrg_step(Lx, Ly, a, e, chi)
        e1 = C.apply_fixed_gauge(Lx, Ly, e1, sig)
        return _flat_env(Lx, Ly, e1)

    def Efun(e_in, a_in):
        return energy(Lx, Ly, _unflat_A(Lx, Ly, a_in), _unflat_env(Lx, Ly, e_in), ham)

    E, vjp_E = vjp(Efun, e_flat, a_flat)
    ebar, abar_direct = vjp_E(torch.ones((), dtype=C.DT))
    _, vjp_F = vjp(F, e_flat, a_flat)

    def mv(v):
        lam = _unvec(v, e_flat)
        je, _ = vjp_F(lam)
        return v - _vec(je)

    b = _vec(ebar)
    lam, rel, nmv = gmres(mv, b, krylov=60, restarts=max(1, adj_maxmv // 60), rtol=adj_tol)
    _, abar_fp = vjp_F(_unvec(lam, e_flat))
    g = [[None] * Ly for _ in range(Lx)]
    for x in range(Lx):
        for y in range(Ly):
            k = x * Ly + y
            g[x][y] = (abar_direct[k] + abar_fp[k]).numpy()
    if return_info:
        info = dict(converged=bool(rel <= 10 * adj_tol), ctm_iters=iters, ctm_err=err, fixed_point_residual=res,
                    adjoint_residual=rel, adjoint_matvecs=nmv, env=env, sigma=sig)
        return float(E), g, info
    return float(E), g


def energy_at(cell, ham, chi, tol=1e-12, maxit=2000, env=None):
    """E at the CTMRG fixed point (no gradient)."""
    Lx, Ly = len(cell), len(cell[0])
    env, _, _ = C.ctmrg(cell, chi, tol=tol, maxit=maxit, env=env)
    with torch.no_grad():
        return float(energy(Lx, Ly, C.as_torch_cell(cell), env, ham)), env


def unrolled_gradient(cell, ham, chi, n_unroll, tol=1e-12, maxit=2000):
    """Gradient from differentiating n_unroll CTMRG iterations started at the
    converged environment (the paper's (n+N) scheme with N = n_unroll)."""
    Lx, Ly = len(cell), len(cell[0])
    env, _, _ = C.ctmrg(cell, chi, tol=tol, maxit=maxit)
    A = [[torch.as_tensor(np.asarray(a), dtype=C.DT).requires_grad_(True) for a in col] for col in cell]
    e = {n: [[env[n][x][y].detach() for y in range(Ly)] for x in range(Lx)] for n in C.NAMES}
    for _ in range(n_unroll):
        e = C.ctmrg_step(Lx, Ly, A, e, chi)
    E = energy(Lx, Ly, A, e, ham)
    E.backward()
    return float(E.detach()), [[A[x][y].grad.numpy() for y in range(Ly)] for x in range(Lx)]
