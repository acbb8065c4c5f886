"""iPEPS energy minimisation with plain, local-metric or mean-field (chi = 1)
preconditioned L-BFGS (oracle, test infrastructure).

Sec. IV.A: the objective is E(A) of Sec. III.A with its gradient; the
preconditioner is the local metric of Eq. (equ:local_metric), regularised by
delta I (Sec. III.B) and inverted by GMRES with Krylov dimension 30 and one
outer iteration (Sec. III.C), tensor by tensor for a unit cell (Sec. IV.B).
Reading: every energy evaluation warm-starts CTMRG from the environment of
the point the line search started from.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ctmrg as C
from .gradient import energy_and_gradient
from .lbfgs import lbfgs
from .bp import bp_precondition
from .metric import local_metric, precondition


def _pack(cell):
    return np.concatenate([a.ravel() for col in cell for a in col])


def _unpack(x, Lx, Ly, shape):
    n = int(np.prod(shape))
    return [[x[(i * Ly + j) * n:(i * Ly + j + 1) * n].reshape(shape) for j in range(Ly)] for i in range(Lx)]


def optimize(cell, ham, chi, *, precond=True, maxiter=10, tol=1e-12, krylov=30, restarts=1,
             m=200, callback=None, stop=None, ctm_maxit=300, bp_tol=1e-12, bp_maxit=1000):
    """precond: False (plain L-BFGS), True or "local" (local metric), "bp"
    (the chi = 1 mean-field metric of Sec. III.B, oracle/bp.py)."""
    Lx, Ly = len(cell), len(cell[0])
    shape = cell[0][0].shape

    def fg(x, st):
        c = _unpack(x, Lx, Ly, shape)
        env0 = None if st is None else st["env"]
        E, g, info = energy_and_gradient(c, ham, chi, tol=tol, env=env0, maxit=ctm_maxit,
                                         return_info=True)
        if not info["converged"]:
            return np.inf, None, st
        return E, _pack(g), {"env": info["env"], "cell": c}

    def pc_bp(st, v, delta):
        vv = _unpack(v, Lx, Ly, shape)
        out, _, _ = bp_precondition(st["cell"], vv, delta, tol=bp_tol, maxit=bp_maxit)
        return np.concatenate([out[x][y].ravel() for x in range(Lx) for y in range(Ly)])

    def pc(st, v, delta):
        c, env = st["cell"], st["env"]
        A = C.as_torch_cell(c)
        vv = _unpack(v, Lx, Ly, shape)
        out = []
        for x in range(Lx):
            for y in range(Ly):
                M = local_metric(env, A[x][y], x, y).numpy()
                px, _ = precondition(M, vv[x][y], delta, krylov=krylov, restarts=restarts)
                out.append(px.ravel())
        return np.concatenate(out)

    pcf = pc_bp if precond == "bp" else (pc if precond else None)
    x, f, g, log = lbfgs(fg, _pack(cell), precond=pcf, m=m, maxiter=maxiter,
                         callback=callback, stop=stop)
    return _unpack(x, Lx, Ly, shape), f, log
