"""GMRES(m) for the regularised preconditioner solve (oracle, test infrastructure).

Sec. III.C: P g' = g is solved implicitly with matrix-vector products only;
one outer iteration of GMRES with a Krylov dimension of 30 is used.  Reading
of the unstated details: x0 = 0, Arnoldi with classical Gram-Schmidt applied
twice, Givens rotations for the small least-squares problem, and an early
stop once the residual estimate falls to rtol * |b|.

Parity pins: with a Krylov dimension >= n the result equals a direct
solve (tests/test_oracle_precond.py).
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, krylov=30, restarts=1, rtol=1e-14, x0=None):
    """Returns (x, relative residual estimate, matvec count)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64).ravel()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0.0, 0
    nmv = 0
    rel = 1.0
    for _cycle in range(restarts):
        r = b - matvec(x) if np.any(x) else b.copy()
        if np.any(x):
            nmv += 1
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= rtol:
            break
        m = krylov
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(m):
            w = matvec(V[j])
            nmv += 1
            # classical Gram-Schmidt, twice
            h = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            # previous rotations on the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation annihilating H[j+1, j]
            den = np.hypot(H[j, j], H[j + 1, j])
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            j_used = j + 1
            rel = abs(gvec[j + 1]) / bnorm
            if rel <= rtol or hn == 0.0:
                break
            V[j + 1] = w / hn
        # back substitution
        k = j_used
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (gvec[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        if rel <= rtol:
            break
    return x, rel, nmv
