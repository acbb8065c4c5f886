"""Local-metric preconditioner (oracle, test infrastructure).

Eq. (equ:local_metric), Sec. III.A: the local metric keeps only the first
term of the tangent-space metric, the one where both vacancies sit on the
same site.  That term is the single-site environment of the tensor, so
N_local = 1_d (x) M with M[(u l d r), (u' l' d' r')] the ring of the eight
environment tensors of the site with A and conj(A) removed (physical legs of
ket and bra joined by the identity).  The diagram is lost; this reading
follows from the statement that it is available once the norm is computed.

Readings (paper silent): M is symmetrised, (M + M^T) / 2, and scaled so that
<A| 1 (x) M |A> = 1, i.e. relative to the norm per site.  Sec. IV.B: for a
unit cell every tensor gets its own M from its own environment.
Sec. III.B: P = N_local + delta I.  Sec. III.C: P g' = g by GMRES, one outer
iteration with Krylov dimension 30.

Parity pins: symmetry before symmetrising, positive semi-definiteness,
<A|1 (x) M|A> equal to the norm network, D=1 closed form, GMRES against
a direct solve (tests/test_oracle_precond.py).
"""
from __future__ import annotations

import numpy as np
import torch

from .gmres import gmres


def hole_env(env, x, y):
    """Unnormalised M[(u l d r), (u' l' d' r')] of site (x, y)."""
    C1, T1, C2, T2 = env["C1"][x][y], env["T1"][x][y], env["C2"][x][y], env["T2"][x][y]
    C3, T3, C4, T4 = env["C3"][x][y], env["T3"][x][y], env["C4"][x][y], env["T4"][x][y]
    top = torch.einsum("ab,buvc,ce->auve", C1, T1, C2)          # [C1.p, u, u', C2.n]
    bot = torch.einsum("fg,gdwh,hi->fdwi", C3, T3, C4)          # [C3.p, d, d', C4.n]
    X = torch.einsum("auve,erzf->auvrzf", top, T2)             # [C1.p, u, u', r, r', C3.p]
    X = torch.einsum("auvrzf,fdwi->auvrzdwi", X, bot)          # [..., d, d', C4.n]
    X = torch.einsum("auvrzdwi,ilma->ulrdvmzw", X, T4)          # ket (u l r d), bra (u' l' r' d')
    D = T1.shape[1]
    # reorder to ket (u l d r), bra (u' l' d' r')
    X = X.permute(0, 1, 3, 2, 4, 5, 7, 6)
    return X.reshape(D ** 4, D ** 4)


def norm_network(env, A, x, y):
    """<psi|psi> per site from the 3x3 patch of site (x, y)."""
    M = hole_env(env, x, y)
    a = A.reshape(A.shape[0], -1)
    return torch.einsum("si,ij,sj->", a, M, a)


def local_metric(env, A, x, y):
    """Symmetrised M of site (x, y), scaled so that <A|1 (x) M|A> = 1."""
    M = hole_env(env, x, y)
    M = 0.5 * (M + M.T)
    a = A.reshape(A.shape[0], -1)
    nrm = torch.einsum("si,ij,sj->", a, M, a)
    return M / nrm


def precondition(M, g, delta, krylov=30, restarts=1, rtol=1e-14):
    """Solve (1_d (x) M + delta I) x = g for one tensor by GMRES.
    g has shape (d, D, D, D, D).  Returns (x, relative residual)."""
    M = np.asarray(M)
    shape = g.shape
    d = shape[0]

    def mv(v):
        v = v.reshape(d, -1)
        return (v @ M.T + delta * v).ravel()

    x, rel, _ = gmres(mv, np.asarray(g).ravel(), krylov=krylov, restarts=restarts, rtol=rtol)
    return x.reshape(shape), rel
