"""C4v-symmetric one-tensor iPEPS: symmetric CTMRG with a fixed number of
steps and the energy gradient by differentiating the last steps (oracle, test
infrastructure: only tests/, the smoke check and the benchmark's CPU baseline
use it).

Sec. IV.A: the Heisenberg benchmarks use a real C4v-symmetric iPEPS with a
single tensor (the spin on every second site is flipped, so the rotated bond
operator of oracle/models.py applies), environments from a CTMRG with a fixed
(n + N) = (3 + 20) steps, and the gradient by automatic differentiation
through the last N steps; imposing C4v on real tensors fixes the local gauge.

Readings (the paper cites its QR-CTMRG variant without giving it):

* C4v projection: A = the mean of B over the eight symmetries of the square
  acting on the virtual legs (u, l, d, r); it is an orthogonal projection, so
  the gradient with respect to the free parameters B is the projection of the
  gradient with respect to A.
* Symmetric CTMRG (one corner C[chi, chi], symmetric; one edge
  T[chi, D, D, chi], symmetric in its two chi legs): the enlarged corner
  M[(c4, d, d'), (c3, r, r')] = C T T a is a symmetric (chi D^2)-square
  matrix; its chi eigenvalues of largest magnitude and their eigenvectors P
  give C <- P^T M P (= the kept eigenvalues) and the edge that absorbed one
  column of double-layer tensors, T <- P^T (T a) P; both are divided by their
  largest magnitude.  The projectors come from the eigendecomposition where
  the cited variant uses QR decompositions; both aim at the same fixed point.
* Initial environment: the double-layer tensor with its outward legs traced
  ket against bra (bond D^2), grown by the steps up to chi.
* Energy: the environment is written as the general one-site environment
  (all corners C, all edges T) and passed to oracle/energy.py.
* Gradient: n steps without derivatives, then N steps and the energy with
  torch autograd (torch.linalg.eigh's derivative; degenerate kept spectra
  have none, so the pins use random tensors).

Parity pins (tests/test_oracle_c4v.py): the Ising PEPS gives Onsager's
nearest-neighbour correlator; a D=1 product state gives the closed form; a
C4v-symmetric random tensor gives the energy of the general CTMRG; the
unrolled gradient equals central differences of the same unrolled energy and
approaches the projected fixed-point gradient of the general CTMRG as N grows;
the projection is idempotent and its image invariant under the eight
symmetries.
"""
from __future__ import annotations

import numpy as np
import torch

from .ctmrg import DT
from .energy import energy as general_energy
from .bp import bp_precondition
from .lbfgs import lbfgs
from .metric import local_metric, precondition

# the eight symmetries of the square as permutations of the virtual legs
# (u, l, d, r) = axes (1, 2, 3, 4) of A[s, u, l, d, r]: the four rotations
# and the four reflections
_ROT = (0, 4, 1, 2, 3)            # A'[s, u, l, d, r] = A[s, r, u, l, d]
_REF = (0, 1, 4, 3, 2)            # swap l and r (reflection through the vertical axis)


def _compose(p, q):
    return tuple(p[i] for i in q)


def symmetries():
    """The eight axis permutations of C4v acting on A[s, u, l, d, r]."""
    out, g = [], (0, 1, 2, 3, 4)
    for _ in range(4):
        out.append(g)
        out.append(_compose(g, _REF))
        g = _compose(g, _ROT)
    return out


def c4v_project(B):
    """The C4v-symmetric part of B (torch or numpy, shape [d, D, D, D, D])."""
    t = torch.as_tensor(B, dtype=DT)
    return sum(t.permute(*p) for p in symmetries()) / 8.0


def double_layer(A):
    """a[(u u'), (l l'), (d d'), (r r')] of the real tensor A."""
    D = A.shape[1]
    a = torch.einsum("sulcr,sULCR->uUlLcCrR", A, A)
    return a.reshape(D * D, D * D, D * D, D * D)


def init_env(A):
    """C[(d d'), (r r')] and T[(u u'), (r r'), (d d')] traced from the double layer."""
    D = A.shape[1]
    a = torch.einsum("sulcr,sULCR->uUlLcCrR", A, A)
    # corner: the up and left legs traced (ket = bra), the down and right legs kept
    C = torch.einsum("uullcCrR->cCrR", a).reshape(D * D, D * D)
    # edge on the left boundary: the left leg traced; (up, right, down) kept
    T = torch.einsum("uUllcCrR->uUrRcC", a).reshape(D * D, D * D, D * D)
    C = 0.5 * (C + C.T)
    T = 0.5 * (T + T.permute(2, 1, 0))
    return C / C.abs().max(), T / T.abs().max()


def enlarged_corner(C, T, a):
    """M[(c4, n), (c3, e)] = C T T a for the upper-left quadrant: C joins the
    left edge (leg c1 -> its end c4 below) and the top edge (-> c3 on the
    right); n is a's down leg and e its right leg."""
    chi, D2 = C.shape[0], a.shape[0]
    top = torch.einsum("xy,ywz->xwz", C, T)            # [c1, w (into a's up), c3]
    X = torch.einsum("xwz,xvq->wzvq", top, T)          # T (left edge) [c1, v (into a's left), c4]
    M = torch.einsum("wzvq,wvne->qnze", X, a)           # [c4, n, c3, e]
    return M.reshape(chi * D2, chi * D2)


def ctmrg_step(C, T, a, chi):
    """One symmetric CTMRG step: truncate the enlarged corner to its chi
    eigenpairs of largest magnitude, renormalise corner and edge."""
    D2 = a.shape[0]
    M = enlarged_corner(C, T, a)
    M = 0.5 * (M + M.T)
    lam, U = torch.linalg.eigh(M)
    k = min(chi, M.shape[0])
    idx = torch.argsort(lam.abs(), descending=True)[:k]
    lam, P = lam[idx], U[:, idx]
    Cn = torch.diag(lam)
    P3 = P.reshape(T.shape[0], D2, k)                  # [(c, a-leg), new]
    # the left edge absorbs one column: T[c1, v, c2] a[u, v, n, e] with (c1, u) and (c2, n) projected
    X = torch.einsum("xvy,uvne->xuyne", T, a)          # [c1, u, c2, n, e]
    Tn = torch.einsum("xuyne,xup,ynq->peq", X, P3, P3)  # [new1, e, new2]
    Tn = 0.5 * (Tn + Tn.permute(2, 1, 0))
    return Cn / Cn.abs().max(), Tn / Tn.abs().max()


def as_general_env(C, T, D):
    """The one-site environment dict of oracle/ctmrg.py with every corner C and
    every edge T[c, (ket, bra), c'] split into [c, ket, bra, c']."""
    chi = C.shape[0]
    T4 = T.reshape(chi, D, D, chi)
    names = ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4")
    return {n: [[C if n[0] == "C" else T4]] for n in names}


def ctmrg(A, chi, steps, env=None):
    """`steps` symmetric CTMRG steps from env (or the traced start).  Returns (C, T)."""
    a = double_layer(A)
    C, T = init_env(A) if env is None else env
    for _ in range(steps):
        C, T = ctmrg_step(C, T, a, chi)
    return C, T


def energy(A, chi, ham, n=3, N=20, env=None):
    """Energy per site after n + N steps (A: torch, C4v symmetric)."""
    C, T = ctmrg(A, chi, n + N, env)
    return general_energy(1, 1, [[A]], as_general_env(C, T, A.shape[1]), ham)


def energy_and_gradient(B, chi, ham, n=3, N=20, env=None):
    """E(c4v_project(B)) after (n + N) steps and its gradient with respect to
    B: n steps without derivatives, the last N differentiated.  Returns
    (E, g[d, D, D, D, D] numpy)."""
    Bt = torch.as_tensor(np.asarray(B), dtype=DT).clone().requires_grad_(True)
    A = c4v_project(Bt)
    with torch.no_grad():
        C, T = ctmrg(A.detach(), chi, n, env)
    a = double_layer(A)
    for _ in range(N):
        C, T = ctmrg_step(C, T, a, chi)
    E = general_energy(1, 1, [[A]], as_general_env(C, T, A.shape[1]), ham)
    E.backward()
    return float(E.detach()), Bt.grad.detach().numpy().copy()


def optimize(B0, chi, ham, *, precond=True, maxiter=100, n=3, N=20, callback=None, stop=None):
    """L-BFGS (m = 200, Hager-Zhang; oracle/lbfgs.py) on the free tensor B of
    the C4v-symmetric iPEPS A = c4v_project(B), each evaluation the (n + N)-step
    energy and its unrolled gradient from the traced start (Sec. IV.A), with
    the local-metric preconditioner (precond=True or "local": Eq.
    equ:local_metric, from the environment after the n + N steps), the
    mean-field one (precond="bp": oracle/bp.py, App. A) or none (False); the
    preconditioned vector is projected back onto the C4v subspace.
    Returns (B, E, log)."""
    shape = np.asarray(B0).shape
    D = shape[1]

    def fg(x, st):
        B = x.reshape(shape)
        E, g = energy_and_gradient(B, chi, ham, n=n, N=N)
        if not np.isfinite(E):
            return np.inf, None, st
        return E, g.ravel(), {"B": B}

    def pc(st, v, delta):
        A = c4v_project(st["B"])
        with torch.no_grad():
            C, T = ctmrg(A, chi, n + N)
            M = local_metric(as_general_env(C, T, D), A, 0, 0).numpy()
        x, _ = precondition(M, v.reshape(shape), delta)
        return c4v_project(x).numpy().ravel()

    def pc_bp(st, v, delta):
        A = c4v_project(st["B"]).numpy()
        out, _, _ = bp_precondition([[A]], [[v.reshape(shape)]], delta)
        return c4v_project(out[0][0]).numpy().ravel()

    pcf = pc_bp if precond == "bp" else (pc if precond else None)
    x, f, g, log = lbfgs(fg, np.asarray(B0, dtype=np.float64).ravel(), precond=pcf, m=200,
                         maxiter=maxiter, callback=callback, stop=stop)
    return x.reshape(shape), f, log
