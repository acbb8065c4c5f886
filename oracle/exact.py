"""Brute-force and closed-form references that pin the oracle (test infrastructure).

* Onsager's free energy and nearest-neighbour correlation of the 2D Ising model, reached by
  the 'Ising PEPS' A[s,u,l,d,r] = Q[s,u] Q[s,l] Q[s,d] Q[s,r] with
  Q Q^T = [[e^{K/2}, e^{-K/2}], [e^{-K/2}, e^{K/2}]], whose norm network is
  the Ising partition function at coupling K.
* The infinite cylinder of circumference W: the exact dominant eigenvectors of
  the double-layer column transfer matrix (dimension D^(2W)) give the
  bond density matrices; they approach the 2D (CTMRG) values as W grows.
* Exact expectation values on small periodic tori by full contraction.

None of these share code with the CTMRG oracle: they contract the
network in a different order, from scratch.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ellipk


def ising_peps(K: float) -> np.ndarray:
    W = np.array([[np.exp(K / 2), np.exp(-K / 2)], [np.exp(-K / 2), np.exp(K / 2)]])
    w, v = np.linalg.eigh(W)
    Q = v @ np.diag(np.sqrt(w)) @ v.T
    return np.einsum("su,sl,sd,sr->suldr", Q, Q, Q, Q)


def onsager_nn(K: float) -> float:
    """<sigma_i sigma_j> for nearest neighbours of the square-lattice Ising
    model (Onsager), with the modulus k = 2 sinh 2K / cosh^2 2K and the
    complete elliptic integral K(k) (scipy takes the parameter m = k^2)."""
    k = 2.0 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    return 0.5 / np.tanh(2 * K) * (1.0 + (2.0 / np.pi) * (2.0 * np.tanh(2 * K) ** 2 - 1.0) * ellipk(k * k))


def onsager_log_z(K: float) -> float:
    """ln Z / N of the square-lattice Ising model at coupling K (Onsager), as
    the double integral ln 2 + 1/(8 pi^2) int int ln[cosh^2 2K - sinh 2K (cos a + cos b)]."""
    from scipy.integrate import dblquad
    c2, s2 = np.cosh(2 * K) ** 2, np.sinh(2 * K)
    val, _ = dblquad(lambda a, b: np.log(c2 - s2 * (np.cos(a) + np.cos(b))), 0, 2 * np.pi, 0, 2 * np.pi,
                     epsabs=1e-13, epsrel=1e-13)
    return float(np.log(2.0) + val / (8 * np.pi ** 2))


def onsager_log_z_1d(K: float) -> float:
    """The same in Onsager's one-dimensional form:
    ln(2 cosh 2K) + (1/pi) int_0^{pi/2} ln[(1 + sqrt(1 - k^2 sin^2 t)) / 2] dt, k = 2 sinh 2K / cosh^2 2K."""
    from scipy.integrate import quad
    k = 2.0 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    val, _ = quad(lambda t: np.log((1.0 + np.sqrt(1.0 - (k * np.sin(t)) ** 2)) / 2.0), 0, np.pi / 2,
                  epsabs=1e-14, epsrel=1e-14)
    return float(np.log(2 * np.cosh(2 * K)) + val / np.pi)


def _site(A, kb=None):
    """Double-layer site tensor a[(u u'), (l l'), (d d'), (r r')]; with kb = (k, b)
    the physical legs are fixed to ket k and bra b instead of summed."""
    D = A.shape[1]
    if kb is None:
        a = np.einsum("suldr,svmek->uvlmderk", A, A)
    else:
        k, b = kb
        a = np.einsum("uldr,vmek->uvlmderk", A[k], A[b])
    return a.reshape(D * D, D * D, D * D, D * D)


def _column(sites):
    """Column transfer matrix T[(l_1..l_W), (r_1..r_W)] of a periodic column
    of double-layer tensors sites[i][u, l, d, r] (row i's d joins row i+1's u)."""
    W = len(sites)
    X = sites[0]                                    # [u1, l1, d1, r1]
    X = X.reshape(X.shape[0], X.shape[1], X.shape[2], X.shape[3])
    # X[u1, L, u_next, R] with L, R flattened
    X = X.transpose(0, 1, 3, 2)                    # [u1, l1, r1, d1]
    for i in range(1, W):
        a = sites[i]                                # [u, l, d, r]
        X = np.einsum("aLRu,ulds->aLlRsd", X, a)
        s = X.shape
        X = X.reshape(s[0], s[1] * s[2], s[3] * s[4], s[5])
    T = np.einsum("aLRa->LR", X)
    return T


def cylinder_rdms(A, W):
    """Exact horizontal and vertical two-site density matrices rho[k1, b1, k2, b2]
    (trace one) on the infinite cylinder of circumference W (periodic in y)."""
    d = A.shape[0]
    a = _site(A)
    T = _column([a] * W)
    ev, vr = np.linalg.eig(T)
    i = np.argmax(np.abs(ev))
    lam = ev[i].real
    vR = vr[:, i].real
    evl, vl = np.linalg.eig(T.T)
    j = np.argmax(np.abs(evl))
    vL = vl[:, j].real
    norm2 = vL @ T @ T @ vR
    norm1 = vL @ T @ vR
    rho_h = np.zeros((d, d, d, d))
    rho_v = np.zeros((d, d, d, d))
    Topen = {}
    for k in range(d):
        for b in range(d):
            Topen[k, b] = _column([_site(A, (k, b))] + [a] * (W - 1))
    for k1 in range(d):
        for b1 in range(d):
            left = vL @ Topen[k1, b1]
            for k2 in range(d):
                for b2 in range(d):
                    rho_h[k1, b1, k2, b2] = left @ Topen[k2, b2] @ vR / norm2
                    Tv = _column([_site(A, (k1, b1)), _site(A, (k2, b2))] + [a] * (W - 2))
                    rho_v[k1, b1, k2, b2] = vL @ Tv @ vR / norm1
    return rho_h, rho_v, lam


def cylinder_diag_rdms(A, W):
    """Exact density matrices rho[k1, b1, k2, b2] (trace one) of the diagonal
    pair (x, y)-(x+1, y+1) and of the anti-diagonal pair (x+1, y)-(x, y+1) on the
    infinite cylinder of circumference W (W >= 2)."""
    d = A.shape[0]
    a = _site(A)
    T = _column([a] * W)
    ev, vr = np.linalg.eig(T)
    vR = vr[:, np.argmax(np.abs(ev))].real
    evl, vl = np.linalg.eig(T.T)
    vL = vl[:, np.argmax(np.abs(evl))].real
    norm2 = vL @ T @ T @ vR
    row0 = {(k, b): _column([_site(A, (k, b))] + [a] * (W - 1)) for k in range(d) for b in range(d)}
    row1 = {(k, b): _column([a, _site(A, (k, b))] + [a] * (W - 2)) for k in range(d) for b in range(d)}
    rho1 = np.zeros((d, d, d, d))
    rho2 = np.zeros((d, d, d, d))
    for k1 in range(d):
        for b1 in range(d):
            for k2 in range(d):
                for b2 in range(d):
                    # column x then column x+1; rows grow downwards
                    rho1[k1, b1, k2, b2] = vL @ row0[k1, b1] @ row1[k2, b2] @ vR / norm2
                    rho2[k1, b1, k2, b2] = vL @ row1[k2, b2] @ row0[k1, b1] @ vR / norm2
    return rho1, rho2


def bond_energy(rho, h):
    d = rho.shape[0]
    hh = h.reshape(d, d, d, d)                       # [b1, b2, k1, k2]
    return float(np.einsum("kbmc,bckm->", rho, hh) / np.einsum("kkmm->", rho))


def torus_state(A, L):
    """Amplitudes psi[s_1..s_{L*L}] of the uniform PEPS on an L x L torus
    (sites ordered row-major by (y, x)); small L only."""
    import itertools
    cnt = itertools.count()

    def sym():
        return next(cnt)
    hb = {(x, y): sym() for x in range(L) for y in range(L)}   # bond right of (x, y)
    vb = {(x, y): sym() for x in range(L) for y in range(L)}   # bond below (x, y)
    phys = {(x, y): sym() for x in range(L) for y in range(L)}
    ops = []
    for y in range(L):
        for x in range(L):
            u = vb[x, (y - 1) % L]
            l = hb[(x - 1) % L, y]
            dn = vb[x, y]
            r = hb[x, y]
            ops += [A, [phys[x, y], u, l, dn, r]]
    out = [phys[x, y] for y in range(L) for x in range(L)]
    return np.einsum(*ops, out, optimize="greedy")


def torus_bond_energies(A, L, h, v):
    """<h> on the horizontal bond (0, 0)-(1, 0) and <v> on the vertical bond
    (0, 0)-(0, 1) of the uniform PEPS on the L x L torus, from the full state
    vector (exact; small L only).  h, v in the convention op[(b1 b2), (k1 k2)]."""
    psi = torus_state(A, L)
    d = A.shape[0]
    nrm = float(np.sum(psi * psi))

    def pair(op, i, j):
        # sites i, j in the row-major (y, x) order of torus_state
        o = np.asarray(op).reshape(d, d, d, d)                  # [b1, b2, k1, k2]
        x = np.moveaxis(psi, (i, j), (0, 1))
        hx = np.einsum("abkm,km...->ab...", o, x)
        return float(np.sum(x * hx)) / nrm

    return pair(h, 0, 1), pair(v, 0, L)


def cylinder_cell_rdms(cell, W):
    """Exact density matrices of a unit cell cell[x][y] (Lx columns, Ly rows) on
    the infinite cylinder of circumference W (periodic in y, W a multiple of Ly):
    per site (x, y) the horizontal pair (x, y)-(x+1, y), the vertical pair
    (x, y)-(x, y+1) (rho[k1, b1, k2, b2], trace one) and the single site
    (rho[k, b]).  The column transfer matrices T_x of the cell's columns are
    multiplied along the cylinder's axis; the boundary vectors are the dominant
    left and right eigenvectors of one unit T_0 ... T_{Lx-1}."""
    Lx, Ly = len(cell), len(cell[0])
    assert W % Ly == 0
    d = np.asarray(cell[0][0]).shape[0]
    A = [[np.asarray(a) for a in col] for col in cell]
    closed = [[_site(A[x][y % Ly]) for y in range(W)] for x in range(Lx)]
    T = [_column(closed[x]) for x in range(Lx)]
    U = T[0]
    for x in range(1, Lx):
        U = U @ T[x]
    ev, vr = np.linalg.eig(U)
    vR = vr[:, np.argmax(np.abs(ev))].real
    evl, vl = np.linalg.eig(U.T)
    vL = vl[:, np.argmax(np.abs(evl))].real

    def opened(x, fixed):
        sites = list(closed[x])
        for y, kb in fixed.items():
            sites[y % W] = _site(A[x][y % Ly], kb)
        return _column(sites)

    def chain(cols):
        # vL (product over the 2 Lx columns of two units) vR, columns given per position
        vec = vL
        for M in cols:
            vec = vec @ M
        return float(vec @ vR)

    two = [T[i % Lx] for i in range(2 * Lx)]
    norm2 = chain(two)
    norm1 = chain(two[:Lx])
    out = {}
    for x in range(Lx):
        for y in range(Ly):
            rh = np.zeros((d, d, d, d))
            rv = np.zeros((d, d, d, d))
            r1 = np.zeros((d, d))
            for k1 in range(d):
                for b1 in range(d):
                    cols = list(two[:Lx])
                    cols[x] = opened(x, {y: (k1, b1)})
                    r1[k1, b1] = chain(cols) / norm1
                    for k2 in range(d):
                        for b2 in range(d):
                            cols = list(two)
                            cols[x] = opened(x, {y: (k1, b1)})
                            cols[x + 1] = opened((x + 1) % Lx, {y: (k2, b2)})
                            rh[k1, b1, k2, b2] = chain(cols) / norm2
                            cols = list(two[:Lx])
                            cols[x] = opened(x, {y: (k1, b1), y + 1: (k2, b2)})
                            rv[k1, b1, k2, b2] = chain(cols) / norm1
            out[x, y] = (rh, rv, r1)
    return out


def site_energy(rho1, op):
    return float(np.einsum("kb,bk->", rho1, np.asarray(op)) / np.trace(rho1))
