"""Directional CTMRG environment of an iPEPS unit cell (oracle, test infrastructure).

The paper contracts the network with CTMRG (Sec. III.A; Sec. IV.A uses the QR
variant without stating it).  This oracle follows the reading fixed for the
build: directional corner-transfer-matrix moves with four-corner SVD
projectors, iterated to a fixed point of the corner spectra.

Conventions
-----------
A[s, u, l, d, r] (physical, up, left, down, right); the picture has x to the
right and y downwards, sites (x, y) with 0 <= x < Lx, 0 <= y < Ly, periodic.
Every site (x, y) owns the eight tensors of its 3x3 patch

    C1 T1 C2
    T4 A  T2
    C4 T3 C3

whose legs run clockwise round the ring C1 T1 C2 T2 C3 T3 C4 T4: a corner is
C[prev, next], an edge is T[prev, ket, bra, next], where prev joins the
counter-clockwise neighbour and next the clockwise one, and (ket, bra) join
the A and conj(A) leg facing the edge.

Steps of one CTMRG iteration: a left move (absorb every column x into the
left boundary of column x+1, all columns at once), then the same move after
rotating the picture by 90, 180 and 270 degrees (top, right and bottom moves).
A left move:
  1. the four enlarged corners of the 2x2 patch with upper-left site (x, y);
  2. the halves R1 = Q_ul Q_ur and R2 = Q_lr Q_ll, the ring opened at the
     right cut M = R2 R1, and its truncated SVD M ~ U S V^T (top chi);
  3. projectors P_up = R2^T U S^-1/2 (upper side) and P_dn = R1 V S^-1/2
     (lower side) of the left cut between rows y and y+1; the inserted
     P_up P_dn^T reproduces the best rank-chi approximation of M;
  4. absorb: C1 <- P_up^T (C1 T1), T4 <- P_up^T (T4 A conj(A)) P_dn,
     C4 <- (T3 C4) P_dn, each divided by its Frobenius norm.

Convergence: the largest change, over all corners, of the normalised corner
singular values between iterations.

Parity pins: D=1 product states (exact energies), the Ising PEPS against
Onsager's nearest-neighbour correlator, and infinite-cylinder transfer
matrices (tests/test_oracle_ctmrg.py).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64
SV_CUTOFF = 1e-12
NAMES = ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4")
# rotating the picture counter-clockwise: new tensor name <- old tensor name
_ROT = {"C1": "C2", "C2": "C3", "C3": "C4", "C4": "C1",
        "T1": "T2", "T2": "T3", "T3": "T4", "T4": "T1"}


def rot_A(A):
    """A of the picture rotated counter-clockwise by 90 degrees: new up = old
    right, new left = old up, new down = old left, new right = old down."""
    return A.permute(0, 4, 1, 2, 3)


def rotate(Lx, Ly, A, env):
    """Rotate the unit cell counter-clockwise by 90 degrees.
    Site (x, y) moves to (y, -x mod Lx); the environment is relabelled."""
    Lx2, Ly2 = Ly, Lx
    A2 = [[rot_A(A[(-yp) % Lx][xp]) for yp in range(Ly2)] for xp in range(Lx2)]
    env2 = {new: [[env[old][(-yp) % Lx][xp] for yp in range(Ly2)] for xp in range(Lx2)]
            for new, old in _ROT.items()}
    return Lx2, Ly2, A2, env2


def as_torch_cell(cell):
    return [[torch.as_tensor(np.asarray(a), dtype=DT) for a in col] for col in cell]


# ---------------------------------------------------------------- init
def init_env(Lx, Ly, A):
    """Deterministic start: each boundary tensor is the neighbouring site's
    double-layer tensor with its outward legs traced ket against bra
    (bond dimension D^2)."""
    env = {n: [[None] * Ly for _ in range(Lx)] for n in NAMES}
    for x in range(Lx):
        for y in range(Ly):
            xm, xp, ym, yp = (x - 1) % Lx, (x + 1) % Lx, (y - 1) % Ly, (y + 1) % Ly
            a = A[xm][ym]; D = a.shape[1]
            # C1 from the up-left site: trace u, l; legs (d d') down, (r r') right
            env["C1"][x][y] = torch.einsum("suldr,sulek->derk", a, a).reshape(D * D, D * D)
            a = A[x][ym]
            # T1 from the site above: trace u; [ (l l'), (d d'), (r r') ]
            env["T1"][x][y] = torch.einsum("suldr,sumek->lmderk", a, a).reshape(D * D, D, D, D * D)
            a = A[xp][ym]
            # C2 from the up-right site: trace u, r; legs (l l') left, (d d') down
            env["C2"][x][y] = torch.einsum("suldr,sumer->lmde", a, a).reshape(D * D, D * D)
            a = A[xp][y]
            # T2 from the right site: trace r; [ (u u'), (l l'), (d d') ]
            env["T2"][x][y] = torch.einsum("suldr,svmer->uvlmde", a, a).reshape(D * D, D, D, D * D)
            a = A[xp][yp]
            # C3 from the down-right site: trace d, r; legs (u u') up, (l l') left
            env["C3"][x][y] = torch.einsum("suldr,svmdr->uvlm", a, a).reshape(D * D, D * D)
            a = A[x][yp]
            # T3 from the site below: trace d; [ (r r'), (u u'), (l l') ]
            env["T3"][x][y] = torch.einsum("suldr,svmdk->rkuvlm", a, a).reshape(D * D, D, D, D * D)
            a = A[xm][yp]
            # C4 from the down-left site: trace d, l; legs (r r') right, (u u') up
            env["C4"][x][y] = torch.einsum("suldr,svldk->rkuv", a, a).reshape(D * D, D * D)
            a = A[xm][y]
            # T4 from the left site: trace l; [ (d d'), (r r'), (u u') ]
            env["T4"][x][y] = torch.einsum("suldr,svlek->derkuv", a, a).reshape(D * D, D, D, D * D)
    for n in NAMES:
        for x in range(Lx):
            for y in range(Ly):
                t = env[n][x][y]
                env[n][x][y] = t / torch.linalg.norm(t)
    return env


# ---------------------------------------------------------------- moves
def corner_ul(C1, T1, T4, A):
    """Upper-left enlarged corner C1 T1 T4 A conj(A) as a matrix
    [(T4.prev, d, d'), (T1.next, r, r')]."""
    X = torch.einsum("ab,bcde->acde", C1, T1)            # [C1.p, u, u', T1.n]
    X = torch.einsum("fgha,acde->fghcde", T4, X)         # [T4.p, l, l', u, u', T1.n]
    X = torch.einsum("fghcde,scgjk->fhdesjk", X, A)      # [T4.p, l', u', T1.n, s, d, r]
    X = torch.einsum("fhdesjk,sdhmn->fjmekn", X, A)      # [T4.p, d, d', T1.n, r, r']
    p, D1, _, n, D2, _ = X.shape
    return X.reshape(p * D1 * D1, n * D2 * D2)


class _TruncSVD(torch.autograd.Function):
    """Top-k singular triplets from LAPACK's full SVD; the backward is the
    standard real-SVD adjoint written over the complete square basis
    (U^T dU antisymmetric),

        Mbar = U [ diag(Sbar) + (F o (U^T Ubar - Ubar^T U)) S
                   + S (F o (V^T Vbar - Vbar^T V)) ] V^T,
        F_ij = 1 / (s_j^2 - s_i^2)  (i != j),

    where Ubar, Vbar and Sbar vanish outside the kept columns, so only the
    entries with i or j kept are formed; this is the exact derivative of the
    truncated triplets (discarded directions included)."""

    @staticmethod
    def forward(M, k):
        U, S, Vh = torch.linalg.svd(M)
        V = Vh.T
        idx = torch.argmax(torch.abs(U[:, :k]), dim=0)
        sgn = torch.sign(U[idx, torch.arange(k)])
        sgn = torch.where(sgn == 0, torch.ones_like(sgn), sgn)
        U = U.clone(); V = V.clone()
        U[:, :k] *= sgn
        V[:, :k] *= sgn
        return U[:, :k], S[:k], V[:, :k], U, S, V

    @staticmethod
    def setup_context(ctx, inputs, output):
        _, k = inputs
        ctx.k = k
        ctx.save_for_backward(output[3], output[4], output[5])
        ctx.mark_non_differentiable(output[3], output[4], output[5])

    @staticmethod
    def backward(ctx, gU, gS, gV, _a, _b, _c):
        U, S, V = ctx.saved_tensors
        k = ctx.k
        n = S.shape[0]
        Ub = torch.zeros_like(U); Vb = torch.zeros_like(V); Sb = torch.zeros_like(S)
        if gU is not None:
            Ub[:, :k] = gU
        if gV is not None:
            Vb[:, :k] = gV
        if gS is not None:
            Sb[:k] = gS
        s2 = S * S
        diff = s2[None, :] - s2[:, None]                     # s_j^2 - s_i^2
        involved = torch.zeros((n, n), dtype=torch.bool)
        involved[:k, :] = True
        involved[:, :k] = True
        ok = involved & (diff != 0)
        F = torch.where(ok, 1.0 / torch.where(ok, diff, torch.ones_like(diff)), torch.zeros_like(diff))
        J = F * (U.T @ Ub - Ub.T @ U)
        K = F * (V.T @ Vb - Vb.T @ V)
        inner = torch.diag(Sb) + J * S[None, :] + S[:, None] * K
        return U @ inner @ V.T, None


def truncated_svd(M, chi):
    """Top-chi singular triplets of M with the sign convention that the
    largest-magnitude entry of every left vector is positive."""
    k = min(chi, M.shape[0], M.shape[1])
    U, S, V, _, _, _ = _TruncSVD.apply(M, k)
    return U, S, V


def projectors(Qul, Qur, Qlr, Qll, chi):
    R1 = Qul @ Qur
    R2 = Qlr @ Qll
    M = R2 @ R1
    U, S, V = truncated_svd(M, chi)
    keep = S > SV_CUTOFF * S[0]
    s_safe = torch.where(keep, S, torch.ones_like(S))
    inv_sqrt = torch.where(keep, s_safe ** -0.5, torch.zeros_like(S))
    P_up = (R2.T @ U) * inv_sqrt
    P_dn = (R1 @ V) * inv_sqrt
    return P_up, P_dn


def left_move(Lx, Ly, A, env, chi):
    P_up, P_dn = {}, {}
    for x in range(Lx):
        for y in range(Ly):
            x1, y1 = (x + 1) % Lx, (y + 1) % Ly
            Qul = corner_ul(env["C1"][x][y], env["T1"][x][y], env["T4"][x][y], A[x][y])
            Qur = corner_ul(env["C2"][x1][y], env["T2"][x1][y], env["T1"][x1][y], rot_A(A[x1][y]))
            Qlr = corner_ul(env["C3"][x1][y1], env["T3"][x1][y1], env["T2"][x1][y1],
                            rot_A(rot_A(A[x1][y1])))
            Qll = corner_ul(env["C4"][x][y1], env["T4"][x][y1], env["T3"][x][y1],
                            rot_A(rot_A(rot_A(A[x][y1]))))
            P_up[x, y], P_dn[x, y] = projectors(Qul, Qur, Qlr, Qll, chi)
    new = {n: [list(col) for col in env[n]] for n in NAMES}
    for x in range(Lx):
        x1 = (x + 1) % Lx
        for y in range(Ly):
            ym = (y - 1) % Ly
            C1, T1, T4 = env["C1"][x][y], env["T1"][x][y], env["T4"][x][y]
            T3, C4, a = env["T3"][x][y], env["C4"][x][y], A[x][y]
            # C1 <- P_up^T (C1 T1)    (cut between rows y-1 and y)
            X = torch.einsum("ab,bcde->acde", C1, T1)
            X = X.reshape(-1, X.shape[-1])
            c1 = P_up[x, ym].T @ X
            # T4 <- P_up^T (T4 A conj(A)) P_dn   (p: cut y|y+1, n: cut y-1|y)
            Y = torch.einsum("plqn,suldr->pqnsudr", T4, a)
            Y = torch.einsum("pqnsudr,svqeg->pdergnuv", Y, a)   # [p,d,d',r,r',n,u,u']
            p, D1, _, D2, _, n, D3, _ = Y.shape
            Y = Y.reshape(p * D1 * D1, D2, D2, n * D3 * D3)
            t4 = torch.einsum("ak,arsb,bm->krsm", P_up[x, y], Y, P_dn[x, ym])
            # C4 <- (T3 C4) P_dn    (cut between rows y and y+1)
            Z = torch.einsum("pden,nm->pmde", T3, C4)                 # [T3.p, C4.n, d, d']
            Z = Z.reshape(Z.shape[0], -1)
            c4 = Z @ P_dn[x, y]
            new["C1"][x1][y] = c1 / torch.linalg.norm(c1)
            new["T4"][x1][y] = t4 / torch.linalg.norm(t4)
            new["C4"][x1][y] = c4 / torch.linalg.norm(c4)
    return new


def cut_gaps(Lx, Ly, A, env, chi):
    """(s_chi - s_{chi+1}) / s_1 of the four-corner product M of every projector
    cut (all four directions, every site).  A gap at rounding level means the
    kept block of the truncation is not unique (a degenerate cut); parity of
    gradients is then not asserted."""
    gaps = []
    for _ in range(4):
        for x in range(Lx):
            for y in range(Ly):
                x1, y1 = (x + 1) % Lx, (y + 1) % Ly
                Qul = corner_ul(env["C1"][x][y], env["T1"][x][y], env["T4"][x][y], A[x][y])
                Qur = corner_ul(env["C2"][x1][y], env["T2"][x1][y], env["T1"][x1][y], rot_A(A[x1][y]))
                Qlr = corner_ul(env["C3"][x1][y1], env["T3"][x1][y1], env["T2"][x1][y1], rot_A(rot_A(A[x1][y1])))
                Qll = corner_ul(env["C4"][x][y1], env["T4"][x][y1], env["T3"][x][y1],
                                rot_A(rot_A(rot_A(A[x][y1]))))
                S = torch.linalg.svdvals((Qlr @ Qll) @ (Qul @ Qur))
                if S.numel() > chi:
                    gaps.append(float((S[chi - 1] - S[chi]) / S[0]))
        Lx, Ly, A, env = rotate(Lx, Ly, A, env)
    return gaps


def ctmrg_step(Lx, Ly, A, env, chi):
    """One CTMRG iteration: left, top, right and bottom moves."""
    for _ in range(4):
        env = left_move(Lx, Ly, A, env, chi)
        Lx, Ly, A, env = rotate(Lx, Ly, A, env)
    return env


def corner_spectra(Lx, Ly, env):
    out = []
    for n in ("C1", "C2", "C3", "C4"):
        for x in range(Lx):
            for y in range(Ly):
                s = torch.linalg.svdvals(env[n][x][y].detach())
                out.append((s / torch.linalg.norm(s)).numpy())
    return out


def spectra_change(old, new):
    err = 0.0
    for a, b in zip(old, new):
        n = max(a.shape[0], b.shape[0])
        aa, bb = np.zeros(n), np.zeros(n)
        aa[: a.shape[0]] = a
        bb[: b.shape[0]] = b
        err = max(err, float(np.linalg.norm(aa - bb)))
    return err


def ctmrg(cell, chi, tol=1e-10, maxit=500, env=None, miniter=2):
    """Run CTMRG to a fixed point of the corner spectra.
    Returns (env, iterations, final spectral change)."""
    Lx, Ly = len(cell), len(cell[0])
    A = as_torch_cell(cell)
    with torch.no_grad():
        if env is None:
            env = init_env(Lx, Ly, A)
        spec = corner_spectra(Lx, Ly, env)
        err = np.inf
        it = 0
        for it in range(1, maxit + 1):
            env = ctmrg_step(Lx, Ly, A, env, chi)
            new_spec = corner_spectra(Lx, Ly, env)
            err = spectra_change(spec, new_spec)
            spec = new_spec
            if err < tol and it >= miniter:
                break
    return env, it, err


# ---------------------------------------------------------------- gauge
def bond_of(name, x, y, Lx, Ly):
    """The two chi bonds (prev, next) of a boundary tensor; a bond is
    (side, column-or-cut, row-or-cut)."""
    xp, yp = (x + 1) % Lx, (y + 1) % Ly
    return {
        "C1": (("L", x, y), ("T", x, y)),
        "T1": (("T", x, y), ("T", xp, y)),
        "C2": (("T", xp, y), ("R", x, y)),
        "T2": (("R", x, y), ("R", x, yp)),
        "C3": (("R", x, yp), ("B", xp, y)),
        "T3": (("B", xp, y), ("B", x, y)),
        "C4": (("B", x, y), ("L", x, yp)),
        "T4": (("L", x, yp), ("L", x, y)),
    }[name]


def _as3(t):
    return t.reshape(t.shape[0], -1, t.shape[-1])


def solve_signs(Lx, Ly, env_ref, env_new):
    """Sign gauge sigma (one +-1 vector per chi bond) with
    env_ref ~ sigma . env_new elementwise.

    Every boundary tensor t with bonds (p, n) gives the overlaps
    W[i, j] = sum_mid ref[i, mid, j] new[i, mid, j] = sigma_p[i] sigma_n[j] |W[i, j]|.
    The nodes (bond, index) are joined by these weighted sign constraints and
    the signs are read off a maximum-weight spanning tree (Prim), so that
    structurally small entries (the ket/bra parity blocks of the corners)
    never decide a sign."""
    import heapq

    adj = {}
    for n in NAMES:
        for x in range(Lx):
            for y in range(Ly):
                ref = _as3(env_ref[n][x][y].detach()).numpy()
                new = _as3(env_new[n][x][y].detach()).numpy()
                W = np.einsum("imj,imj->ij", ref, new)
                bp, bn = bond_of(n, x, y, Lx, Ly)
                for i in range(W.shape[0]):
                    for j in range(W.shape[1]):
                        w = W[i, j]
                        if w == 0.0 or (bp == bn and i == j):
                            continue
                        a, b = (bp, i), (bn, j)
                        adj.setdefault(a, []).append((abs(w), b, 1.0 if w > 0 else -1.0))
                        adj.setdefault(b, []).append((abs(w), a, 1.0 if w > 0 else -1.0))
    val = {}
    # Prim's algorithm from the strongest node of each component
    order = sorted(adj, key=lambda k: -max(e[0] for e in adj[k]))
    for root in order:
        if root in val:
            continue
        val[root] = 1.0
        heap = [(-w, nb, s, root) for (w, nb, s) in adj[root]]
        heapq.heapify(heap)
        while heap:
            negw, nb, s, frm = heapq.heappop(heap)
            if nb in val:
                continue
            val[nb] = s * val[frm]
            for (w, nb2, s2) in adj[nb]:
                if nb2 not in val:
                    heapq.heappush(heap, (-w, nb2, s2, nb))
    sig = {}
    for n in NAMES:
        for x in range(Lx):
            for y in range(Ly):
                t = env_new[n][x][y]
                for b, dim in zip(bond_of(n, x, y, Lx, Ly), (t.shape[0], t.shape[-1])):
                    if b not in sig:
                        sig[b] = np.array([val.get((b, i), 1.0) for i in range(dim)])
    return sig


def apply_signs(Lx, Ly, env, sig):
    out = {n: [[None] * Ly for _ in range(Lx)] for n in NAMES}
    for n in NAMES:
        for x in range(Lx):
            for y in range(Ly):
                bp, bn = bond_of(n, x, y, Lx, Ly)
                t = env[n][x][y]
                sp = torch.as_tensor(sig[bp], dtype=DT)
                sn = torch.as_tensor(sig[bn], dtype=DT)
                shape = [t.shape[0]] + [1] * (t.dim() - 1)
                t = t * sp.reshape(shape)
                shape = [1] * (t.dim() - 1) + [t.shape[-1]]
                out[n][x][y] = t * sn.reshape(shape)
    return out


def refine_gauge(Lx, Ly, env_ref, env_new, sig, sweeps=400):
    """Orthogonal gauge G_b per chi bond (starting from the signs sig) with
    env_ref ~ G . env_new elementwise, G acting on the first and last legs of
    every boundary tensor: t'[i, ., j] = sum G_p[i, i'] t[i', ., j'] G_n[j, j'].

    Needed when the projector spectra have exactly degenerate pairs (a
    C4v-symmetric tensor gives them): a diagonal sign gauge cannot undo the
    rotation inside a pair.  Alternating orthogonal Procrustes: with the other
    bonds fixed, the overlap is linear in G_b (a bond that meets itself in an
    edge uses its current value on the other side), maximised by the polar
    factor of the accumulated overlap matrix."""
    G = {b: np.diag(v).astype(np.float64) for b, v in sig.items()}
    mats = []
    for n in NAMES:
        for x in range(Lx):
            for y in range(Ly):
                ref = _as3(env_ref[n][x][y].detach()).numpy()
                new = _as3(env_new[n][x][y].detach()).numpy()
                mats.append((bond_of(n, x, y, Lx, Ly), ref, new))
    for _ in range(sweeps):
        moved = 0.0
        for b in list(G):
            M = np.zeros_like(G[b])
            for (bp, bn), ref, new in mats:
                if bp == b:   # ref ~ G_b (new G_n^T): overlap with new on its last leg gauged
                    X = np.einsum("imj,kj->imk", new, G[bn])
                    M += np.einsum("imk,jmk->ij", ref, X)
                if bn == b:   # ref ~ (G_p new) G_b^T
                    Y = np.einsum("ki,imj->kmj", G[bp], new)
                    M += np.einsum("kmi,kmj->ij", ref, Y)
            u, _, vt = np.linalg.svd(M)
            Gb = u @ vt
            moved = max(moved, float(np.max(np.abs(Gb - G[b]))))
            G[b] = Gb
        if moved < 1e-15:
            break
    return G


def apply_gauge(Lx, Ly, env, G):
    """t'[i, ., j] = sum G_p[i, i'] t[i', ., j'] G_n[j, j'] for every boundary tensor."""
    out = {n: [[None] * Ly for _ in range(Lx)] for n in NAMES}
    for n in NAMES:
        for x in range(Lx):
            for y in range(Ly):
                bp, bn = bond_of(n, x, y, Lx, Ly)
                t = env[n][x][y]
                t3 = _as3(t)
                gp = torch.as_tensor(G[bp], dtype=DT)
                gn = torch.as_tensor(G[bn], dtype=DT)
                out[n][x][y] = torch.einsum("ik,kmj,lj->iml", gp, t3, gn).reshape(t.shape)
    return out


def env_diff(Lx, Ly, e1, e2):
    return max(float(torch.linalg.norm(e1[n][x][y] - e2[n][x][y]))
               for n in NAMES for x in range(Lx) for y in range(Ly))


def fixed_point(cell, chi, tol=1e-12, maxit=2000, env=None, gauge_refine_above=1e-8):
    """CTMRG to convergence, then the gauge that makes the converged
    environment an elementwise fixed point of one more iteration: the sign
    gauge, refined to an orthogonal gauge (refine_gauge) when the sign gauge
    leaves an elementwise residual above gauge_refine_above.
    Returns (env*, gauge, iterations, spectral change, elementwise residual);
    gauge is a dict of sign vectors or of orthogonal matrices (apply_fixed_gauge)."""
    Lx, Ly = len(cell), len(cell[0])
    env, it, err = ctmrg(cell, chi, tol=tol, maxit=maxit, env=env)
    A = as_torch_cell(cell)
    with torch.no_grad():
        e1 = ctmrg_step(Lx, Ly, A, env, chi)
        gauge = solve_signs(Lx, Ly, env, e1)
        res = env_diff(Lx, Ly, env, apply_signs(Lx, Ly, e1, gauge))
        if res > gauge_refine_above:
            G = refine_gauge(Lx, Ly, env, e1, gauge)
            res_g = env_diff(Lx, Ly, env, apply_gauge(Lx, Ly, e1, G))
            if res_g < res:
                gauge, res = G, res_g
    return env, gauge, it, err, res


def apply_fixed_gauge(Lx, Ly, env, gauge):
    """Apply a gauge returned by fixed_point (signs or orthogonal matrices)."""
    if next(iter(gauge.values())).ndim == 1:
        return apply_signs(Lx, Ly, env, gauge)
    return apply_gauge(Lx, Ly, env, gauge)
