"""Energy per site from a CTMRG environment (oracle, test infrastructure).

Eq. (equ:energy), Sec. III.A: the energy is the expectation value of the
local Hamiltonian in the network of the iPEPS tensor, its conjugate and the
environment tensors, divided by the same network without the Hamiltonian.
The diagram is lost; the reading used here is the standard nearest-neighbour
two-site reduced density matrix:

    E = scale / (Lx Ly) * sum_{x, y} [ Tr(rho_h h) / Tr rho_h
                                      + Tr(rho_v v) / Tr rho_v
                                      + Tr(rho_1 h_site) / Tr rho_1 ]

rho_h of the bond (x, y)-(x+1, y) uses the left half of site (x, y)'s 3x3
patch and the right half of site (x+1, y)'s patch; rho_v is rho_h of the
picture rotated counter-clockwise (the lower site becomes the right site);
rho_1 is the single-site density matrix of the 3x3 patch.

Next-nearest-neighbour terms (J1-J2 model): a Hamiltonian with 'd1' / 'd2' operators adds, per
site (x, y), Tr(rho_d1 d1)/Tr rho_d1 for the diagonal (x, y)-(x+1, y+1) and
Tr(rho_d2 d2)/Tr rho_d2 for the anti-diagonal (x+1, y)-(x, y+1).  Both come
from the ring of the four enlarged corners of the 2x2 plaquette with upper-left
site (x, y) (the ring the projectors are built from), with the physical legs
of the two sites of the pair left open.

Parity pins: D=1 product states (closed forms), the Ising PEPS (Onsager),
infinite cylinders (tests/test_oracle_ctmrg.py).
"""
from __future__ import annotations

import numpy as np
import torch

from .ctmrg import DT, corner_ul, rot_A, rotate


def _env_left(C1, T1, T4, T3, C4):
    Lt = torch.einsum("ab,buvc->auvc", C1, T1)           # [C1.p, u, u', T1.n]
    Lb = torch.einsum("edfh,hg->edfg", T3, C4)           # [T3.p, d, d', C4.n]
    X = torch.einsum("auvc,glma->cuvlmg", Lt, T4)        # [T1.n, u, u', l, l', C4.n]
    return torch.einsum("cuvlmg,edfg->cuvlmdfe", X, Lb)  # [c, u, u', l, l', d, d', e]


def _env_right(T1, C2, T2, C3, T3):
    Rt = torch.einsum("cuvh,hi->cuvi", T1, C2)           # [T1.p, u, u', C2.n]
    Rb = torch.einsum("jk,kdfe->jdfe", C3, T3)           # [C3.p, d, d', T3.n]
    X = torch.einsum("cuvi,irwj->cuvrwj", Rt, T2)        # [T1.p, u, u', r, r', C3.p]
    return torch.einsum("cuvrwj,jdfe->cuvrwdfe", X, Rb)  # [c, u, u', r, r', d, d', e]


def _open_left(envL, A):
    # L[c, r, r', e, s, s'] with A ket (s) and bra (s') physical legs open
    X = torch.einsum("cuvlmdfe,suldr->cvmfesr", envL, A)
    return torch.einsum("cvmfesr,tvmfw->crwest", X, A)


def _open_right(envR, A):
    # R[c, l, l', e, s, s']
    X = torch.einsum("cuvrwdfe,suldr->cvwfesl", envR, A)
    return torch.einsum("cvwfesl,tvmfw->clmest", X, A)


def rho_h(Lx, Ly, A, env, x, y):
    """Two-site density matrix rho[s1, s1', s2, s2'] of the bond (x, y)-(x+1, y)."""
    x1 = (x + 1) % Lx
    eL = _env_left(env["C1"][x][y], env["T1"][x][y], env["T4"][x][y], env["T3"][x][y], env["C4"][x][y])
    eR = _env_right(env["T1"][x1][y], env["C2"][x1][y], env["T2"][x1][y], env["C3"][x1][y], env["T3"][x1][y])
    L = _open_left(eL, A[x][y])
    R = _open_right(eR, A[x1][y])
    return torch.einsum("cxyest,cxyeuv->stuv", L, R)


def rho_1(A, env, x, y):
    eL = _env_left(env["C1"][x][y], env["T1"][x][y], env["T4"][x][y], env["T3"][x][y], env["C4"][x][y])
    L = _open_left(eL, A[x][y])
    RC = torch.einsum("ci,irwj,je->crwe", env["C2"][x][y], env["T2"][x][y], env["C3"][x][y])
    return torch.einsum("crwest,crwe->st", L, RC)


def norm_per_site(A, env, x=0, y=0):
    """Norm per site kappa of the iPEPS from the environment of site (x, y):
    kappa = Z(3x3) Z(2x2) / (Z(3x2) Z(2x3)), the networks of the site's own
    eight boundary tensors with the double-layer site in the middle, with no
    site (corners only), and with the middle row or column removed (the facing
    edge legs joined).  Each boundary tensor appears equally often above and
    below the fraction line, so their normalisation cancels."""
    C1, C2, C3, C4 = (env[n][x][y] for n in ("C1", "C2", "C3", "C4"))
    T1, T2, T3, T4 = (env[n][x][y] for n in ("T1", "T2", "T3", "T4"))
    a = A[x][y]
    z9 = torch.einsum("ab,buvc,ce,erwf,fg,gdth,hi,ilma,suldr,svmtw->", C1, T1, C2, T2, C3, T3, C4, T4, a, a)
    z4 = torch.einsum("ab,bc,cd,da->", C1, C2, C3, C4)
    # middle row removed: T1's (ket, bra) meet T3's; C2 meets C3, C4 meets C1
    z6h = torch.einsum("ab,buvc,ce,eg,guvh,ha->", C1, T1, C2, C3, T3, C4)
    # middle column removed: T2's (ket, bra) meet T4's; C1 meets C2, C3 meets C4
    z6v = torch.einsum("ab,be,erwf,fg,gh,hrwa->", C1, C2, T2, C3, C4, T4)
    return z9 * z4 / (z6h * z6v)


def corner_open(C1, T1, T4, A):
    """Upper-left enlarged corner with the site's ket and bra physical legs open:
    [(T4.prev, d, d'), (T1.next, r, r'), s, s']."""
    X = torch.einsum("ab,bcde->acde", C1, T1)            # [C1.p, u, u', T1.n]
    X = torch.einsum("fgha,acde->fghcde", T4, X)         # [T4.p, l, l', u, u', T1.n]
    X = torch.einsum("fghcde,scgjk->fhdesjk", X, A)      # ket A on (u, l)
    X = torch.einsum("fhdesjk,tdhmn->fjmeknst", X, A)    # bra A on (u', l'), physical t open
    p, D1, _, n, D2, _, d, _ = X.shape
    return X.reshape(p * D1 * D1, n * D2 * D2, d, d)


def rho_diag(Lx, Ly, A, env, x, y, which):
    """Two-site density matrix rho[s1, s1', s2, s2'] of the plaquette with
    upper-left site (x, y): which=1 pairs (x, y) with (x+1, y+1), which=2 pairs
    (x+1, y) with (x, y+1)."""
    x1, y1 = (x + 1) % Lx, (y + 1) % Ly
    args = [
        (env["C1"][x][y], env["T1"][x][y], env["T4"][x][y], A[x][y]),
        (env["C2"][x1][y], env["T2"][x1][y], env["T1"][x1][y], rot_A(A[x1][y])),
        (env["C3"][x1][y1], env["T3"][x1][y1], env["T2"][x1][y1], rot_A(rot_A(A[x1][y1]))),
        (env["C4"][x][y1], env["T4"][x][y1], env["T3"][x][y1], rot_A(rot_A(rot_A(A[x][y1])))),
    ]
    opened = (0, 2) if which == 1 else (1, 3)
    Q = [corner_open(*a) if i in opened else corner_ul(*a) for i, a in enumerate(args)]
    if which == 1:
        R = torch.einsum("abst,bc->acst", Q[0], Q[1])
        Y = torch.einsum("ceuv,ea->cauv", Q[2], Q[3])
    else:
        R = torch.einsum("ab,bcst->acst", Q[0], Q[1])
        Y = torch.einsum("ce,eauv->cauv", Q[2], Q[3])
    return torch.einsum("acst,cauv->stuv", R, Y)


def bond_value(rho, h):
    """Tr(rho h) / Tr(rho) with rho[k1, b1, k2, b2] and h[(b1 b2), (k1 k2)]."""
    d = rho.shape[0]
    hh = h.reshape(d, d, d, d)                              # [b1, b2, k1, k2]
    num = torch.einsum("kbmc,bckm->", rho, hh)
    den = torch.einsum("kkmm->", rho)
    return num / den


def site_value(rho, h):
    return torch.einsum("kb,bk->", rho, h) / torch.einsum("kk->", rho)


def energy_terms(Lx, Ly, A, env, ham):
    """Per-site (x, y) -> [e_h, e_v, e_site, e_diagonals] before the per-site scale."""
    h = torch.as_tensor(np.asarray(ham["h"]), dtype=DT)
    v = torch.as_tensor(np.asarray(ham["v"]), dtype=DT)
    hs = None if ham.get("site") is None else torch.as_tensor(np.asarray(ham["site"]), dtype=DT)
    nnn = [None if ham.get(k) is None else torch.as_tensor(np.asarray(ham[k]), dtype=DT) for k in ("d1", "d2")]
    out = {}
    for x in range(Lx):
        for y in range(Ly):
            out[x, y] = [bond_value(rho_h(Lx, Ly, A, env, x, y), h), None,
                         site_value(rho_1(A, env, x, y), hs) if hs is not None else torch.zeros((), dtype=DT),
                         torch.zeros((), dtype=DT)]
            for which, op in ((1, nnn[0]), (2, nnn[1])):
                if op is not None:
                    out[x, y][3] = out[x, y][3] + bond_value(rho_diag(Lx, Ly, A, env, x, y, which), op)
    # vertical bonds: rotate counter-clockwise; site (x, y) -> (y, -x mod Lx) and
    # its lower neighbour becomes its right neighbour
    Lx2, Ly2, A2, env2 = rotate(Lx, Ly, A, env)
    for x in range(Lx):
        for y in range(Ly):
            xr, yr = y, (-x) % Lx
            out[x, y][1] = bond_value(rho_h(Lx2, Ly2, A2, env2, xr, yr), v)
    return out


def energy(Lx, Ly, A, env, ham):
    terms = energy_terms(Lx, Ly, A, env, ham)
    tot = sum(t[0] + t[1] + t[2] + t[3] for t in terms.values())
    return ham.get("scale", 1.0) * tot / (Lx * Ly)
