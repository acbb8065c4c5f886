"""Mean-field (chi = 1, belief-propagation) metric preconditioner (oracle,
test infrastructure: only tests/, the smoke check and the benchmark's CPU
baseline use it).

Sec. III.B: setting the bond dimension of the environment of the local
metric (Eq. equ:local_metric) to 1 cuts the preconditioner's cost further;
such a chi = 1 environment is what belief propagation on the double-layer
network gives, a mean-field approximation of the environment, and the
inverse preconditioner then becomes almost trivial.  App. A compares this
preconditioner with the local metric and with no preconditioner.

Readings (the paper gives no formulas for this variant):

* A message lives on a bond and a direction: a real D x D matrix m[k, b]
  over the ket and bra index of that bond.  Site s sends through its leg
  lam the contraction of A_s and A_s (physical legs joined) with the
  messages arriving on its other three legs:
      out_s^lam[k, b] = sum A_s[p, .. k ..] A_s[p, .. b ..] prod_{mu != lam} in_s^mu,
  symmetrised and divided by its trace.  All messages of one sweep are
  computed from the previous sweep's (parallel schedule), starting from
  identity / D; the sweeps stop when no entry of any message changes by
  more than tol.
* The message arriving at site (x, y) on leg u is the one sent downwards
  by (x, y-1) (y grows downwards), on leg l the one sent right by (x-1, y),
  on leg d the one sent up by (x, y+1), on leg r the one sent left by
  (x+1, y); indices are periodic in the unit cell.
* The metric of site s is 1_d (x) in_u (x) in_l (x) in_d (x) in_r on
  A[p, u, l, d, r], scaled (as the local metric) so that <A|N|A> = 1.
  P = N + delta I is inverted exactly in the eigenbases of the four
  messages (Sec. III.B regularisation).

Parity pins (tests/test_oracle_bp.py): a D=1 product state gives the closed
form g / (1/|A|^2 + delta); with trivial vertical legs the horizontal
messages are the dominant eigenvectors of the MPS transfer matrix
(numpy eig); the eigenbasis solve equals a dense solve of the Kronecker
matrix; messages are symmetric positive semi-definite fixed points.
"""
from __future__ import annotations

import numpy as np

LEGS = ("u", "l", "d", "r")
# the leg of the neighbour that faces leg `lam`, and that neighbour's offset
_OPP = {"u": "d", "l": "r", "d": "u", "r": "l"}
_STEP = {"u": (0, -1), "l": (-1, 0), "d": (0, 1), "r": (1, 0)}


def _outgoing(A, ins, lam):
    """The message site A sends through leg lam, from the three incoming ones."""
    k = dict(zip(LEGS, "ulde"))   # ket labels (e stands for r)
    b = dict(zip(LEGS, "ULDE"))   # bra labels
    ket = "p" + "".join(k[m] for m in LEGS)
    bra = "p" + "".join(b[m] for m in LEGS)
    ops, subs = [A], [ket]
    for m in LEGS:
        if m != lam:
            ops.append(ins[m])
            subs.append(k[m] + b[m])
    ops.append(A)
    subs.append(bra)
    out = np.einsum(",".join(subs) + "->" + k[lam] + b[lam], *ops, optimize=True)
    return out


def _normalise(m):
    m = 0.5 * (m + m.T)
    return m / np.trace(m)


def incoming(msgs, Lx, Ly, x, y):
    """The four messages arriving at site (x, y), by leg."""
    ins = {}
    for lam in LEGS:
        dx, dy = _STEP[lam]
        nx, ny = (x + dx) % Lx, (y + dy) % Ly
        ins[lam] = msgs[(nx, ny, _OPP[lam])]
    return ins


def bp_messages(cell, tol=1e-12, maxit=1000):
    """Fixed point of the message sweeps.  cell[x][y] = A[p, u, l, d, r].
    Returns (messages keyed (x, y, leg sent), sweeps, last change)."""
    Lx, Ly = len(cell), len(cell[0])
    D = cell[0][0].shape[1]
    msgs = {(x, y, lam): np.eye(D) / D for x in range(Lx) for y in range(Ly) for lam in LEGS}
    change = np.inf
    it = 0
    for it in range(1, maxit + 1):
        new = {}
        for x in range(Lx):
            for y in range(Ly):
                ins = incoming(msgs, Lx, Ly, x, y)
                for lam in LEGS:
                    new[(x, y, lam)] = _normalise(_outgoing(np.asarray(cell[x][y]), ins, lam))
        change = max(np.max(np.abs(new[k] - msgs[k])) for k in msgs)
        msgs = new
        if change <= tol:
            break
    return msgs, it, change


def bp_metric_factors(cell, msgs, x, y):
    """The four incoming messages of site (x, y) and the scale c with
    c <A| 1 (x) m_u (x) m_l (x) m_d (x) m_r |A> = 1."""
    Lx, Ly = len(cell), len(cell[0])
    ins = incoming(msgs, Lx, Ly, x, y)
    A = np.asarray(cell[x][y])
    nrm = np.einsum("puldr,uU,lL,dD,rR,pULDR->", A, ins["u"], ins["l"], ins["d"], ins["r"], A, optimize=True)
    return ins, 1.0 / nrm


def bp_precondition(cell, g_cell, delta, tol=1e-12, maxit=1000):
    """(N_bp + delta I)^-1 g for every tensor of the cell.  Returns
    (cell of preconditioned tensors, sweeps, last change)."""
    msgs, it, change = bp_messages(cell, tol=tol, maxit=maxit)
    Lx, Ly = len(cell), len(cell[0])
    out = [[None] * Ly for _ in range(Lx)]
    for x in range(Lx):
        for y in range(Ly):
            ins, c = bp_metric_factors(cell, msgs, x, y)
            lam, V = {}, {}
            for k in LEGS:
                lam[k], V[k] = np.linalg.eigh(ins[k])
            g = np.asarray(g_cell[x][y])
            gt = np.einsum("puldr,ua,lb,dc,re->pabce", g, V["u"], V["l"], V["d"], V["r"], optimize=True)
            den = c * np.einsum("a,b,c,e->abce", lam["u"], lam["l"], lam["d"], lam["r"]) + delta
            xt = gt / den[None]
            out[x][y] = np.einsum("pabce,ua,lb,dc,re->puldr", xt, V["u"], V["l"], V["d"], V["r"], optimize=True)
    return out, it, change
