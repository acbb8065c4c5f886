"""Model Hamiltonians for the oracle (test infrastructure).

Sec. IV.A, Eq. (eq:H_heisenberg): H = sum_<ij> S_i . S_j, spin-1/2, square lattice.
The 1x1 unit cell uses the sublattice spin flip of Sec. IV.A (rotate every second
spin by pi about the y axis, U = i sigma_y), which turns the bond operator into
-SxSx + SySy - SzSz; this is real because SySy is real.
Sec. IV.B: Kitaev model H = -sum_<ij>_gamma S^gamma_i S^gamma_j on the honeycomb
lattice mapped to the square lattice by merging two sites (a, b) per tensor.
The workload here is spin-1/2 with K = -1 (K_gamma S S, K_gamma = -1): the z link
is inside the tensor, the x link joins b(x, y) to a(x+1, y), the y link joins
b(x, y) to a(x, y+1); the energy is reported per honeycomb site.

A Hamiltonian is a dict:
  'h'    : (d*d, d*d) horizontal bond operator on (left site, right site),
  'v'    : (d*d, d*d) vertical bond operator on (upper site, lower site),
  'site' : (d, d) on-site operator or None,
  'd1', 'd2' (optional): (d*d, d*d) operators on the diagonal (x, y)-(x+1, y+1)
           and the anti-diagonal (x+1, y)-(x, y+1) pairs of every plaquette,
  'scale': factor turning the per-tensor sum into the per-site energy.
Matrix convention: op[(b1*d + b2), (k1*d + k2)] = <b1 b2| op |k1 k2>.

Parity pins: the bond spectrum {-3/4, 1/4, 1/4, 1/4} (tests/test_oracle_models.py).
"""
from __future__ import annotations

import numpy as np

SX = np.array([[0.0, 0.5], [0.5, 0.0]])
SZ = np.array([[0.5, 0.0], [0.0, -0.5]])
# S^y = [[0, -i/2], [i/2, 0]]; only the real products S^y (x) S^y appear.
SY_SY = np.kron(np.array([[0.0, -0.5], [0.5, 0.0]]), np.array([[0.0, -0.5], [0.5, 0.0]])) * -1.0


def heisenberg_bond(rotated: bool) -> np.ndarray:
    """S_i . S_j as a 4x4 real matrix; with rotated=True the second spin is
    flipped by U = i sigma_y (S^x -> -S^x, S^z -> -S^z)."""
    sgn = -1.0 if rotated else 1.0
    return sgn * np.kron(SX, SX) + SY_SY + sgn * np.kron(SZ, SZ)


def heisenberg(rotated: bool = True, J: float = 1.0) -> dict:
    h = J * heisenberg_bond(rotated)
    return {"h": h, "v": h.copy(), "site": None, "scale": 1.0}


def j1j2(J1: float, J2: float, rotated: bool = True) -> dict:
    """J1-J2 Heisenberg model: J1 S.S on nearest-neighbour bonds (rotated frame
    as heisenberg()), J2 S.S on both diagonals.  Diagonal neighbours sit on the
    same sublattice, so the sublattice rotation leaves their bond unrotated."""
    ham = heisenberg(rotated, J1)
    ham["d1"] = J2 * heisenberg_bond(False)
    ham["d2"] = ham["d1"].copy()
    return ham


def kitaev_dimer(K: float = -1.0) -> dict:
    """Spin-1/2 Kitaev honeycomb model with two sites (a, b) merged per tensor."""
    I2 = np.eye(2)
    # single-dimer operators, basis s = 2*s_a + s_b
    sz_a, sz_b = np.kron(SZ, I2), np.kron(I2, SZ)
    sx_a, sx_b = np.kron(SX, I2), np.kron(I2, SX)
    # S^y_b (x) S^y_a across two dimers, built from the real product S^y (x) S^y
    # on the (b of site 1, a of site 2) pair embedded in the 16-dim space.
    site = K * sz_a @ sz_b
    h = K * np.kron(sx_b, sx_a)
    # embed SY_SY acting on (b1, a2) into (a1 b1) x (a2 b2)
    v = np.zeros((16, 16))
    for a1 in range(2):
        for b1 in range(2):
            for a2 in range(2):
                for b2 in range(2):
                    for b1p in range(2):
                        for a2p in range(2):
                            row = ((2 * a1 + b1) * 4) + (2 * a2 + b2)
                            col = ((2 * a1 + b1p) * 4) + (2 * a2p + b2)
                            v[row, col] += SY_SY[b1 * 2 + a2, b1p * 2 + a2p]
    v = K * v
    # energy per honeycomb site: each tensor carries one z, one x and one y link
    # (three links) for two sites
    return {"h": h, "v": v, "site": site, "scale": 0.5}


def sigma_z_bond() -> dict:
    """sigma^z sigma^z on every bond (used for the Ising-PEPS contraction pin)."""
    sz2 = np.diag([1.0, -1.0])
    h = np.kron(sz2, sz2)
    return {"h": h, "v": h.copy(), "site": None, "scale": 1.0}
