"""Seeded synthetic iPEPS inputs shared by the CUDA path, the tests and the bench.

This module holds input generation only: random tensors with the shapes, value
distributions and seeds of the workloads the paper's method is exercised on
(random real iPEPS tensors, Sec. IV.A and IV.B).  It contains none of the
method's arithmetic, so both the oracle and the CUDA path may draw from it.

Tensor layout everywhere: A[x][y] has shape (d, D, D, D, D) with legs
(s, u, l, d, r) = (physical, up, left, down, right), row-major, float64.
"""
from __future__ import annotations

import numpy as np


def uniform_cell(Lx: int, Ly: int, d: int, D: int, seed: int, unit_max: bool = True):
    """Unit cell of i.i.d. uniform[-1, 1] tensors, each scaled to max|A| = 1."""
    rng = np.random.default_rng(seed)
    cell = []
    for _x in range(Lx):
        col = []
        for _y in range(Ly):
            a = rng.uniform(-1.0, 1.0, size=(d, D, D, D, D))
            if unit_max:
                a = a / np.max(np.abs(a))
            col.append(a)
        cell.append(col)
    return cell


def gaussian_cell(Lx: int, Ly: int, d: int, D: int, seed: int):
    """Unit cell of i.i.d. standard normal tensors."""
    rng = np.random.default_rng(seed)
    return [[rng.standard_normal((d, D, D, D, D)) for _y in range(Ly)] for _x in range(Lx)]


def neel_seed_cell(D: int, seed: int, eps_uniform: float = 1e-2, eps_gauss: float = 1e-2):
    """1x1 cell: the D=1 product state (spinor (1, 0), uniform in the sublattice-rotated
    frame) embedded at virtual index 0 of a D-dimensional tensor, plus
    eps_gauss * N(0, 1) and eps_uniform * U[-1, 1] noise on every entry."""
    rng = np.random.default_rng(seed)
    a = np.zeros((2, D, D, D, D))
    a[0, 0, 0, 0, 0] = 1.0
    a = a + eps_gauss * rng.standard_normal(a.shape) + eps_uniform * rng.uniform(-1.0, 1.0, a.shape)
    return [[a]]


def product_state_cell(Lx: int, Ly: int, spinors, D: int = 1):
    """Product state: A[s, 0, 0, 0, 0] = spinor[s] for each site, zero elsewhere."""
    cell = []
    k = 0
    for _x in range(Lx):
        col = []
        for _y in range(Ly):
            sp = np.asarray(spinors[k % len(spinors)], dtype=np.float64)
            a = np.zeros((sp.shape[0], D, D, D, D))
            a[:, 0, 0, 0, 0] = sp
            col.append(a)
            k += 1
        cell.append(col)
    return cell


def perturbed_cells(cell, count: int, eps: float, seed: int):
    """`count` copies of the unit cell, copy k with eps * U[-1, 1] added to every
    entry (generator seeded by (seed, k)): the sequence of nearby tensors a
    benchmark visits, as an optimiser's trial points do."""
    out = []
    for k in range(count):
        rng = np.random.default_rng([seed, k])
        out.append([[np.asarray(a) + eps * rng.uniform(-1.0, 1.0, np.shape(a)) for a in col] for col in cell])
    return out


def random_entries(n_total: int, count: int, seed: int):
    """Distinct flat indices for finite-difference probes."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=count, replace=False))


# Named workloads: (Lx, Ly, d, D, chi) and the generator producing A.
WORKLOADS = {
    # Heisenberg 1x1, D=2, chi=16, uniform[-1,1] normalised to unit max-abs, seed 0
    "heis_d2_chi16": dict(Lx=1, Ly=1, d=2, D=2, chi=16, gen=lambda: uniform_cell(1, 1, 2, 2, 0)),
    # Heisenberg 1x1, D=2, chi=16, Neel-like D=1 seed embedded in D=2 plus noise, seed 0
    "heis_d2_chi16_neel": dict(Lx=1, Ly=1, d=2, D=2, chi=16, gen=lambda: neel_seed_cell(2, 0)),
    # Heisenberg 1x1, D=2, chi=32 (chi = 8 D^2), Neel-like D=1 seed embedded in D=2 plus noise, seed 0
    "heis_d2_chi32": dict(Lx=1, Ly=1, d=2, D=2, chi=32, gen=lambda: neel_seed_cell(2, 0)),
    # Heisenberg 1x1, D=2, chi=32 (chi = 8 D^2), uniform[-1,1] normalised to unit max-abs, seed 0
    "heis_d2_chi32_rand": dict(Lx=1, Ly=1, d=2, D=2, chi=32, gen=lambda: uniform_cell(1, 1, 2, 2, 0)),
    # Heisenberg 1x1, D=4, chi=64, Neel-like D=1 seed embedded in D=4 plus noise, seed 0
    "heis_d4_chi64": dict(Lx=1, Ly=1, d=2, D=4, chi=64, gen=lambda: neel_seed_cell(4, 0)),
    # Kitaev (spin-1/2 dimers, d=4), 1x2 cell (Lx=2, Ly=1), D=6, chi=72, N(0,1), seed 0
    "kitaev_d6_chi72": dict(Lx=2, Ly=1, d=4, D=6, chi=72, gen=lambda: gaussian_cell(2, 1, 4, 6, 0)),
    # Heisenberg 2x2, D=8, chi=128, uniform[-1,1], seed 0
    "heis_2x2_d8_chi128": dict(Lx=2, Ly=2, d=2, D=8, chi=128, gen=lambda: uniform_cell(2, 2, 2, 8, 0)),
}
