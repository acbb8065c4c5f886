"""Pins of the oracle's multi-site unit cells (1x2 and 2x2) for CTMRG, the
energy and the fixed-point gradient (Sec. III.A; Sec. IV.B: every tensor of the
cell is its own variable).

Each pin uses tensors that differ from site to site, so that a wrong neighbour
offset anywhere in the cell's bookkeeping (which boundary tensor a move reads or
writes, which site an energy term pairs) changes the result:
  * the Ising PEPS with a different invertible gauge on every bond (the norm
    network is still the Ising partition function: every bond term equals
    Onsager's nearest-neighbour correlator);
  * one D=2 tensor dressed with a different orthogonal gauge on every bond of
    the cell (the state is the translation-invariant 1x1 state, and CTMRG's
    SVD projectors are covariant under orthogonal gauges): bond terms and
    corner spectra equal the 1x1 ones, and the per-site gradients are the
    gauge-transformed 1x1 gradient divided by the number of sites;
  * random distinct tensors against the exact infinite cylinder of the same
    cell (circumference 4), which approaches the 2D values;
  * central finite differences of the cell's energy.
"""
import numpy as np
import pytest

from oracle import ctmrg as C
from oracle import energy as En
from oracle import exact as X
from oracle import gradient as G
from oracle import models
from paper_2511_09546_gb300 import inputs


def _orth(rng, D):
    q, r = np.linalg.qr(rng.standard_normal((D, D)))
    return q * np.sign(np.diag(r))


def _dress(A, Lx, Ly, mats, inv_transpose):
    """cell[x][y] = A with bond matrix H[x][y] on the right leg of (x, y) and its
    partner on the left leg of (x+1, y); V[x][y] on the down leg of (x, y) and the
    partner on the up leg of (x, y+1).  The partner of G is G^-T (G itself for an
    orthogonal G), so that every bond carries G G^-1 = 1."""
    H, V = mats
    part = (lambda g: np.linalg.inv(g).T) if inv_transpose else (lambda g: g)
    cell = []
    for x in range(Lx):
        col = []
        for y in range(Ly):
            a = np.einsum("suldr,rR->suldR", A, H[x][y])
            a = np.einsum("suldr,lL->suLdr", a, part(H[(x - 1) % Lx][y]))
            a = np.einsum("suldr,dE->sulEr", a, V[x][y])
            a = np.einsum("suldr,uU->sUldr", a, part(V[x][(y - 1) % Ly]))
            col.append(a)
        cell.append(col)
    return cell


def _terms(cell, ham, chi, tol=1e-11, maxit=800):
    Lx, Ly = len(cell), len(cell[0])
    env, it, err = C.ctmrg(cell, chi, tol=tol, maxit=maxit)
    assert err < tol, (it, err)
    return En.energy_terms(Lx, Ly, C.as_torch_cell(cell), env, ham), env


@pytest.mark.parametrize("Lx,Ly,K", [(2, 2, 0.3), (2, 1, 0.6)])
def test_ising_with_bond_gauges_is_onsager(Lx, Ly, K):
    rng = np.random.default_rng(7)
    rnd = lambda: 1.5 * np.eye(2) + 0.4 * rng.standard_normal((2, 2))  # noqa: E731
    mats = ([[rnd() for _ in range(Ly)] for _ in range(Lx)], [[rnd() for _ in range(Ly)] for _ in range(Lx)])
    cell = _dress(X.ising_peps(K), Lx, Ly, mats, inv_transpose=True)
    assert not np.allclose(cell[0][0], cell[1][0])
    terms, _ = _terms(cell, models.sigma_z_bond(), 8, tol=1e-10)
    ref = X.onsager_nn(K)
    for x in range(Lx):
        for y in range(Ly):
            assert abs(float(terms[x, y][0]) - ref) < 1e-9, (x, y, "h")
            assert abs(float(terms[x, y][1]) - ref) < 1e-9, (x, y, "v")


@pytest.fixture(scope="module")
def one_by_one():
    A = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()[0][0]
    ham = models.heisenberg(False)
    E, g, info = G.energy_and_gradient([[A]], ham, 12, tol=1e-12, return_info=True)
    terms = En.energy_terms(1, 1, C.as_torch_cell([[A]]), info["env"], ham)
    spec = C.corner_spectra(1, 1, info["env"])
    return A, ham, E, g[0][0], terms[0, 0], spec


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (2, 1)])
def test_orthogonal_bond_gauges_reproduce_1x1(one_by_one, Lx, Ly):
    A, ham, E1, g1, t1, spec1 = one_by_one
    rng = np.random.default_rng(11)
    mats = ([[_orth(rng, 2) for _ in range(Ly)] for _ in range(Lx)],
            [[_orth(rng, 2) for _ in range(Ly)] for _ in range(Lx)])
    cell = _dress(A, Lx, Ly, mats, inv_transpose=False)
    assert not np.allclose(cell[0][0], cell[1][0])
    E, g, info = G.energy_and_gradient(cell, ham, 12, tol=1e-12, return_info=True)
    assert abs(E - E1) < 1e-10
    terms = En.energy_terms(Lx, Ly, C.as_torch_cell(cell), info["env"], ham)
    for x in range(Lx):
        for y in range(Ly):
            assert abs(float(terms[x, y][0]) - float(t1[0])) < 1e-10
            assert abs(float(terms[x, y][1]) - float(t1[1])) < 1e-10
    spec = C.corner_spectra(Lx, Ly, info["env"])
    for k in range(4):
        for i in range(Lx * Ly):
            s = spec[k * Lx * Ly + i]
            n = min(len(s), len(spec1[k]))
            assert np.max(np.abs(s[:n] - spec1[k][:n])) < 1e-9
    # per-site gradient = gauge-transformed 1x1 gradient / (Lx Ly)
    ref = _dress(g1, Lx, Ly, mats, inv_transpose=False)
    for x in range(Lx):
        for y in range(Ly):
            r = ref[x][y] / (Lx * Ly)
            assert np.linalg.norm(g[x][y] - r) <= 1e-8 * np.linalg.norm(r), (x, y)


def test_random_2x2_cell_matches_exact_cylinder():
    ham = models.heisenberg(False)
    cell = inputs.uniform_cell(2, 2, 2, 2, seed=3)
    terms, _ = _terms(cell, ham, 12)
    d2 = X.cylinder_cell_rdms(cell, 2)
    d4 = X.cylinder_cell_rdms(cell, 4)
    for (x, y), (rh, rv, _) in d4.items():
        for k, rho, op in ((0, rh, ham["h"]), (1, rv, ham["v"])):
            e = float(terms[x, y][k])
            far = abs(X.bond_energy(d2[x, y][k], op) - e)
            near = abs(X.bond_energy(rho, op) - e)
            assert near < far and near < 1e-2, (x, y, k, near, far)


def test_kitaev_1x2_cell_matches_exact_cylinder():
    ham = models.kitaev_dimer(-1.0)
    cell = inputs.gaussian_cell(2, 1, 4, 2, seed=0)
    terms, _ = _terms(cell, ham, 8)
    d2 = X.cylinder_cell_rdms(cell, 2)
    d4 = X.cylinder_cell_rdms(cell, 4)
    for (x, y), (rh, rv, r1) in d4.items():
        pairs = ((0, rh, d2[x, y][0], ham["h"], X.bond_energy), (1, rv, d2[x, y][1], ham["v"], X.bond_energy),
                 (2, r1, d2[x, y][2], ham["site"], X.site_energy))
        for k, rho, rho2, op, f in pairs:
            e = float(terms[x, y][k])
            near, far = abs(f(rho, op) - e), abs(f(rho2, op) - e)
            assert near < 1e-2 and near <= far + 1e-12, (x, y, k, near, far)


@pytest.mark.parametrize("case", ["heis_2x2", "kitaev_1x2"])
def test_cell_gradient_central_differences(case):
    if case == "heis_2x2":
        cell, ham, chi = inputs.uniform_cell(2, 2, 2, 2, seed=3), models.heisenberg(False), 8
    else:
        cell, ham, chi = inputs.gaussian_cell(2, 1, 4, 2, seed=0), models.kitaev_dimer(-1.0), 8
    Lx, Ly = len(cell), len(cell[0])
    E, g, info = G.energy_and_gradient(cell, ham, chi, tol=1e-12, return_info=True)
    h = 1e-6
    n = cell[0][0].size
    rng = np.random.default_rng(2)
    for x, y in [(Lx - 1, Ly - 1), (0, 0)]:
        for i in rng.choice(n, 2, replace=False):
            vals = []
            for sgn in (1, -1):
                c = [[a.copy() for a in col] for col in cell]
                c[x][y].ravel()[i] += sgn * h
                e, _ = G.energy_at(c, ham, chi, tol=1e-12, maxit=800, env=info["env"])
                vals.append(e)
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[x][y].ravel()[i]) < 5e-8, (x, y, i, fd, g[x][y].ravel()[i])


def test_tiny_tori_approach_ctmrg():
    # exact L x L tori (full state vector) close in on the CTMRG energy as L
    # grows, and the CTMRG energy settles as chi grows
    A = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()[0][0]
    ham = models.heisenberg(True)
    ectm = {}
    for chi in (6, 8, 16):
        t, _ = _terms([[A]], ham, chi, tol=1e-10, maxit=600)
        ectm[chi] = float(t[0, 0][0]) + float(t[0, 0][1])
    assert abs(ectm[16] - ectm[8]) < abs(ectm[8] - ectm[6])
    etor = {}
    for L in (2, 3, 4):
        eh, ev = X.torus_bond_energies(A, L, ham["h"], ham["v"])
        etor[L] = eh + ev
    gaps = [abs(etor[L] - ectm[16]) for L in (2, 3, 4)]
    assert gaps[0] > gaps[1] > gaps[2], gaps
    assert gaps[2] < 1e-2, gaps
