"""Pins of the oracle's CTMRG environment and energy (Sec. III.A, Eq. equ:energy)."""
import numpy as np
import pytest
import torch

from oracle import ctmrg as C
from oracle import energy as En
from oracle import exact, models
from paper_2511_09546_gb300 import inputs


def _E(cell, ham, chi, tol=1e-11, maxit=400):
    env, it, err = C.ctmrg(cell, chi, tol=tol, maxit=maxit)
    Lx, Ly = len(cell), len(cell[0])
    return En.energy_terms(Lx, Ly, C.as_torch_cell(cell), env, ham), env


def test_product_state_heisenberg_rotated():
    # D=1 real spinors: every rotated bond gives -<Sx>^2 - <Sz>^2 = -1/4, E = -1/2
    rng = np.random.default_rng(3)
    for _ in range(3):
        sp = rng.standard_normal(2)
        terms, _ = _E(inputs.product_state_cell(1, 1, [sp]), models.heisenberg(True), 1)
        e = sum(float(t) for t in terms[0, 0])
        assert abs(e + 0.5) < 1e-13


def test_product_state_ferro_unrotated_2x2():
    sp = np.array([0.3, -1.1])
    cell = inputs.product_state_cell(2, 2, [sp])
    terms, _ = _E(cell, models.heisenberg(False), 1)
    for t in terms.values():
        assert abs(float(t[0]) - 0.25) < 1e-13 and abs(float(t[1]) - 0.25) < 1e-13


def test_product_state_kitaev_closed_form():
    # D=1 dimer product state: E = 1/2 [K<SzSz>_dimer + K<Sx_b><Sx_a> + K<Sy_b><Sy_a>],
    # <S^y> = 0 for a real state
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(4)
    psi /= np.linalg.norm(psi)
    sx = np.array([[0, 0.5], [0.5, 0]]); sz = np.diag([0.5, -0.5]); I2 = np.eye(2)
    ex = lambda op: psi @ op @ psi
    K = -1.0
    closed = 0.5 * (K * ex(np.kron(sz, sz)) + K * ex(np.kron(I2, sx)) * ex(np.kron(sx, I2)))
    cell = inputs.product_state_cell(2, 1, [psi])
    terms, env = _E(cell, models.kitaev_dimer(K), 1)
    E = En.energy(2, 1, C.as_torch_cell(cell), env, models.kitaev_dimer(K))
    assert abs(float(E) - closed) < 1e-13


@pytest.mark.parametrize("K", [0.3, 0.6])
def test_ising_peps_onsager(K):
    # symmetric Ising PEPS: <sigma^z sigma^z> on both bonds equals Onsager's
    terms, _ = _E([[exact.ising_peps(K)]], models.sigma_z_bond(), 16, tol=1e-9, maxit=120)
    ref = exact.onsager_nn(K)
    assert abs(float(terms[0, 0][0]) - ref) < 1e-10
    assert abs(float(terms[0, 0][1]) - ref) < 1e-10


def _chiral_ising_peps(K, h0, seed):
    """Non-symmetric PEPS whose norm is the Ising model at coupling K: bond
    weights w(s, s') = exp(K s s' + h0 (s - s')) (the h0 factors telescope
    along every closed row or column), each W = sqrt(w) split as Q P^T with a
    random invertible Q, so that no leg of A equals another."""
    rng = np.random.default_rng(seed)
    spins = np.array([1.0, -1.0])
    w = np.exp(K * np.outer(spins, spins) + h0 * (spins[:, None] - spins[None, :]))
    Wm = np.sqrt(w)
    Qh = rng.standard_normal((2, 2)) + 2 * np.eye(2)
    Qv = rng.standard_normal((2, 2)) + 2 * np.eye(2)
    Ph = (np.linalg.solve(Qh, Wm)).T        # Qh Ph^T = W
    Pv = (np.linalg.solve(Qv, Wm)).T
    # left leg uses Ph, right leg Qh, up leg Pv, down leg Qv
    return np.einsum("su,sl,sd,sr->suldr", Pv, Ph, Qv, Qh)


@pytest.mark.parametrize("K,h0", [(0.3, 0.4), (0.6, -0.25)])
def test_nonsymmetric_ising_peps_onsager(K, h0):
    A = _chiral_ising_peps(K, h0, seed=11)
    assert not np.allclose(A, A.transpose(0, 2, 1, 4, 3))
    terms, _ = _E([[A]], models.sigma_z_bond(), 8, tol=1e-10, maxit=500)
    ref = exact.onsager_nn(K)
    assert abs(float(terms[0, 0][0]) - ref) < 1e-9
    assert abs(float(terms[0, 0][1]) - ref) < 1e-9


def test_onsager_limits():
    # high-temperature series <ss> = tanh K + O(K^3); ordered limit -> 1
    assert abs(exact.onsager_nn(0.01) - np.tanh(0.01)) < 1e-5
    assert abs(exact.onsager_nn(2.0) - 1.0) < 1e-6


def test_rotation_and_gauge_invariance():
    ham = models.heisenberg(True)
    A = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()[0][0]
    t0, _ = _E([[A]], ham, 16)
    eh, ev = float(t0[0, 0][0]), float(t0[0, 0][1])
    # rotating the picture turns vertical bonds into horizontal ones
    t1, _ = _E([[A.transpose(0, 4, 1, 2, 3)]], ham, 16)
    assert abs(float(t1[0, 0][0]) - ev) < 1e-5 and abs(float(t1[0, 0][1]) - eh) < 1e-5
    # orthogonal gauge on both virtual bonds leaves the state unchanged
    rng = np.random.default_rng(2)
    G, _ = np.linalg.qr(rng.standard_normal((2, 2)))
    H, _ = np.linalg.qr(rng.standard_normal((2, 2)))
    Ag = np.einsum("ue,selbr,bd->suldr", G.T, A, G)
    Ag = np.einsum("lb,subdf,fr->suldr", H.T, Ag, H)
    t2, _ = _E([[Ag]], ham, 16)
    assert abs(float(t2[0, 0][0]) - eh) < 1e-9 and abs(float(t2[0, 0][1]) - ev) < 1e-9


def test_cylinders_approach_ctmrg():
    # the exact infinite-cylinder energies approach the 2D value with the circumference
    ham = models.heisenberg(True)
    A = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()[0][0]
    t0, _ = _E([[A]], ham, 16)
    ev = float(t0[0, 0][1])
    gaps = []
    for W in (3, 4, 5):
        _rh, rv, _ = exact.cylinder_rdms(A, W)
        gaps.append(abs(exact.bond_energy(rv, ham["v"]) - ev))
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 1e-2


def test_convergence_reported():
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    env, it, err = C.ctmrg(cell, 16, tol=1e-10, maxit=300)
    assert err < 1e-10 and it < 300


def test_c4v_state_has_equal_bonds():
    # a tensor symmetric under the 8 operations of the square: horizontal and
    # vertical bonds carry the same energy
    rng = np.random.default_rng(6)
    A = rng.uniform(-1, 1, (2, 2, 2, 2, 2))
    outs = []
    for rot in range(4):
        B = A
        for _ in range(rot):
            B = B.transpose(0, 4, 1, 2, 3)
        outs += [B, B.transpose(0, 1, 4, 3, 2)]
    A = sum(outs) / 8.0
    t, _ = _E([[A / np.max(np.abs(A))]], models.heisenberg(False), 12)
    assert abs(float(t[0, 0][0]) - float(t[0, 0][1])) < 1e-9


def test_degenerate_cut_detection():
    # the Neel-like D=4 seed at chi = 64 keeps numerically zero singular values
    # (degenerate cut); a random D=4 tensor at chi = 32 has a resolvable cut
    cell = inputs.WORKLOADS["heis_d4_chi64"]["gen"]()
    env, _, _ = C.ctmrg(cell, 64, tol=1e-10, maxit=200)
    assert min(C.cut_gaps(1, 1, C.as_torch_cell(cell), env, 64)) < 1e-8
    cell = inputs.uniform_cell(1, 1, 2, 4, 3)
    env, _, _ = C.ctmrg(cell, 32, tol=1e-10, maxit=300)
    assert min(C.cut_gaps(1, 1, C.as_torch_cell(cell), env, 32)) > 1e-8


@pytest.mark.parametrize("K", [0.3, 0.6])
def test_norm_per_site_is_onsager_free_energy(K):
    # the Ising PEPS norm network is the Ising partition function, so the CTMRG
    # norm per site kappa = Z(3x3) Z(2x2) / (Z(3x2) Z(2x3)) gives ln Z / N; the
    # two published forms of Onsager's result check each other
    assert abs(exact.onsager_log_z(K) - exact.onsager_log_z_1d(K)) < 1e-12
    A = exact.ising_peps(K)
    env, _, _ = C.ctmrg([[A]], 16, tol=1e-11, maxit=600)
    kappa = float(En.norm_per_site(C.as_torch_cell([[A]]), env))
    assert abs(np.log(kappa) - exact.onsager_log_z(K)) < 1e-11
