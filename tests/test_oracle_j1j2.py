"""Oracle pins of the next-nearest-neighbour (J1-J2) plaquette terms.

* D=1 product states: every real spinor in the sublattice-rotated frame is a
  Neel state, E = -J1/2 + J2/2 per site exactly.
* Partial traces: tracing either site of a diagonal pair's density matrix
  (2x2 plaquette network) gives the single-site density matrix of the 3x3
  patch network at the CTMRG fixed point.
* Reflection: for a C4v-symmetric tensor the two diagonals carry equal energy.
* Infinite cylinders: exact diagonal density matrices of circumference W
  approach the CTMRG values as W grows.
"""
import numpy as np
import pytest
import torch

from oracle import ctmrg as C
from oracle import energy as En
from oracle import exact
from oracle import models as M
from paper_2511_09546_gb300 import inputs


def _norm(r):
    d = r.shape[0]
    return r / torch.einsum("kkmm->", r) if r.dim() == 4 else r / torch.trace(r.reshape(d, d))


@pytest.mark.parametrize("theta", [0.0, 0.7, 2.1])
def test_product_state_closed_form(theta):
    spin = [np.cos(theta), np.sin(theta)]
    cell = inputs.product_state_cell(1, 1, [spin])
    J1, J2 = 1.0, 0.37
    env, _, _ = C.ctmrg(cell, 2, tol=1e-12, maxit=50)
    E = float(En.energy(1, 1, C.as_torch_cell(cell), env, M.j1j2(J1, J2)))
    assert E == pytest.approx(-J1 / 2 + J2 / 2, abs=1e-12)


@pytest.fixture(scope="module")
def converged_d2():
    cell = inputs.uniform_cell(1, 1, 2, 2, 0)
    env, it, err = C.ctmrg(cell, 16, tol=1e-12, maxit=600)
    assert err < 1e-12
    return C.as_torch_cell(cell), env


def test_partial_traces_match_single_site(converged_d2):
    A, env = converged_d2
    r1 = En.rho_1(A, env, 0, 0)
    r1 = (r1 / torch.trace(r1)).numpy()
    for which in (1, 2):
        rho = En.rho_diag(1, 1, A, env, 0, 0, which)
        rho = (rho / torch.einsum("kkmm->", rho)).numpy()
        first = np.einsum("kbmm->kb", rho)
        second = np.einsum("kkmb->mb", rho)
        # the two networks agree up to the chi = 16 truncation (~1e-8 here); a
        # leg or site mix-up changes the density matrix at O(1)
        assert np.max(np.abs(first - r1)) < 1e-6
        assert np.max(np.abs(second - r1)) < 1e-6


def _c4v(A):
    # average over the 8 symmetries of the square acting on (u, l, d, r)
    outs = []
    for rot in range(4):
        B = A
        for _ in range(rot):
            B = B.transpose(0, 4, 1, 2, 3)
        outs.append(B)
        outs.append(B.transpose(0, 1, 4, 3, 2))  # mirror l <-> r
    return sum(outs) / 8.0


def test_c4v_state_has_equal_diagonals():
    rng = np.random.default_rng(5)
    A = _c4v(rng.uniform(-1, 1, (2, 2, 2, 2, 2)))
    cell = [[A / np.max(np.abs(A))]]
    env, _, err = C.ctmrg(cell, 12, tol=1e-11, maxit=600)
    At = C.as_torch_cell(cell)
    h = M.heisenberg_bond(False)
    e1 = float(En.bond_value(En.rho_diag(1, 1, At, env, 0, 0, 1), torch.as_tensor(h)))
    e2 = float(En.bond_value(En.rho_diag(1, 1, At, env, 0, 0, 2), torch.as_tensor(h)))
    assert abs(e1 - e2) < 1e-9


def test_cylinders_approach_ctmrg(converged_d2):
    # exact cylinders of circumference 3, 4, 5 (diagonal: 0.00990, 0.01123,
    # 0.00935; anti-diagonal: -0.01160, -0.00687, -0.00616 against the CTMRG
    # 0.00959 and -0.00384 at chi = 16): both within 3e-3 at W = 5 and closer
    # than at W = 3 on average; swapping the two diagonals misses by ~1e-2
    A, env = converged_d2
    h = M.heisenberg_bond(False)
    ht = torch.as_tensor(h)
    ctm = [float(En.bond_value(En.rho_diag(1, 1, A, env, 0, 0, w), ht)) for w in (1, 2)]
    A0 = A[0][0].numpy()
    gap = {}
    for W in (3, 5):
        r1, r2 = exact.cylinder_diag_rdms(A0, W)
        gap[W] = (abs(exact.bond_energy(r1, h) - ctm[0]), abs(exact.bond_energy(r2, h) - ctm[1]))
    assert max(gap[5]) < 3e-3, gap
    assert sum(gap[5]) < sum(gap[3]), gap


def test_energy_adds_diagonals(converged_d2):
    A, env = converged_d2
    e0 = float(En.energy(1, 1, A, env, M.heisenberg(True)))
    eJ = float(En.energy(1, 1, A, env, M.j1j2(1.0, 0.5)))
    h = torch.as_tensor(M.heisenberg_bond(False))
    diag = sum(float(En.bond_value(En.rho_diag(1, 1, A, env, 0, 0, w), h)) for w in (1, 2))
    assert eJ == pytest.approx(e0 + 0.5 * diag, abs=1e-13)


def test_gradient_central_differences():
    # the fixed-point gradient with the diagonal terms against central differences
    from oracle import gradient as G

    cell = inputs.uniform_cell(1, 1, 2, 2, 0)
    ham = M.j1j2(1.0, 0.5)
    E, g, info = G.energy_and_gradient(cell, ham, 12, tol=1e-12, return_info=True)
    A = cell[0][0]
    h = 1e-6
    for i in inputs.random_entries(A.size, 3, seed=2):
        vals = []
        for sgn in (1, -1):
            Ap = A.copy().ravel()
            Ap[i] += sgn * h
            Ei, _ = G.energy_at([[Ap.reshape(A.shape)]], ham, 12, tol=1e-12, maxit=400, env=info["env"])
            vals.append(Ei)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[0][0].ravel()[i]) < 2e-8, (i, fd, g[0][0].ravel()[i])
