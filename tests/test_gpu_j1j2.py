"""J1-J2 next-nearest-neighbour terms (2x2 plaquette ring) on the GPU against
the oracle: energy and fixed-point gradient at the FP64 bar (|dE| <= 1e-10,
relative gradient error <= 1e-8), and the Neel closed form."""
import numpy as np
import pytest
import torch

from oracle import gradient as OG
from oracle import models as OM
from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


def _dev(ip, cell):
    return torch.as_tensor(ip.cell_tensor(cell), device="cuda")


def test_neel_closed_form(ip):
    cell = inputs.product_state_cell(1, 1, [[0.6, 0.8]])
    A = _dev(ip, cell)
    env, _, _ = ip.ctmrg(A, 4, tol=1e-13, maxit=50)
    E, g = ip.energy_grad(A, env, ip.ham_j1j2(1.0, 0.37, True))
    assert abs(E - (-0.5 + 0.37 / 2)) < 1e-13


def test_j1j2_1x1_rotated(ip):
    cell = inputs.uniform_cell(1, 1, 2, 2, 0)
    A = _dev(ip, cell)
    env, _, err = ip.ctmrg(A, 12, tol=1e-12, maxit=600)
    assert err < 1e-12
    E, g = ip.energy_grad(A, env, ip.ham_j1j2(1.0, 0.5, True))
    Eo, go = OG.energy_and_gradient(cell, OM.j1j2(1.0, 0.5, True), 12, tol=1e-12)
    assert abs(E - Eo) <= 1e-10
    gg = g.cpu().numpy()[0, 0]
    assert np.linalg.norm(gg - go[0][0]) <= 1e-8 * np.linalg.norm(go[0][0])


def test_j1j2_2x2_unrotated(ip):
    cell = inputs.uniform_cell(2, 2, 2, 2, seed=3)
    A = _dev(ip, cell)
    env, _, _ = ip.ctmrg(A, 8, tol=1e-11, maxit=800)
    E, g = ip.energy_grad(A, env, ip.ham_j1j2(1.0, 0.3, False))
    Eo, go = OG.energy_and_gradient(cell, OM.j1j2(1.0, 0.3, False), 8, tol=1e-11, maxit=800)
    assert abs(E - Eo) <= 1e-10
    gg = g.cpu().numpy()
    num = sum(np.linalg.norm(gg[x, y] - go[x][y]) ** 2 for x in range(2) for y in range(2)) ** 0.5
    den = sum(np.linalg.norm(go[x][y]) ** 2 for x in range(2) for y in range(2)) ** 0.5
    assert num <= 1e-8 * den
