"""GPU path against the CPU oracle on the same seeded inputs (gauge-invariant outputs)."""
import numpy as np
import pytest
import torch

from oracle import ctmrg as OC
from oracle import energy as OE
from oracle import exact as OX
from oracle import gradient as OG
from oracle import metric as OMt
from oracle import models as OM
from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


def _dev(cell):
    from paper_2511_09546_gb300 import ipeps

    return torch.as_tensor(ipeps.cell_tensor(cell), device="cuda")


def test_heisenberg_d2_chi16_energy_spectra_gradient(ip):
    # D=2, chi=16 Heisenberg 1x1 (seeded uniform[-1,1], unit max-abs): FP64 bar
    # |dE| <= 1e-10, relative gradient error <= 1e-8
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    A = _dev(cell)
    env, it, err = ip.ctmrg(A, 16, tol=1e-12, maxit=600)
    assert err < 1e-12
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    Eo, go, info = OG.energy_and_gradient(cell, OM.heisenberg(True), 16, tol=1e-12, return_info=True)
    assert abs(E - Eo) <= 1e-10
    gg = g.cpu().numpy()[0, 0]
    assert np.linalg.norm(gg - go[0][0]) <= 1e-8 * np.linalg.norm(go[0][0])
    # corner spectra agree (gauge invariant)
    sp = env.corner_spectra()
    so = OC.corner_spectra(1, 1, info["env"])
    for k in range(4):
        n = so[k].shape[0]
        assert np.max(np.abs(sp[k, 0, :n] - so[k])) < 1e-9


def test_precondition_matches_oracle(ip):
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    A = _dev(cell)
    env, _, _ = ip.ctmrg(A, 16, tol=1e-12, maxit=600)
    rng = np.random.default_rng(4)
    gh = rng.standard_normal((1, 1, 2, 2, 2, 2, 2))
    oenv, _, _ = OC.ctmrg(cell, 16, tol=1e-12, maxit=600)
    M = OMt.local_metric(oenv, OC.as_torch_cell(cell)[0][0], 0, 0).numpy()
    for delta, kry in ((0.05, 30), (1e-3, 32), (0.5, 5)):
        x, res = ip.precondition(A, env, torch.as_tensor(gh, device="cuda"), delta, krylov=kry, restarts=1)
        xo, reso = OMt.precondition(M, gh[0, 0], delta, krylov=kry, restarts=1)
        xx = x.cpu().numpy()[0, 0]
        assert np.linalg.norm(xx - xo) <= 1e-9 * np.linalg.norm(xo), (delta, kry)
        assert abs(res - reso) < 1e-9


def test_product_state_closed_form(ip):
    cell = inputs.product_state_cell(1, 1, [[0.8, -0.35]])
    A = _dev(cell)
    env, _, _ = ip.ctmrg(A, 4, tol=1e-13, maxit=50)
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    assert abs(E + 0.5) < 1e-13
    assert float(g.abs().max()) < 1e-12


@pytest.mark.parametrize("K", [0.3, 0.6])
def test_ising_peps_onsager(ip, K):
    A = _dev([[OX.ising_peps(K)]])
    sz = np.kron(np.diag([1.0, -1.0]), np.diag([1.0, -1.0]))
    ham = ip.ham_create(2, sz, sz, None, 0.5)
    env, _, _ = ip.ctmrg(A, 16, tol=1e-9, maxit=150, allow_unconverged=True)
    assert abs(ip.energy(A, env, ham) - OX.onsager_nn(K)) < 1e-10


def test_kitaev_1x2_energy_gradient(ip):
    cell = inputs.gaussian_cell(2, 1, 4, 2, seed=0)
    A = _dev(cell)
    env, _, err = ip.ctmrg(A, 8, tol=1e-11, maxit=800)
    E, g = ip.energy_grad(A, env, ip.ham_kitaev(-1.0))
    Eo, go = OG.energy_and_gradient(cell, OM.kitaev_dimer(-1.0), 8, tol=1e-11, maxit=800)
    assert abs(E - Eo) <= 1e-10
    gg = g.cpu().numpy()
    num = sum(np.linalg.norm(gg[x, 0] - go[x][0]) ** 2 for x in range(2)) ** 0.5
    den = sum(np.linalg.norm(go[x][0]) ** 2 for x in range(2)) ** 0.5
    assert num <= 1e-8 * den


def test_heisenberg_2x2_unrotated(ip):
    cell = inputs.uniform_cell(2, 2, 2, 2, seed=3)
    A = _dev(cell)
    env, _, _ = ip.ctmrg(A, 8, tol=1e-11, maxit=800)
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(False))
    Eo, go = OG.energy_and_gradient(cell, OM.heisenberg(False), 8, tol=1e-11, maxit=800)
    assert abs(E - Eo) <= 1e-10
    gg = g.cpu().numpy()
    num = sum(np.linalg.norm(gg[x, y] - go[x][y]) ** 2 for x in range(2) for y in range(2)) ** 0.5
    den = sum(np.linalg.norm(go[x][y]) ** 2 for x in range(2) for y in range(2)) ** 0.5
    assert num <= 1e-8 * den


def test_errors_are_reported(ip):
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    A = _dev(cell)
    bad = A.clone()
    bad[0, 0, 0, 0, 0, 0, 0] = float("nan")
    with pytest.raises(ip.IpepsError) as e:
        ip.ctmrg(bad, 16)
    assert e.value.status == 4
    with pytest.raises(ip.IpepsError) as e:
        ip.ctmrg(A, 0)
    assert e.value.status == 1
    with pytest.raises(ip.IpepsError) as e:
        ip.ctmrg(A, 16, tol=1e-14, maxit=2)
    assert e.value.status == 5
