"""Pins of the oracle's local metric and regularised GMRES solve
(Eq. equ:local_metric, Sec. III.B, Sec. III.C)."""
import numpy as np
import pytest
import torch

from oracle import ctmrg as C
from oracle import energy as En
from oracle import metric as Mt
from oracle.gmres import gmres
from paper_2511_09546_gb300 import inputs


@pytest.fixture(scope="module")
def cfg1_env():
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    env, _, _ = C.ctmrg(cell, 16, tol=1e-11, maxit=400)
    return cell, env


def test_metric_symmetric_and_psd(cfg1_env):
    cell, env = cfg1_env
    M = Mt.hole_env(env, 0, 0).numpy()
    assert np.linalg.norm(M - M.T) < 1e-10 * np.linalg.norm(M)
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev[0] >= -1e-10 * ev[-1]


def test_metric_norm_equals_norm_network(cfg1_env):
    # <A| 1 (x) M |A> is the norm network of the 3x3 patch, here computed
    # through the single-site density matrix instead
    cell, env = cfg1_env
    A = C.as_torch_cell(cell)
    n1 = float(Mt.norm_network(env, A[0][0], 0, 0))
    n2 = float(torch.einsum("ss->", En.rho_1(A, env, 0, 0)))
    assert abs(n1 - n2) < 1e-12 * abs(n2)
    Mn = Mt.local_metric(env, A[0][0], 0, 0).numpy()
    a = cell[0][0].reshape(2, -1)
    assert abs(np.einsum("si,ij,sj->", a, Mn, a) - 1.0) < 1e-12


def test_metric_has_physical_identity_structure(cfg1_env):
    # N_local acts as 1_d (x) M: the solve decouples over the physical index
    cell, env = cfg1_env
    A = C.as_torch_cell(cell)
    M = Mt.local_metric(env, A[0][0], 0, 0).numpy()
    rng = np.random.default_rng(0)
    g = rng.standard_normal((2, 2, 2, 2, 2))
    g[1] = 0.0
    x, _ = Mt.precondition(M, g, 0.1, krylov=40)
    assert np.max(np.abs(x[1])) == 0.0


def test_gmres_full_krylov_equals_direct(cfg1_env):
    cell, env = cfg1_env
    A = C.as_torch_cell(cell)
    M = Mt.local_metric(env, A[0][0], 0, 0).numpy()
    rng = np.random.default_rng(1)
    g = rng.standard_normal((2, 2, 2, 2, 2))
    delta = 0.05
    P = np.kron(np.eye(2), M) + delta * np.eye(32)
    direct = np.linalg.solve(P, g.ravel())
    x, rel = Mt.precondition(M, g, delta, krylov=32, restarts=1)
    assert np.linalg.norm(x.ravel() - direct) < 1e-9 * np.linalg.norm(direct)
    # the paper's rough solve: one cycle of Krylov dimension 30
    x30, rel30 = Mt.precondition(M, g, delta, krylov=30, restarts=1)
    assert rel30 < 1.0
    res = np.linalg.norm(P @ x30.ravel() - g.ravel()) / np.linalg.norm(g)
    assert abs(res - rel30) < 1e-8


def test_d1_closed_form():
    # D = 1: M is the scalar m = 1 / |A|^2 after normalisation, P^-1 g = g / (m + delta)
    sp = np.array([0.7, -1.3])
    cell = inputs.product_state_cell(1, 1, [sp])
    env, _, _ = C.ctmrg(cell, 1, tol=1e-13)
    A = C.as_torch_cell(cell)
    M = Mt.local_metric(env, A[0][0], 0, 0).numpy()
    m = 1.0 / np.sum(sp ** 2)
    assert abs(M[0, 0] - m) < 1e-14
    g = np.array([0.2, 0.5]).reshape(2, 1, 1, 1, 1)
    x, _ = Mt.precondition(M, g, 0.3)
    assert np.allclose(x, g / (m + 0.3), atol=1e-14)


def test_gmres_small_spd():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((50, 50))
    P = B @ B.T + 0.5 * np.eye(50)
    b = rng.standard_normal(50)
    x, rel, nmv = gmres(lambda v: P @ v, b, krylov=50, restarts=1)
    assert np.linalg.norm(P @ x - b) < 1e-9 * np.linalg.norm(b)
    assert nmv <= 50
