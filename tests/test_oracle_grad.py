"""Pins of the oracle's fixed-point gradient (Sec. III.A gradient; Sec. IV.A (n+N) scheme)."""
import numpy as np
import pytest

from oracle import gradient as G
from oracle import models
from paper_2511_09546_gb300 import inputs


@pytest.fixture(scope="module")
def cfg1():
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    ham = models.heisenberg(True)
    E, g, info = G.energy_and_gradient(cell, ham, 16, tol=1e-12, return_info=True)
    return cell, ham, E, g, info


def test_fixed_point_and_adjoint_converge(cfg1):
    _, _, _, _, info = cfg1
    assert info["fixed_point_residual"] < 1e-8
    assert info["adjoint_residual"] < 1e-12


def test_scale_invariance(cfg1):
    # E(cA) = E(A)  =>  <g, A> = 0
    cell, _, _, g, _ = cfg1
    assert abs(np.sum(g[0][0] * cell[0][0])) < 1e-10 * np.linalg.norm(g[0][0]) * np.linalg.norm(cell[0][0])


def test_central_differences_every_entry(cfg1):
    # all 32 entries of the D=2 tensor (the survey's cfg1 pin), step 1e-6
    cell, ham, _, g, info = cfg1
    A = cell[0][0]
    h = 1e-6
    fd = np.zeros(A.size)
    for i in range(A.size):
        vals = []
        for sgn in (1, -1):
            Ap = A.copy().ravel()
            Ap[i] += sgn * h
            E, _ = G.energy_at([[Ap.reshape(A.shape)]], ham, 16, tol=1e-12, maxit=400, env=info["env"])
            vals.append(E)
        fd[i] = (vals[0] - vals[1]) / (2 * h)
    assert np.max(np.abs(fd - g[0][0].ravel())) < 2e-8


def test_product_state_gradient_vanishes():
    # D=1 real spinors all have E = -1/2 in the rotated frame: g = 0
    cell = inputs.product_state_cell(1, 1, [[0.8, -0.35]])
    E, g = G.energy_and_gradient(cell, models.heisenberg(True), 1, tol=1e-13)
    assert abs(E + 0.5) < 1e-13
    assert np.max(np.abs(g[0][0])) < 1e-12


def test_unrolled_converges_to_fixed_point(cfg1):
    cell, ham, _, g, _ = cfg1
    errs = []
    for n in (2, 8, 32):
        _, gu = G.unrolled_gradient(cell, ham, 16, n, tol=1e-12)
        errs.append(np.linalg.norm(gu[0][0] - g[0][0]) / np.linalg.norm(g[0][0]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_gradient_orthogonal_to_gauge_directions(cfg1):
    # E is invariant under A -> G on (u, l), G^-1 on (d, r): the gradient is
    # orthogonal to the infinitesimal directions X A - A X^T on each bond (to the
    # chi = 16 truncation, which is not gauge covariant: ~5e-6 here, against
    # ~7e-2 for a random direction)
    cell, _, _, g, _ = cfg1
    A, g0 = cell[0][0], g[0][0]
    rng = np.random.default_rng(4)
    for _ in range(3):
        X, Y = rng.standard_normal((2, 2)), rng.standard_normal((2, 2))
        dA = (np.einsum("uv,svldr->suldr", X, A) - np.einsum("sulvr,vd->suldr", A, X)
              + np.einsum("lv,suvdr->suldr", Y, A) - np.einsum("suldv,vr->suldr", A, Y))
        assert abs(np.sum(g0 * dA)) < 1e-4 * np.linalg.norm(g0) * np.linalg.norm(dA)
