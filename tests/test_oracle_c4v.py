"""Pins of the oracle's C4v-symmetric CTMRG and unrolled gradient (Sec. IV.A:
C4v-symmetric one-tensor iPEPS, CTMRG with a fixed number of steps, gradient
through the last steps)."""
import numpy as np
import pytest
import torch

from oracle import c4v
from oracle import ctmrg as OC
from oracle import energy as OE
from oracle import exact
from oracle import models as OM

HAM = OM.heisenberg(True)


def _sym_tensor(seed, d=2, D=2):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (d, D, D, D, D))


def test_symmetry_group_and_projection():
    g = c4v.symmetries()
    assert len(set(g)) == 8
    # closed under composition
    for p in g:
        for q in g:
            assert tuple(p[i] for i in q) in g
    A = c4v.c4v_project(_sym_tensor(4, D=3))
    assert float((c4v.c4v_project(A) - A).abs().max()) < 1e-15
    for p in g:
        assert float((A.permute(*p) - A).abs().max()) < 1e-15
    # an orthogonal projection does not increase the norm
    B = torch.as_tensor(_sym_tensor(5, D=3))
    assert float(torch.linalg.norm(c4v.c4v_project(B))) <= float(torch.linalg.norm(B)) + 1e-12


@pytest.mark.parametrize("chi", [8, 16])
def test_energy_equals_general_ctmrg(chi):
    # for a C4v-symmetric tensor the symmetric CTMRG (enlarged-corner
    # eigenvectors) and the general one (four-corner SVD projectors) reach the
    # same environment: the energies agree to rounding
    A = c4v.c4v_project(_sym_tensor(0))
    with torch.no_grad():
        E = float(c4v.energy(A, chi, HAM, n=150, N=0))
    cell = [[A.numpy()]]
    env, it, err = OC.ctmrg(cell, chi, tol=1e-12, maxit=1000)
    Eg = float(OE.energy(1, 1, OC.as_torch_cell(cell), env, HAM))
    assert err < 1e-11
    assert abs(E - Eg) < 1e-12


def test_ising_peps_onsager():
    # the Ising PEPS is C4v symmetric; <sz sz> on the two bonds per site is Onsager's
    K = 0.3
    A = torch.as_tensor(exact.ising_peps(K))
    assert float((c4v.c4v_project(A) - A).abs().max()) < 1e-15
    with torch.no_grad():
        E = float(c4v.energy(A, 16, OM.sigma_z_bond(), n=200, N=0))
    assert abs(E - 2.0 * exact.onsager_nn(K)) < 1e-10


def test_product_state_closed_form():
    # D = 1 real spinor in the rotated frame: E = -1/2 per site
    A = torch.as_tensor(np.array([0.6, 0.8]).reshape(2, 1, 1, 1, 1))
    with torch.no_grad():
        E = float(c4v.energy(A, 1, HAM, n=5, N=0))
    assert abs(E + 0.5) < 1e-14


def test_unrolled_gradient_equals_central_differences_of_the_same_function():
    B = _sym_tensor(1)
    chi, n, N = 8, 3, 20
    E, g = c4v.energy_and_gradient(B, chi, HAM, n=n, N=N)

    def f(Bv):
        with torch.no_grad():
            return float(c4v.energy(c4v.c4v_project(torch.as_tensor(Bv)), chi, HAM, n=n, N=N))

    assert abs(f(B) - E) < 1e-14
    rng = np.random.default_rng(2)
    h = 1e-6
    for i in rng.choice(B.size, 8, replace=False):
        Bp, Bm = B.copy().ravel(), B.copy().ravel()
        Bp[i] += h
        Bm[i] -= h
        fd = (f(Bp.reshape(B.shape)) - f(Bm.reshape(B.shape))) / (2 * h)
        assert abs(g.ravel()[i] - fd) < 1e-8 * max(1.0, abs(fd)), (i, g.ravel()[i], fd)


def test_unrolled_gradient_reaches_the_converged_derivative():
    # with many undifferentiated steps and N differentiated ones the gradient is
    # the derivative of the converged energy: compare along C4v-symmetric
    # directions with central differences of fully converged general-CTMRG energies
    B = _sym_tensor(0)
    A = c4v.c4v_project(B).numpy()
    chi, h = 8, 1e-5
    _, g40 = c4v.energy_and_gradient(B, chi, HAM, n=60, N=40)
    _, g80 = c4v.energy_and_gradient(B, chi, HAM, n=60, N=80)
    assert np.linalg.norm(g80 - g40) < 1e-9 * np.linalg.norm(g80)
    rng = np.random.default_rng(3)

    def Egen(Av):
        env, it, err = OC.ctmrg([[Av]], chi, tol=1e-13, maxit=5000)
        assert err < 1e-12
        return float(OE.energy(1, 1, OC.as_torch_cell([[Av]]), env, HAM))

    for _ in range(2):
        dlt = c4v.c4v_project(rng.normal(size=B.shape)).numpy()
        fd = (Egen(A + h * dlt) - Egen(A - h * dlt)) / (2 * h)
        assert abs(np.sum(g80 * dlt) - fd) < 1e-7 * abs(fd), (np.sum(g80 * dlt), fd)


def test_fixed_point_gradient_at_a_c4v_tensor_needs_the_orthogonal_gauge():
    # a C4v-symmetric tensor gives exactly degenerate pairs in the general
    # CTMRG's projector spectra; the sign gauge alone leaves the environment
    # off its elementwise fixed point, the orthogonal refinement restores it,
    # and the implicit gradient then equals the unrolled C4v gradient along C4v
    # directions and central differences along a non-symmetric one
    from oracle import gradient as OG

    B = _sym_tensor(0)
    A = c4v.c4v_project(B).numpy()
    chi = 8
    env, gauge, it, err, res = OC.fixed_point([[A]], chi, tol=1e-11, maxit=3000)
    assert next(iter(gauge.values())).ndim == 2 and res < 1e-10
    with torch.no_grad():
        e1 = OC.ctmrg_step(1, 1, OC.as_torch_cell([[A]]), env, chi)
    signs = OC.solve_signs(1, 1, env, e1)
    assert OC.env_diff(1, 1, env, OC.apply_signs(1, 1, e1, signs)) > 1e-6
    E, g, info = OG.energy_and_gradient([[A]], HAM, chi, tol=1e-11, maxit=3000, return_info=True)
    assert info["converged"] and info["fixed_point_residual"] < 1e-10
    _, gu = c4v.energy_and_gradient(B, chi, HAM, n=60, N=80)
    rng = np.random.default_rng(3)
    dlt = c4v.c4v_project(rng.normal(size=B.shape)).numpy()
    assert abs(np.sum(g[0][0] * dlt) - np.sum(gu * dlt)) < 1e-9 * abs(np.sum(gu * dlt))
    dn = np.random.default_rng(4).normal(size=B.shape)
    h = 1e-5

    def Egen(Av):
        e, _, er = OC.ctmrg([[Av]], chi, tol=1e-13, maxit=5000)
        assert er < 1e-12
        return float(OE.energy(1, 1, OC.as_torch_cell([[Av]]), e, HAM))

    fd = (Egen(A + h * dn) - Egen(A - h * dn)) / (2 * h)
    assert abs(np.sum(g[0][0] * dn) - fd) < 1e-6 * abs(fd)


def test_random_tensor_keeps_the_sign_gauge():
    rng = np.random.default_rng(9)
    A = rng.uniform(-1, 1, (2, 2, 2, 2, 2))
    env, gauge, it, err, res = OC.fixed_point([[A]], 8, tol=1e-11, maxit=3000)
    assert next(iter(gauge.values())).ndim == 1 and res < 1e-8


@pytest.mark.parametrize("precond", [True, "bp"])
def test_preconditioned_c4v_optimisation_reaches_table_one_energy(precond):
    # end to end: C4v CTMRG (3 + 20 steps), unrolled gradient, local-metric (or
    # mean-field) preconditioned L-BFGS from a seeded random C4v tensor reach
    # the D=2, chi=32 reference energy the paper prints (Table I, seven digits)
    import json
    import os

    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1_heisenberg_eref.json")))
    row = gold["rows"][0]
    D, chi = row["D"], row["chi"]
    rng = np.random.default_rng(0)
    B0 = c4v.c4v_project(rng.uniform(-1, 1, (2, D, D, D, D))).numpy()
    B0 /= np.abs(B0).max()
    _, E, log = c4v.optimize(B0, chi, HAM, precond=precond, maxiter=40,
                             stop=lambda k, f, g: np.linalg.norm(g) < 1e-8)
    assert abs(E - row["E_ref"]) < 1e-7, E


def test_orthogonal_gauge_on_a_two_by_two_cell():
    # four copies of one C4v tensor: the refined gauge makes the 2x2 environment
    # an elementwise fixed point too, and every site's gradient is a quarter of
    # the one-site gradient (same state, four tensors)
    from oracle import gradient as OG

    ham = OM.heisenberg(False)
    A = c4v.c4v_project(_sym_tensor(0)).numpy()
    cell = [[A, A], [A, A]]
    E, g, info = OG.energy_and_gradient(cell, ham, 8, tol=1e-11, maxit=3000, return_info=True)
    assert info["converged"] and info["fixed_point_residual"] < 1e-10
    E1, g1 = OG.energy_and_gradient([[A]], ham, 8, tol=1e-11, maxit=3000)
    assert abs(E - E1) < 1e-12
    for x in range(2):
        for y in range(2):
            assert np.max(np.abs(g[x][y] - g1[0][0] / 4)) < 1e-12
