"""Pins of the oracle's L-BFGS and Hager-Zhang line search (Sec. II, Eq. pregrad; Sec. IV.A)."""
import numpy as np

from oracle.lbfgs import HZParams, hz_linesearch, lbfgs, two_loop


def _quadratic(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.logspace(0, np.log10(cond), n)) @ Q.T
    b = rng.standard_normal(n)
    return A, b


def test_preconditioned_step_reaches_minimum():
    # Eq. (eq:pregrad): with P = A the preconditioned gradient is x - x*, so one
    # preconditioned gradient step of unit length lands on x* = A^-1 b
    A, b = _quadratic(20, 1e4, 0)
    xs = np.linalg.solve(A, b)
    fg = lambda x, st: (0.5 * x @ A @ x - b @ x, A @ x - b, None)
    pc = lambda st, v, delta: np.linalg.solve(A, v)
    x0 = np.ones(20)
    x, f, g, log = lbfgs(fg, x0, precond=pc, maxiter=1)
    assert abs(log[1]["alpha"] - 1.0) < 1e-8
    assert np.linalg.norm(x - xs) < 1e-8 * np.linalg.norm(xs)


def test_two_loop_equals_explicit_bfgs():
    # Nocedal & Wright: the two-loop recursion applies the BFGS inverse Hessian
    # H <- V^T H V + rho s s^T, V = I - rho y s^T, started from gamma H0
    n = 9
    A, _ = _quadratic(n, 50.0, 4)
    rng = np.random.default_rng(7)
    H0m = np.diag(rng.uniform(0.5, 2.0, n))
    hist = []
    for _ in range(5):
        s = rng.standard_normal(n)
        y = A @ s
        hist.append((s, y, 1.0 / (s @ y)))
    s, y, _ = hist[-1]
    H = (s @ y) / (y @ H0m @ y) * H0m
    for s, y, rho in hist:
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    g = rng.standard_normal(n)
    assert np.linalg.norm(two_loop(hist, g, lambda v: H0m @ v) - H @ g) < 1e-12 * np.linalg.norm(H @ g)


def test_lbfgs_converges_on_quadratic():
    n = 12
    A, b = _quadratic(n, 1e3, 1)
    fg = lambda x, st: (0.5 * x @ A @ x - b @ x, A @ x - b, None)
    x, f, g, log = lbfgs(fg, np.zeros(n) + 0.1, maxiter=4 * n, gtol=1e-9)
    assert np.linalg.norm(g) < 1e-8 * np.linalg.norm(b)
    assert abs(f + 0.5 * b @ np.linalg.solve(A, b)) < 1e-12


def test_plain_gd_on_illconditioned_is_slow_but_preconditioned_is_not():
    # Sec. II: the condition number governs steepest descent; P = A removes it
    A, b = _quadratic(30, 1e5, 2)
    fg = lambda x, st: (0.5 * x @ A @ x - b @ x, A @ x - b, None)
    _, _, g_plain, _ = lbfgs(fg, np.zeros(30) + 1, m=0, maxiter=5)
    _, _, g_pre, _ = lbfgs(fg, np.zeros(30) + 1, m=0, maxiter=5,
                            precond=lambda st, v, d: np.linalg.solve(A, v))
    assert np.linalg.norm(g_pre) < 1e-6 * np.linalg.norm(g_plain)


def test_hz_wolfe():
    p = HZParams()
    phi = lambda a: ((a - 3.0) ** 2 + 0.1 * np.sin(5 * a), 2 * (a - 3.0) + 0.5 * np.cos(5 * a), None)
    f0, d0, _ = phi(0.0)
    a, fa, da, _, nev = hz_linesearch(phi, f0, d0, 0.1, p)
    wolfe = (fa - f0 <= p.delta * a * d0) and (da >= p.sigma * d0)
    approx = ((2 * p.delta - 1) * d0 >= da >= p.sigma * d0) and fa <= f0 + p.epsilon * abs(f0)
    assert wolfe or approx
    assert nev < 20
