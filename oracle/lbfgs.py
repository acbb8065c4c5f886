"""Plain and preconditioned L-BFGS with the Hager-Zhang line search
(oracle, test infrastructure).

Sec. II: with a preconditioner P the search direction uses P^-1 g; in a
quasi-Newton method it has to enter the inverse-Hessian approximation
consistently.  Sec. IV.A: L-BFGS with history m = 200 and the Hager-Zhang
line search.  Sec. III.B: delta = |g|^2 (or |E_{i+1} - E_i|).

Readings (paper silent):
  * two-loop recursion (Nocedal & Wright, Algorithm 7.4) whose initial
    inverse Hessian is gamma_k P_k^-1 with gamma_k = s^T y / (y^T P_k^-1 y)
    (plain case P = I: gamma_k = s^T y / y^T y); gamma = 1 without history;
  * the pair (s, y) is stored only if s^T y > 1e-16 |s| |y|;
  * first trial step: alpha = 1 once a pair is stored or when a
    preconditioner is used (P^-1 g is then a displacement in the units of x,
    Eq. pregrad), otherwise psi0 |x|_inf / |d|_inf with psi0 = 0.01 (Hager &
    Zhang's I0);
  * line search: Hager & Zhang (2006), bracket / update / secant^2 with the
    published defaults delta = 0.1, sigma = 0.9, epsilon = 1e-6, theta = 0.5,
    gamma = 0.66, rho = 5; the first evaluated trial point satisfying the
    Wolfe or the approximate Wolfe conditions is accepted;
  * delta_k = max(|g_k|^2, 1e-12) (default) or |E_k - E_{k-1}| with
    delta_0 = |g_0|^2;
  * a trial point whose energy evaluation fails (CTMRG or the adjoint solve
    not converged) is treated as lying beyond the minimiser (value and slope
    +inf), so the line search shrinks the step.

Parity pins: on the quadratic of Sec. II with P = A a preconditioned
gradient step of length one reaches x*; L-BFGS terminates on an
n-dimensional quadratic (tests/test_oracle_lbfgs.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class HZParams:
    delta: float = 0.1
    sigma: float = 0.9
    epsilon: float = 1e-6
    theta: float = 0.5
    gamma: float = 0.66
    rho: float = 5.0
    max_evals: int = 40


class _Found(Exception):
    def __init__(self, a):
        self.a = a


def hz_linesearch(phi, phi0, dphi0, c, p: HZParams = HZParams()):
    """phi(a) -> (value, slope, payload).  Returns (a, value, slope, payload, evals)."""
    fmax = phi0 + p.epsilon * abs(phi0)
    cache = {0.0: (phi0, dphi0, None)}

    def ok(a, fa, da):
        t1 = (fa - phi0 <= p.delta * a * dphi0) and (da >= p.sigma * dphi0)
        t2 = ((2.0 * p.delta - 1.0) * dphi0 >= da >= p.sigma * dphi0) and (fa <= fmax)
        return t1 or t2

    repeats = [0]

    def ev(a):
        if a not in cache:
            repeats[0] = 0
            if len(cache) > p.max_evals:
                raise _Found(None)
            cache[a] = phi(a)
            if ok(a, cache[a][0], cache[a][1]):
                raise _Found(a)
        else:
            # an interval shrunk to adjacent doubles keeps asking for its own
            # ends: end the search as when the budget is spent
            repeats[0] += 1
            if repeats[0] > 50:
                raise _Found(None)
        return cache[a][0], cache[a][1]

    def bisect(a, b):
        while True:
            d = (1.0 - p.theta) * a + p.theta * b
            fd, dd = ev(d)
            if dd >= 0:
                return a, d
            if fd <= fmax:
                a = d
            else:
                b = d

    def update(a, b, c):
        if not (a < c < b):
            return a, b
        fc, dc = ev(c)
        if dc >= 0:
            return a, c
        if fc <= fmax:
            return c, b
        return bisect(a, c)

    def secant(a, b):
        da, db = cache[a][1], cache[b][1]
        if db == da or not (np.isfinite(da) and np.isfinite(db)):
            return 0.5 * (a + b)
        return (a * db - b * da) / (db - da)

    def secant2(a, b):
        c = secant(a, b)
        A, B = update(a, b, c)
        if c == B:
            cb = secant(b, B)
        elif c == A:
            cb = secant(a, A)
        else:
            return A, B
        return update(A, B, cb)

    def bracket(c):
        good = 0.0
        while True:
            fc, dc = ev(c)
            if dc >= 0:
                return good, c
            if fc > fmax:
                return bisect(0.0, c)
            good = c
            c = p.rho * c

    try:
        a, b = bracket(c)
        while True:
            A, B = secant2(a, b)
            if B - A > p.gamma * (b - a):
                A, B = update(A, B, 0.5 * (A + B))
            a, b = A, B
    except _Found as fnd:
        a = fnd.a
    if a is None:  # evaluation budget spent: best point seen
        a = min((k for k in cache if k > 0), key=lambda k: cache[k][0])
    fa, da, pay = cache[a]
    return a, fa, da, pay, len(cache) - 1


def two_loop(hist, g, H0):
    """H g for the L-BFGS inverse Hessian built from hist = [(s, y, 1/s^T y)]
    (oldest first) over the initial matrix gamma H0, where
    gamma = s^T y / (y^T H0 y) of the newest pair (1 without history)."""
    q = g.copy()
    alphas = []
    for s, y, rh in reversed(hist):
        a = rh * (s @ q)
        q = q - a * y
        alphas.append(a)
    if hist:
        s, y, _ = hist[-1]
        gamma = (s @ y) / (y @ H0(y))
    else:
        gamma = 1.0
    r = gamma * H0(q)
    for (s, y, rh), a in zip(hist, reversed(alphas)):
        b = rh * (y @ r)
        r = r + s * (a - b)
    return r


def lbfgs(fg, x0, *, precond=None, m=200, maxiter=100, gtol=1e-10, delta_rule="grad2",
          callback=None, ls=HZParams(), stop=None):
    """Minimise f.  fg(x, state) -> (f, g, state); precond(state, v, delta) -> P^-1 v.
    stop(k, f, g) -> bool ends the run early.  Returns (x, f, g, history)."""
    x = np.array(x0, dtype=np.float64)
    f, g, st = fg(x, None)
    hist = []
    log = [dict(k=0, f=f, gnorm=float(np.linalg.norm(g)), evals=1)]
    f_prev = None
    for k in range(maxiter):
        if np.linalg.norm(g) < gtol or (stop is not None and stop(k, f, g)):
            break
        if delta_rule == "grad2" or f_prev is None:
            delta = max(float(g @ g), 1e-12)
        else:
            delta = max(abs(f - f_prev), 1e-12)
        if precond is not None:
            H0 = lambda v: precond(st, v, delta)
        else:
            H0 = lambda v: v
        d = -two_loop(hist, g, H0)
        if d @ g >= 0:  # not a descent direction: restart from the (preconditioned) gradient
            hist.clear()
            d = -(precond(st, g, delta) if precond is not None else g)
        if hist or precond is not None:
            c = 1.0
        else:
            c = 0.01 * np.max(np.abs(x)) / np.max(np.abs(d))

        def phi(a):
            fa, ga, sa = fg(x + a * d, st)
            if not np.isfinite(fa):   # failed evaluation: treat as beyond the minimiser
                return np.inf, np.inf, (ga, sa)
            return fa, float(ga @ d), (ga, sa)

        a, fa, _, pay, nev = hz_linesearch(phi, f, float(g @ d), c, ls)
        if not np.isfinite(fa):
            log.append(dict(k=k + 1, f=fa, failed=True))
            break
        g_new, st_new = pay
        s = a * d
        y = g_new - g
        sy = float(s @ y)
        if sy > 1e-16 * np.linalg.norm(s) * np.linalg.norm(y):
            hist.append((s, y, 1.0 / sy))
            if len(hist) > m:
                hist.pop(0)
        x = x + s
        f_prev, f, g, st = f, fa, g_new, st_new
        log.append(dict(k=k + 1, f=f, gnorm=float(np.linalg.norm(g)), alpha=a, evals=nev, delta=delta))
        if callback is not None:
            callback(log[-1])
    return x, f, g, log
