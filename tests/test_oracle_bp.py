"""Pins of the oracle's mean-field (chi = 1, belief-propagation) metric
preconditioner (Sec. III.B, App. A)."""
import numpy as np
import pytest

from oracle import bp


def _rand(rng, *shape):
    a = rng.uniform(-1.0, 1.0, shape)
    return a / np.abs(a).max()


def _dominant_left(E):
    """Dominant left eigenvector of E (vector over (l, L)) as a unit-trace matrix."""
    w, v = np.linalg.eig(E.T)
    k = int(np.argmax(np.abs(w)))
    x = v[:, k]
    x = x / x[np.argmax(np.abs(x))]
    assert np.max(np.abs(x.imag)) < 1e-10
    D = int(round(np.sqrt(E.shape[0])))
    X = x.real.reshape(D, D)
    return X / np.trace(X)


def _transfer(a):
    """E[(l, L), (r, R)] = sum_p a[p, l, r] a[p, L, R]."""
    D = a.shape[1]
    return np.einsum("plr,pLR->lLrR", a, a).reshape(D * D, D * D)


def test_product_state_closed_form():
    # D = 1: every message is [[1]], N = 1/|A|^2, P^-1 g = g / (1/|A|^2 + delta)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 1, 1, 1, 1))
    g = rng.normal(size=A.shape)
    delta = 0.37
    out, it, ch = bp.bp_precondition([[A]], [[g]], delta)
    expect = g / (1.0 / np.sum(A * A) + delta)
    assert np.max(np.abs(out[0][0] - expect)) < 1e-14


def test_mps_limit_messages_are_transfer_matrix_eigenvectors():
    # only u = d = 0 components: the vertical messages are e0 e0^T and the
    # horizontal sweep is the power method of the MPS transfer matrix
    rng = np.random.default_rng(5)
    D = 3
    A = np.zeros((2, D, D, D, D))
    A[:, 0, :, 0, :] = _rand(rng, 2, D, D)
    msgs, it, ch = bp.bp_messages([[A]], tol=1e-14, maxit=5000)
    assert ch <= 1e-14
    a = A[:, 0, :, 0, :]
    E = _transfer(a)                                    # (l,L) -> (r,R)
    right = _dominant_left(E)                           # sent to the right
    left = _dominant_left(np.einsum("plr,pLR->rRlL", a, a).reshape(D * D, D * D))
    assert np.max(np.abs(msgs[(0, 0, "r")] - right)) < 1e-10
    assert np.max(np.abs(msgs[(0, 0, "l")] - left)) < 1e-10
    e0 = np.zeros((D, D))
    e0[0, 0] = 1.0
    assert np.max(np.abs(msgs[(0, 0, "u")] - e0)) < 1e-14
    assert np.max(np.abs(msgs[(0, 0, "d")] - e0)) < 1e-14


def _mps_cell(rng, n, D, vertical):
    """n tensors with only the u = d = 0 (horizontal chain) or l = r = 0
    (vertical chain) components nonzero; returns (tensors, their transfer matrices)."""
    ts, Es = [], []
    for _ in range(n):
        A = np.zeros((2, D, D, D, D))
        if vertical:
            A[:, :, 0, :, 0] = _rand(rng, 2, D, D)      # a[p, u, d]
            Es.append(_transfer(A[:, :, 0, :, 0]))      # (u,U) -> (d,D)
        else:
            A[:, 0, :, 0, :] = _rand(rng, 2, D, D)      # a[p, l, r]
            Es.append(_transfer(A[:, 0, :, 0, :]))      # (l,L) -> (r,R)
        ts.append(A)
    return ts, Es


def test_three_column_cell_neighbour_offsets():
    # Lx = 3 in the MPS limit: x grows to the right, so the message site 2
    # sends right arrives at site 0 and is the dominant left eigenvector of
    # E_0 E_1 E_2; the one site 0 sends right, of E_1 E_2 E_0
    rng = np.random.default_rng(7)
    ts, (E0, E1, E2) = _mps_cell(rng, 3, 2, vertical=False)
    msgs, it, ch = bp.bp_messages([[t] for t in ts], tol=1e-14, maxit=5000)
    assert np.max(np.abs(msgs[(2, 0, "r")] - _dominant_left(E0 @ E1 @ E2))) < 1e-10
    assert np.max(np.abs(msgs[(0, 0, "r")] - _dominant_left(E1 @ E2 @ E0))) < 1e-10
    # leftward messages: out^l_x = E_x out^l_{x+1}, a dominant right eigenvector
    assert np.max(np.abs(msgs[(0, 0, "l")] - _dominant_left((E0 @ E1 @ E2).T))) < 1e-10


def test_three_row_cell_neighbour_offsets():
    # Ly = 3 with trivial horizontal legs: y grows downwards, so the message
    # site (0, 2) sends down arrives at (0, 0) from above
    rng = np.random.default_rng(8)
    ts, (F0, F1, F2) = _mps_cell(rng, 3, 2, vertical=True)
    msgs, it, ch = bp.bp_messages([ts], tol=1e-14, maxit=5000)
    assert np.max(np.abs(msgs[(0, 2, "d")] - _dominant_left(F0 @ F1 @ F2))) < 1e-10
    assert np.max(np.abs(msgs[(0, 0, "d")] - _dominant_left(F1 @ F2 @ F0))) < 1e-10
    # upward messages: out^u_y = F_y out^u_{y+1}, a dominant right eigenvector
    assert np.max(np.abs(msgs[(0, 0, "u")] - _dominant_left((F0 @ F1 @ F2).T))) < 1e-10


@pytest.mark.parametrize("Lx,Ly,d,D", [(1, 1, 2, 2), (1, 1, 2, 3), (2, 1, 4, 2), (2, 2, 2, 2)])
def test_eigenbasis_solve_equals_dense_kronecker_solve(Lx, Ly, d, D):
    rng = np.random.default_rng(11 + D + Lx)
    cell = [[_rand(rng, d, D, D, D, D) for _ in range(Ly)] for _ in range(Lx)]
    g = [[rng.normal(size=(d, D, D, D, D)) for _ in range(Ly)] for _ in range(Lx)]
    delta = 1e-3
    out, it, ch = bp.bp_precondition(cell, g, delta)
    assert ch <= 1e-12
    msgs, _, _ = bp.bp_messages(cell)
    for x in range(Lx):
        for y in range(Ly):
            ins, c = bp.bp_metric_factors(cell, msgs, x, y)
            M = np.kron(np.kron(np.kron(ins["u"], ins["l"]), ins["d"]), ins["r"])
            a = cell[x][y].reshape(d, -1)
            assert abs(c * np.einsum("si,ij,sj->", a, M, a) - 1.0) < 1e-12
            N = np.kron(np.eye(d), c * M) + delta * np.eye(d * D ** 4)
            ref = np.linalg.solve(N, g[x][y].ravel())
            assert np.max(np.abs(out[x][y].ravel() - ref)) < 1e-10 * np.max(np.abs(ref))


def test_messages_are_symmetric_psd_fixed_points():
    rng = np.random.default_rng(13)
    cell = [[_rand(rng, 2, 3, 3, 3, 3)] for _ in range(2)]
    msgs, it, ch = bp.bp_messages(cell)
    assert ch <= 1e-12
    for m in msgs.values():
        assert np.max(np.abs(m - m.T)) == 0.0
        assert abs(np.trace(m) - 1.0) < 1e-14
        assert np.linalg.eigvalsh(m)[0] > -1e-14
    # one more sweep leaves them unchanged
    for x in range(2):
        ins = bp.incoming(msgs, 2, 1, x, 0)
        for lam in bp.LEGS:
            new = bp._normalise(bp._outgoing(cell[x][0], ins, lam))
            assert np.max(np.abs(new - msgs[(x, 0, lam)])) < 1e-11


def test_c4v_symmetric_tensor_sends_equal_messages_on_all_legs():
    # the eight symmetries of the square map the four legs onto each other, so a
    # C4v-symmetric tensor's four outgoing messages coincide
    from oracle import c4v

    rng = np.random.default_rng(21)
    A = c4v.c4v_project(rng.uniform(-1, 1, (2, 3, 3, 3, 3))).numpy()
    msgs, it, ch = bp.bp_messages([[A]])
    assert ch <= 1e-12
    for lam in ("l", "d", "r"):
        assert np.max(np.abs(msgs[(0, 0, lam)] - msgs[(0, 0, "u")])) < 1e-12
