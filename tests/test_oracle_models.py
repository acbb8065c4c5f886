"""Pins of the model Hamiltonians (Eq. eq:H_heisenberg, Sec. IV.A spin flip; Sec. IV.B Kitaev)."""
import numpy as np

from oracle import models


def test_heisenberg_bond_spectrum():
    # S_i . S_j of two spins 1/2: singlet -3/4, triplet 1/4 (x3)
    for rot in (False, True):
        ev = np.sort(np.linalg.eigvalsh(models.heisenberg_bond(rot)))
        assert np.allclose(ev, [-0.75, 0.25, 0.25, 0.25], atol=1e-14)


def test_sublattice_rotation_is_conjugation():
    # U = i sigma_y = [[0, 1], [-1, 0]] on the second site
    U = np.array([[0.0, 1.0], [-1.0, 0.0]])
    K = np.kron(np.eye(2), U)
    assert np.allclose(K @ models.heisenberg_bond(False) @ K.T, models.heisenberg_bond(True), atol=1e-14)


def test_kitaev_terms():
    ham = models.kitaev_dimer(-1.0)
    px = np.array([[0, 1], [1, 0]]) / 2.0
    pz = np.array([[1, 0], [0, -1]]) / 2.0
    py_r = np.array([[0, -1], [1, 0]]) / 2.0   # S^y = i * py_r
    I2 = np.eye(2)
    # on-site z link inside the dimer
    assert np.allclose(ham["site"], -np.kron(pz, pz))
    # x link: b of the left dimer with a of the right dimer
    hx = -np.kron(np.kron(I2, px), np.kron(px, I2))
    assert np.allclose(ham["h"], hx)
    # y link: S^y S^y = (i)^2 py_r py_r = -py_r (x) py_r
    hy = -(-np.kron(np.kron(I2, py_r), np.kron(py_r, I2)))
    assert np.allclose(ham["v"], hy)
    for k in ("h", "v"):
        assert np.allclose(ham[k], ham[k].T)
        assert np.allclose(np.sort(np.unique(np.round(np.linalg.eigvalsh(ham[k]), 12))), [-0.25, 0.25])
