"""Host-side pieces of bench.py (CPU only): the algorithmic FLOP model of a
CTMRG iteration and the oracle leg that times whole passes."""
import pytest

import bench
from paper_2511_09546_gb300 import inputs


def test_ctmrg_flop_model_counts_each_step():
    # D=4, chi=64, 1x1: 4 moves x (4 corners + 3 (chi D^2)^3 + absorption), 2 flop per MAC
    w = inputs.WORKLOADS["heis_d4_chi64"]
    chi, D, d, n = 64, 4, 2, 64 * 16
    corner = chi ** 3 * D ** 2 + chi ** 3 * D ** 4 + 2 * chi ** 2 * D ** 6 * d
    absorb = 2 * chi ** 3 * D ** 4 + 2 * chi ** 2 * D ** 6 * d + 3 * chi ** 3 * D ** 2
    assert bench.ctmrg_flops_per_iteration(w) == 2.0 * 4 * (4 * corner + 3 * n ** 3 + absorb)
    # a 2x2 cell has four times the projector pairs
    w2 = dict(w, Lx=2, Ly=2)
    assert bench.ctmrg_flops_per_iteration(w2) == 4 * bench.ctmrg_flops_per_iteration(w)


@pytest.mark.slow
def test_oracle_passes_time_whole_passes():
    times, cores = bench.oracle_passes("heis_d2_chi16", 2)
    assert len(times) == 2 and all(t > 0 for t in times) and cores >= 1


def test_perturbed_cells_are_seeded_and_close():
    c0 = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    a = inputs.perturbed_cells(c0, 3, 1e-3, 5)
    b = inputs.perturbed_cells(c0, 3, 1e-3, 5)
    for ca, cb in zip(a, b):
        assert (ca[0][0] == cb[0][0]).all()
        assert abs(ca[0][0] - c0[0][0]).max() <= 1e-3
    assert not (a[0][0][0] == a[1][0][0]).all()
