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


def test_hbm_kernel_table_uses_data_movement_classes_only():
    prof = {"permute": {"count": 10, "ms": 2.0, "flops": 0.0, "bytes": 4e9},
            "dgemm": {"count": 5, "ms": 1.0, "flops": 1e9, "bytes": 1e8},
            "jacobi_pair": {"count": 3, "ms": 1.0, "flops": 0.0, "bytes": 0.0}}
    t = bench.hbm_kernels(prof, 8000.0)
    assert list(t) == ["permute"]
    assert t["permute"]["achieved_gbs"] == pytest.approx(2000.0)
    assert t["permute"]["frac"] == pytest.approx(0.25)
    assert t["permute"]["gb_per_launch"] == pytest.approx(0.4)


def test_roofline_picks_the_dominant_class():
    prof = {"permute": {"count": 10, "ms": 2.0, "flops": 0.0, "bytes": 4e9},
            "dgemm": {"count": 5, "ms": 6.0, "flops": 3e9, "bytes": 1e8}}
    r = bench.roofline(prof, {"fp64_tflops": 1.0})
    assert r["kernel"] == "dgemm" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(0.5) and r["frac"] == pytest.approx(0.5)
    assert r["share"] == pytest.approx(0.75)


def test_roofline_of_the_jacobi_class_is_an_fp64_rate_with_its_note():
    prof = {"jacobi_pair": {"count": 100, "ms": 8.0, "flops": 4e9, "bytes": 0.0},
            "dgemm": {"count": 5, "ms": 6.0, "flops": 3e9, "bytes": 1e8}}
    r = bench.roofline(prof, {"fp64_tflops": 1.1})
    assert r["kernel"] == "jacobi_pair" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(0.5) and r["frac"] == pytest.approx(0.5 / 1.1)
    assert "lower bound" in r["note"] and r["ncu_sample"]["dram_bytes"] > 0
