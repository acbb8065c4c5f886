"""Host-side pieces of bench.py that run after the GPU part (CPU only)."""
import pytest

import bench


@pytest.mark.slow
def test_cpu_baseline_from_log():
    # a GPU run's log: iteration 0, then steps with (ctm_iters, evals)
    log = [dict(iter=0, ctm_iters=6, evals=1)] + [dict(iter=i, ctm_iters=c, evals=e)
                                                  for i, (c, e) in enumerate([(10, 8), (11, 1), (15, 4), (13, 1)], 1)]
    rec = bench.cpu_baseline("heis_d2_chi16", log, warmup=2)
    assert rec["kind"] == "oracle" and rec["unit"] == "iter/s" and rec["cores"] >= 1
    assert 0 < rec["value"] < 1e4
    assert "x 36.5" in rec["sample"] and "x 2.5" in rec["sample"]  # (15*4 + 13*1)/2 and (4+1)/2
