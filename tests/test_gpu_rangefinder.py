"""The randomised range-finder cold start of the projector SVD (four-corner
product larger than 1024 x 1024) against stored oracle values at the FP64 bar.

Case: Heisenberg 1x1 (rotated), random D=5 tensor (uniform seed 3), chi=44, so
the four-corner product is 1100 x 1100 and its cut is resolvable (relative gap
about 1.8e-8).  tests/golden/rangefinder_d5_chi44.json holds the oracle's E and
gradient (written by tests/golden/make_golden.py from oracle/ only)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rangefinder_d5_chi44.json")


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


@pytest.mark.parametrize("prec", ["FP64", "FP64_TC"])
def test_range_finder_cold_start_at_fp64_bar(ip, prec):
    gold = json.load(open(GOLD))
    assert gold["chi"] * gold["D"] ** 2 > 1024 and gold["min_cut_gap"] > 1e-8
    cell = inputs.uniform_cell(1, 1, 2, gold["D"], gold["seed"])
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    env, it, err = ip.ctmrg(A, gold["chi"], tol=gold["ctm_tol"], maxit=400, prec=getattr(ip, prec))
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    assert abs(E - gold["E"]) <= 1e-10
    go = np.asarray(gold["grad"])
    gg = g.cpu().numpy().ravel()
    assert np.linalg.norm(gg - go) <= 1e-8 * np.linalg.norm(go)
