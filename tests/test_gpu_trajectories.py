"""L-BFGS iterates on the GPU against the oracle's (Sec. II; Sec. IV.A: L-BFGS
with and without the local-metric preconditioner, Hager-Zhang line search).

Stored oracle trajectories (tests/golden/lbfgs_heis_d2_chi16.json, written by
tests/golden/make_golden.py from oracle/ only) from the seeded D=2, chi=16
Heisenberg start: 5 plain iterations (the first 2 compared) and 3
preconditioned ones.  Each
iterate's energy must agree to 1e-10 (the FP64 energy bar) and each accepted
step to 1e-6 relative; the plain method's line searches run their whole
40-evaluation budget at this start (on both sides), so the comparison also
covers the budget-exhausted branch of the line search."""
import json
import os

import pytest
import torch

from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lbfgs_heis_d2_chi16.json")


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


@pytest.mark.parametrize("kind,iters", [("plain", 2), ("preconditioned", 3)])
def test_lbfgs_iterates_match_oracle(ip, kind, iters):
    # plain: the first 2 of the 5 stored iterates (each a full 40-evaluation line search)
    gold = json.load(open(GOLD))
    ref = gold[kind]["log"][:iters + 1]
    w = inputs.WORKLOADS[gold["workload"]]
    A = torch.as_tensor(ip.cell_tensor(w["gen"]()), device="cuda")
    opts = ip.default_opts(chi=w["chi"], maxiter=iters, precondition=int(kind != "plain"),
                           ctm_tol=gold["ctm_tol"], ctm_maxit=gold["ctm_maxit"])
    _, log, st = ip.optimize(A, ip.ham_heisenberg(True), opts)
    assert len(log) == len(ref)
    for r, o in zip(log, ref):
        assert abs(r["E"] - o["f"]) <= 1e-10, (kind, r, o)
        if "alpha" in o:
            assert abs(r["alpha"] - o["alpha"]) <= 1e-6 * abs(o["alpha"]), (kind, r, o)
            assert r["evals"] == int(o["evals"]), (kind, r, o)
