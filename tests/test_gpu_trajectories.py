"""L-BFGS iterates on the GPU against the oracle's (Sec. II; Sec. IV.A: L-BFGS
with and without the local-metric preconditioner, Hager-Zhang line search).

Stored oracle trajectories (tests/golden/lbfgs_heis_d2_chi16.json, written by
tests/golden/make_golden.py from oracle/ only), D=2, chi=16 Heisenberg: 5 plain
iterations from the seeded Neel-like start (the first 4 compared: the fifth
line search runs its whole 40-evaluation budget) and 3 preconditioned ones from
the seeded random start.  Each iterate's energy must agree to 1e-10 (the FP64
energy bar), each accepted step to 1e-6 relative, and the line searches must
take the same number of evaluations."""
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


@pytest.mark.parametrize("kind,iters", [("plain", 4), ("preconditioned", 3)])
def test_lbfgs_iterates_match_oracle(ip, kind, iters):
    gold = json.load(open(GOLD))
    ref = gold[kind]["log"][:iters + 1]
    w = inputs.WORKLOADS[gold[kind]["workload"]]
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
