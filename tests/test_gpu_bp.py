"""Mean-field (chi = 1) metric preconditioner on the GPU against the oracle
(Sec. III.B: the local metric with environment bond dimension 1, from belief
propagation; App. A).  The preconditioned vector is unique (the eigenbases
of degenerate messages are not), so it is compared element by element; the
sweep counts of the message iteration must agree."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import bp as OB
from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lbfgs_bp_heis_d2_chi16.json")


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


def _cells(Lx, Ly, d, D, seed, kind="uniform"):
    rng = np.random.default_rng(seed)
    if kind == "mps":   # only u = d = 0 components: the vertical messages are rank one
        cell = []
        for _ in range(Lx):
            col = []
            for _ in range(Ly):
                A = np.zeros((d, D, D, D, D))
                A[:, 0, :, 0, :] = rng.uniform(-1, 1, (d, D, D))
                col.append(A)
            cell.append(col)
    else:
        cell = [[rng.uniform(-1, 1, (d, D, D, D, D)) for _ in range(Ly)] for _ in range(Lx)]
    g = [[rng.normal(size=(d, D, D, D, D)) for _ in range(Ly)] for _ in range(Lx)]
    return cell, g


CASES = [
    # (Lx, Ly, d, D, seed, kind, delta)
    (1, 1, 2, 2, 1, "uniform", 1e-3),
    (1, 1, 2, 3, 2, "uniform", 1e-2),
    (1, 1, 2, 5, 3, "uniform", 1e-4),
    (1, 1, 2, 8, 4, "uniform", 1e-3),
    (2, 1, 4, 2, 5, "uniform", 1e-3),     # Kitaev-shaped 1x2 cell (two sites per tensor)
    (2, 2, 2, 2, 6, "uniform", 1e-3),
    (3, 1, 2, 2, 7, "uniform", 1e-3),     # three columns: neighbour offsets along x
    (1, 3, 2, 3, 8, "uniform", 1e-3),     # three rows: offsets along y
    (1, 1, 3, 1, 9, "uniform", 0.37),     # D = 1 product state
    (1, 1, 2, 3, 10, "mps", 1e-3),        # rank-one vertical messages (degenerate eigenbases)
]


@pytest.mark.parametrize("Lx,Ly,d,D,seed,kind,delta", CASES)
def test_precondition_bp_matches_oracle(ip, Lx, Ly, d, D, seed, kind, delta):
    cell, g = _cells(Lx, Ly, d, D, seed, kind)
    ref, sweeps, change = OB.bp_precondition(cell, g, delta)
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    gd = torch.as_tensor(ip.cell_tensor(g), device="cuda")
    out, gs, gch = ip.precondition_bp(A, gd, delta)
    R = np.asarray(ip.cell_tensor(ref))
    err = np.max(np.abs(out.cpu().numpy() - R)) / np.max(np.abs(R))
    assert err <= 1e-9, (err, sweeps, gs)
    assert abs(gs - sweeps) <= 1, (gs, sweeps)
    assert gch <= 1e-12


def test_precondition_bp_delta_rule(ip):
    # delta < 0: delta = |g|^2 over the whole cell (Sec. III.B)
    cell, g = _cells(2, 1, 2, 3, 11)
    delta = float(sum(np.sum(x * x) for col in g for x in col))
    ref, _, _ = OB.bp_precondition(cell, g, delta)
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    gd = torch.as_tensor(ip.cell_tensor(g), device="cuda")
    out, _, _ = ip.precondition_bp(A, gd, -1.0)
    R = np.asarray(ip.cell_tensor(ref))
    assert np.max(np.abs(out.cpu().numpy() - R)) <= 1e-9 * np.max(np.abs(R))


def test_precondition_bp_sweep_limit_and_repeatability(ip):
    # bp_maxit ends the sweeps without an error; the same call gives the same bits
    cell, g = _cells(1, 1, 2, 4, 12)
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    gd = torch.as_tensor(ip.cell_tensor(g), device="cuda")
    out3, s3, c3 = ip.precondition_bp(A, gd, 1e-3, maxit=3)
    assert s3 == 3 and c3 > 1e-12
    ref3, rs, rc = OB.bp_precondition(cell, g, 1e-3, maxit=3)
    assert rs == 3 and abs(rc - c3) <= 1e-12
    R = np.asarray(ip.cell_tensor(ref3))
    assert np.max(np.abs(out3.cpu().numpy() - R)) <= 1e-9 * np.max(np.abs(R))
    a, _, _ = ip.precondition_bp(A, gd, 1e-3)
    b, _, _ = ip.precondition_bp(A, gd, 1e-3)
    assert torch.equal(a, b)


def test_bp_preconditioned_lbfgs_iterate_matches_oracle(ip):
    # optimiser option precondition = 2 against the stored oracle iterate
    gold = json.load(open(GOLD))
    w = inputs.WORKLOADS[gold["workload"]]
    A = torch.as_tensor(ip.cell_tensor(w["gen"]()), device="cuda")
    opts = ip.default_opts(chi=w["chi"], maxiter=gold["iterations"], precondition=2,
                           ctm_tol=gold["ctm_tol"], ctm_maxit=gold["ctm_maxit"])
    _, log, st = ip.optimize(A, ip.ham_heisenberg(True), opts)
    ref = gold["log"]
    assert len(log) == len(ref)
    for r, o in zip(log, ref):
        assert abs(r["E"] - o["f"]) <= 1e-10, (r, o)
        if "alpha" in o:
            assert abs(r["alpha"] - o["alpha"]) <= 1e-6 * abs(o["alpha"]), (r, o)
            assert r["evals"] == int(o["evals"]), (r, o)
            assert abs(r["delta"] - o["delta"]) <= 1e-10 * o["delta"], (r, o)
