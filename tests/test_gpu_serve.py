"""The optimisation server: continuous batching of independent jobs on one GPU.

Each job's result must be the same alone and in a mix of overlapping jobs of
different shapes, Hamiltonians and unit cells (Heisenberg 1x1, J1-J2 2x2,
Kitaev 1x2) (every kernel is deterministic
and each job owns its buffers, so the tolerance is rounding-free: 1e-12);
admission by memory budget never runs more jobs than fit; cancellation stops
queued and running jobs; bad submissions are refused."""
import time

import numpy as np
import pytest
import torch

from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


def _mix(ip):
    """(name, A host, ham, opts) of three jobs of different kinds (one iteration each)."""
    def opts(chi, **kw):
        base = dict(chi=chi, maxiter=1, precondition=1, ctm_tol=1e-9, ctm_maxit=300, prec=ip.FP64_TC)
        base.update(kw)
        return ip.default_opts(**base)

    return [
        ("heis_1x1", ip.cell_tensor(inputs.uniform_cell(1, 1, 2, 2, 0)), ip.ham_heisenberg(True), opts(8)),
        ("j1j2_2x2", ip.cell_tensor(inputs.uniform_cell(2, 2, 2, 2, 3)), ip.ham_j1j2(1.0, 0.3, False),
         opts(6, precondition=0)),
        ("kitaev_1x2", ip.cell_tensor(inputs.gaussian_cell(2, 1, 4, 2, 0)), ip.ham_kitaev(-1.0), opts(6)),
    ]


def test_results_are_the_same_alone_and_in_the_mix(ip):
    jobs = _mix(ip)
    alone = {}
    srv = ip.Server(slots=1)
    for name, A, ham, o in jobs:
        j = srv.submit(A, ham, o)
        r = srv.wait(j, 300)
        assert r["state"] == "done", (name, r)
        alone[name] = (r["E"], srv.tensor(j), r["iterations"])
    srv.close()
    # the single-job entry point agrees with the server's job
    name, A, ham, o = jobs[0]
    A1, log, _ = ip.optimize(torch.as_tensor(A, device="cuda"), ham, o)
    assert abs(log[-1]["E"] - alone[name][0]) <= 1e-12
    assert float(np.abs(A1.cpu().numpy() - alone[name][1]).max()) <= 1e-12
    # all at once, overlapping on three slots
    srv = ip.Server(slots=3)
    ids = {name: srv.submit(A, ham, o) for name, A, ham, o in jobs}
    for name, j in ids.items():
        r = srv.wait(j, 300)
        assert r["state"] == "done", (name, r)
        assert r["iterations"] == alone[name][2]
        assert abs(r["E"] - alone[name][0]) <= 1e-12, name
        assert float(np.abs(srv.tensor(j) - alone[name][1]).max()) <= 1e-12, name
    st = srv.stats()
    assert st["jobs_done"] == 3 and st["iter_ms_p99"] >= st["iter_ms_p50"] > 0
    srv.close()


def test_admission_respects_the_memory_budget(ip):
    jobs = _mix(ip)
    fp = ip.job_footprint(1, 1, 2, 2, 8)
    assert fp > 0 and ip.job_footprint(2, 2, 2, 2, 8) > fp
    srv = ip.Server(slots=3, hbm_budget_bytes=fp + 1, autotune=False)  # room for one 1x1 job at a time
    ids = [srv.submit(jobs[0][1], jobs[0][2], jobs[0][3]) for _ in range(2)]
    most = 0
    deadline = time.time() + 300
    while time.time() < deadline:
        states = [srv.poll(j)["state"] for j in ids]
        most = max(most, states.count("running"))
        if all(s in ("done", "failed", "cancelled") for s in states):
            break
        time.sleep(0.005)
    assert all(srv.poll(j)["state"] == "done" for j in ids), [srv.poll(j) for j in ids]
    assert most == 1
    assert srv.poll(ids[0])["E"] == srv.poll(ids[1])["E"]
    assert srv.poll(ids[1])["queued_ms"] > 0
    # a job larger than the whole budget still runs (alone)
    big = srv.submit(jobs[1][1], jobs[1][2], jobs[1][3])
    assert srv.wait(big, 300)["state"] == "done"
    srv.close()


def test_cancel_queued_and_running_jobs(ip):
    name, A, ham, _ = _mix(ip)[0]
    o = ip.default_opts(chi=8, maxiter=10000, precondition=1, ctm_tol=1e-9, ctm_maxit=300, prec=ip.FP64_TC,
                        gtol=0.0)
    fp = ip.job_footprint(1, 1, 2, 2, 8)
    srv = ip.Server(slots=1, hbm_budget_bytes=fp + 1, autotune=False)
    running = srv.submit(A, ham, o)
    queued = srv.submit(A, ham, o)
    deadline = time.time() + 300
    while srv.poll(running)["iterations"] < 1 and srv.poll(running)["state"] == "running":
        assert time.time() < deadline, srv.poll(running)
        time.sleep(0.01)
    assert srv.poll(queued)["state"] == "queued"
    srv.cancel(queued)
    assert srv.poll(queued)["state"] == "cancelled"
    srv.cancel(running)
    r = srv.wait(running, 300)
    assert r["state"] == "cancelled" and r["iterations"] >= 1
    assert np.isfinite(srv.tensor(running)).all()
    srv.close()


def test_bad_submissions_are_refused(ip):
    srv = ip.Server(slots=1)
    A = ip.cell_tensor(inputs.uniform_cell(1, 1, 2, 2, 0))
    with pytest.raises(ip.IpepsError) as e:
        srv.submit(A, ip.ham_kitaev(-1.0), ip.default_opts(chi=8))  # d = 4 Hamiltonian on a d = 2 cell
    assert e.value.status == 1
    bad = A.copy()
    bad.flat[0] = np.nan
    with pytest.raises(ip.IpepsError):
        srv.submit(bad, ip.ham_heisenberg(True), ip.default_opts(chi=8))
    with pytest.raises(ip.IpepsError):
        srv.submit(A, ip.ham_heisenberg(True), ip.default_opts(chi=0))
    srv.close()
