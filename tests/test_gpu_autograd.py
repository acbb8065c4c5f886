"""E(A) as a torch.autograd.Function whose backward is the library's
fixed-point gradient (ipeps_energy_grad), against the CPU oracle's gradient
and central finite differences of the forward (FP64 bar: relative gradient
error <= 1e-8)."""
import numpy as np
import pytest
import torch

from oracle import gradient as OG
from oracle import models as OM
from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


def test_energy_function_backward_is_the_fixed_point_gradient(ip):
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda").requires_grad_(True)
    ham = ip.ham_heisenberg(True)
    state = {}
    E = ip.energy_fn(A, ham, 16, tol=1e-12, maxit=600, state=state)
    E.backward()
    Eo, go = OG.energy_and_gradient(cell, OM.heisenberg(True), 16, tol=1e-12)
    assert abs(float(E) - Eo) <= 1e-10
    g = A.grad.cpu().numpy()[0, 0]
    assert np.linalg.norm(g - go[0][0]) <= 1e-8 * np.linalg.norm(go[0][0])
    # central differences of the forward, warm-started from the same environment
    h = 1e-6
    for i in inputs.random_entries(A.numel(), 4, seed=5):
        vals = []
        for sgn in (1, -1):
            Ap = A.detach().clone()
            Ap.view(-1)[i] += sgn * h
            vals.append(float(ip.energy_fn(Ap, ham, 16, tol=1e-12, maxit=600, state=dict(state))))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g.ravel()[i]) < 2e-8, (i, fd, g.ravel()[i])


def test_backward_refuses_an_advanced_environment(ip):
    cell = inputs.WORKLOADS["heis_d2_chi16"]["gen"]()
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda").requires_grad_(True)
    ham = ip.ham_heisenberg(True)
    state = {}
    E = ip.energy_fn(A, ham, 16, tol=1e-11, state=state)
    ip.energy_fn((A * 1.01).detach(), ham, 16, tol=1e-11, state=state)  # advances the shared environment
    with pytest.raises(RuntimeError):
        E.backward()
