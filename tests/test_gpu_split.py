"""Split-precision path (3xTF32 GEMMs on tcgen05 tensor cores) against the FP64 oracle.

Workload: Heisenberg 1x1, d=2, D=4, chi=32 (chi D^2 = 512, so the enlarged-corner
and half-system GEMMs take the tensor-core path), seeded uniform[-1,1] tensor.
The reduced-precision bar is |dE| <= 1e-7 and relative gradient error <= 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import gradient as OG
from oracle import models as OM
from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu

CHI = 32


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


@pytest.fixture(scope="module")
def case():
    cell = inputs.uniform_cell(1, 1, 2, 4, 3)
    E, g, _ = OG.energy_and_gradient(cell, OM.heisenberg(True), CHI, tol=1e-10, return_info=True)
    return cell, E, g[0][0]


def test_split_precision_matches_oracle(ip, case):
    cell, Eo, go = case
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    ip.profile(True)
    env, it, err = ip.ctmrg(A, CHI, tol=1e-10, maxit=300, prec=ip.TF32X3)
    stats = ip.profile_stats()
    ip.profile(False)
    assert stats.get("tc_gemm", {}).get("count", 0) > 0  # the tensor-core path ran
    assert err < 1e-10
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    assert abs(E - Eo) <= 1e-7
    gg = g.cpu().numpy()[0, 0]
    assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go)


def test_all_tf32_mode_energy(ip, case):
    # every bulk GEMM in 3xTF32, no FP64 phase: the energy stays near the oracle
    # while the spectra change stalls at the 3xTF32 noise floor
    cell, Eo, _ = case
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    env, it, err = ip.ctmrg(A, CHI, tol=1e-10, maxit=100, prec=ip.TF32X3_ALL, allow_unconverged=True)
    assert np.isfinite(err)
    E = ip.energy(A, env, ip.ham_heisenberg(True))
    assert abs(E - Eo) <= 1e-5
