"""Tensor-core precision modes against the FP64 oracle.

Workload: Heisenberg 1x1, d=2, D=4, chi=32 (chi D^2 = 512, so the enlarged-corner
and half-system GEMMs take the tensor-core paths), seeded uniform[-1,1] tensor.
  * IPEPS_FP64_TC: every large GEMM from 8 BF16 digits per operand (36 products
    per term) on tcgen05: held to the FP64 bar (|dE| <= 1e-10, gradient <= 1e-8).
  * IPEPS_TF32X3 and IPEPS_BF16X3: 3xTF32 / BF16x3 iterations, then FP64 /
    FP64-grade iterations to tol: the reduced-precision bar (|dE| <= 1e-7,
    relative gradient error <= 1e-5).
  * IPEPS_TF32X3_ALL: 3xTF32 everywhere, no FP64-grade phase: the spectra stall
    at the 3xTF32 noise floor; its energy is within 1e-6 of the oracle and its
    gradient within 2e-3 (measured 1.8e-7 and 5e-4): pure 3-product arithmetic
    does not reach the 1e-5 gradient bar through the fixed-point adjoint.
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
    E, g, _ = OG.energy_and_gradient(cell, OM.heisenberg(True), CHI, tol=1e-11, return_info=True)
    return cell, E, g[0][0]


@pytest.mark.parametrize("prec,kernel,dE,dg", [("TF32X3", "tc_gemm", 1e-7, 1e-5), ("BF16X3", "oz2_gemm", 1e-7, 1e-5),
                                               ("FP64_TC", "oz8_gemm", 1e-10, 1e-8)])
def test_tensor_core_modes_match_oracle(ip, case, prec, kernel, dE, dg):
    cell, Eo, go = case
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    ip.profile(True)
    env, it, err = ip.ctmrg(A, CHI, tol=1e-11, maxit=300, prec=getattr(ip, prec))
    stats = ip.profile_stats()
    ip.profile(False)
    assert stats.get(kernel, {}).get("count", 0) > 0  # the tensor-core path ran
    assert err < 1e-11
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    assert abs(E - Eo) <= dE
    gg = g.cpu().numpy()[0, 0]
    assert np.linalg.norm(gg - go) <= dg * np.linalg.norm(go)


def test_all_tf32_mode(ip, case):
    # every bulk GEMM in 3xTF32, no FP64 phase: CTMRG stops at the noise floor
    cell, Eo, go = case
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    env, it, err = ip.ctmrg(A, CHI, tol=1e-10, maxit=100, prec=ip.TF32X3_ALL, allow_unconverged=True)
    assert np.isfinite(err) and err < 1e-2
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    assert abs(E - Eo) <= 1e-6
    gg = g.cpu().numpy()[0, 0]
    assert np.linalg.norm(gg - go) <= 2e-3 * np.linalg.norm(go)
