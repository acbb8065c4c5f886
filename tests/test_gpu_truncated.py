"""FP64 path on the truncated-SVD branch (chi D^2 = 1024 > 256: warm-started
subspace SVD, block adjoint with the complement CG) against the oracle at the
FP64 bar.  Degenerate-cut reading: where the four-corner product's relative gap
(s_chi - s_{chi+1}) / s_1 is at rounding level the kept block is not unique and
only the energy is compared (the Neel-like seed of the D=4, chi=64 workload)."""
import numpy as np
import pytest
import torch

from oracle import ctmrg as OC
from oracle import gradient as OG
from oracle import models as OM
from paper_2511_09546_gb300 import inputs

pytestmark = pytest.mark.gpu

CHI = 64


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


@pytest.mark.parametrize("prec", ["FP64", "FP64_TC"])
@pytest.mark.parametrize("name", ["random_d4", "neel_seed_d4"])
def test_truncated_path_fp64(ip, name, prec):
    # FP64_TC: every large GEMM from BF16 digits on the tensor cores, same FP64 bar
    cell = inputs.uniform_cell(1, 1, 2, 4, 3) if name == "random_d4" else inputs.WORKLOADS["heis_d4_chi64"]["gen"]()
    A = torch.as_tensor(ip.cell_tensor(cell), device="cuda")
    ip.profile(True)
    env, it, err = ip.ctmrg(A, CHI, tol=1e-11, maxit=300, prec=getattr(ip, prec))
    if prec == "FP64_TC":
        assert ip.profile_stats().get("oz8_gemm", {}).get("count", 0) > 0  # the tensor-core path ran
    ip.profile(False)
    E, g = ip.energy_grad(A, env, ip.ham_heisenberg(True))
    Eo, go, info = OG.energy_and_gradient(cell, OM.heisenberg(True), CHI, tol=1e-11, return_info=True)
    assert abs(E - Eo) <= 1e-10
    gap = min(OC.cut_gaps(1, 1, OC.as_torch_cell(cell), info["env"], CHI))
    if gap <= 1e-8:
        pytest.skip(f"degenerate cut (relative gap {gap:.1e}): energy compared, gradient not asserted")
    gg = g.cpu().numpy()[0, 0]
    assert np.linalg.norm(gg - go[0][0]) <= 1e-8 * np.linalg.norm(go[0][0])
