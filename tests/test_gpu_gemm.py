"""The contraction engine's GEMM against torch float64 matmul (every kernel path)."""
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [
    (64, 64, 64), (130, 70, 33),          # tiled, ragged tails
    (1024, 1024, 1024),                   # full tiles
    (40, 1, 278528), (7, 3, 5000),        # multi-dot split-K (tiny output, long K)
    (278528, 1, 40), (2, 256, 256),       # one thin side: per-output kernel
    (96, 96, 8192), (64, 128, 4096),      # few tiles, long K: tiled split-K
    (1, 1, 1), (3, 5, 0),
]


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_f64(ip, M, N, K, ta, tb):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((K, M) if ta else (M, K), generator=g, dtype=torch.float64).cuda()
    B = torch.randn((N, K) if tb else (K, N), generator=g, dtype=torch.float64).cuda()
    C0 = torch.randn((M, N), generator=g, dtype=torch.float64).cuda()
    ref = 0.7 * ((A.T if ta else A) @ (B.T if tb else B)) - 0.3 * C0
    out = ip.gemm(A, B, ta=ta, tb=tb, alpha=0.7, beta=-0.3, C=C0.clone())
    scale = max(1.0, float(ref.abs().max()))
    assert float((out - ref).abs().max()) <= 1e-12 * scale * max(1, K) ** 0.5
