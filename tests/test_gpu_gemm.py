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
    (64, 1024, 64), (1024, 64, 64),       # few 64 x 64 tiles: 32 x 32 tiles, split K
    (40, 50, 12), (256, 256, 16),         # 32 x 32 tiles, K unsplit
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


TC_SHAPES = [(128, 128, 32), (130, 70, 33), (256, 256, 256), (1000, 300, 777), (300, 1000, 96), (1, 5, 40),
             (257, 129, 2049)]
TRANS = [(False, False), (True, False), (False, True), (True, True)]


def _operands(M, N, K, ta, tb, seed, kind):
    g = torch.Generator(device="cpu").manual_seed(seed)
    sa, sb = ((K, M) if ta else (M, K)), ((N, K) if tb else (K, N))
    if kind == "int":
        A = torch.randint(-4, 5, sa, generator=g).double()
        B = torch.randint(-4, 5, sb, generator=g).double()
    else:
        A = torch.randn(sa, generator=g, dtype=torch.float64)
        B = torch.randn(sb, generator=g, dtype=torch.float64)
    C0 = torch.randint(-4, 5, (M, N), generator=g).double()
    return A.cuda(), B.cuda(), C0.cuda()


@pytest.mark.parametrize("M,N,K", TC_SHAPES)
@pytest.mark.parametrize("ta,tb", TRANS)
def test_gemm_tf32x3_integers_exact(ip, M, N, K, ta, tb):
    # small integers are exact in TF32 (lo = 0) and every partial sum here is an
    # integer below 2^24, so the tensor-core result must be exact: this pins
    # the pack layout, the transposes, the tails and the tile indexing bit for bit
    A, B, C0 = _operands(M, N, K, ta, tb, M * 7 + N * 3 + K, "int")
    ref = 2.0 * ((A.T if ta else A) @ (B.T if tb else B)) - C0
    out = ip.gemm(A, B, ta=ta, tb=tb, alpha=2.0, beta=-1.0, C=C0.clone(), prec=ip.TF32X3)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("M,N,K", TC_SHAPES)
@pytest.mark.parametrize("ta,tb", TRANS)
def test_gemm_tf32x3_random(ip, M, N, K, ta, tb):
    # 3xTF32: dropping lo*lo costs ~2^-22 |a||b| per product; FP32 accumulation in
    # chunks (truncated per MMA) with a compensated sum across chunks stays near
    # 2^-21 of sum |a||b|.  A dropped correction term (error ~2^-12) fails this.
    A, B, C0 = _operands(M, N, K, ta, tb, M * 11 + N * 5 + K, "randn")
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = 1.3 * (opA @ opB) + 0.25 * C0
    out = ip.gemm(A, B, ta=ta, tb=tb, alpha=1.3, beta=0.25, C=C0.clone(), prec=ip.TF32X3)
    scale = 1.3 * (opA.abs() @ opB.abs())
    assert float(((out - ref).abs() / scale).max()) <= 2.0 ** -19


# BF16-digit tensor-core GEMM: tile tails, every transpose pair, split K (few
# output tiles and long K) and K shorter than one slice
OZ_SHAPES = [(128, 64, 32), (130, 70, 33), (257, 129, 2049), (1000, 300, 777), (64, 16, 9000), (1024, 64, 1024),
             (5, 40, 13)]


@pytest.mark.parametrize("slices,prec", [(8, "FP64_TC"), (2, "BF16X3")])
@pytest.mark.parametrize("M,N,K", OZ_SHAPES)
@pytest.mark.parametrize("ta,tb", TRANS)
def test_gemm_digits_integers_exact(ip, slices, prec, M, N, K, ta, tb):
    # integers |x| <= 4 are exact in the leading 7-bit digit and every level sum
    # is an exact integer, so the result must equal the FP64 product bit for bit
    A, B, C0 = _operands(M, N, K, ta, tb, M * 13 + N * 7 + K + slices, "int")
    ref = 2.0 * ((A.T if ta else A) @ (B.T if tb else B)) - C0
    out = ip.gemm(A, B, ta=ta, tb=tb, alpha=2.0, beta=-1.0, C=C0.clone(), prec=getattr(ip, prec))
    assert torch.equal(out, ref)


@pytest.mark.parametrize("M,N,K", OZ_SHAPES)
@pytest.mark.parametrize("ta,tb", TRANS)
def test_gemm_fp64_tc_random(ip, M, N, K, ta, tb):
    # 8 digits: the error of an FP64 GEMM, measured against the row and column
    # maxima (K 2^-52 max|a_i.| max|b_.j|); a dropped level (>= 2^-42) or a
    # digit off by one ulp of its scale fails this by orders of magnitude
    A, B, C0 = _operands(M, N, K, ta, tb, M * 17 + N * 3 + K, "randn")
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = 1.3 * (opA @ opB) + 0.25 * C0
    out = ip.gemm(A, B, ta=ta, tb=tb, alpha=1.3, beta=0.25, C=C0.clone(), prec=ip.FP64_TC)
    bound = 1.3 * K * 2.0 ** -52 * opA.abs().amax(1, keepdim=True) * opB.abs().amax(0, keepdim=True) + 1e-300
    assert float(((out - ref).abs() / bound).max()) <= 1.0


def test_gemm_fp64_tc_wide_row_scales(ip):
    # rows and columns spanning 2^-60 .. 2^60: each keeps its own exponent
    g = torch.Generator(device="cpu").manual_seed(9)
    M, N, K = 200, 150, 700
    A = torch.randn((M, K), generator=g, dtype=torch.float64) * torch.pow(2.0, torch.randint(-60, 61, (M, 1), generator=g).double())
    B = torch.randn((K, N), generator=g, dtype=torch.float64) * torch.pow(2.0, torch.randint(-60, 61, (1, N), generator=g).double())
    A, B = A.cuda(), B.cuda()
    ref = A @ B
    out = ip.gemm(A, B, prec=ip.FP64_TC)
    bound = K * 2.0 ** -52 * A.abs().amax(1, keepdim=True) * B.abs().amax(0, keepdim=True)
    assert float(((out - ref).abs() / bound).max()) <= 1.0


@pytest.mark.parametrize("M,N,K", [(257, 129, 2049), (1024, 64, 1024)])
def test_gemm_bf16x3_random(ip, M, N, K):
    # 2 digits, 3 products: about 2^-15 of the row and column maxima per product
    A, B, C0 = _operands(M, N, K, False, True, M + N + K, "randn")
    ref = A @ B.T
    out = ip.gemm(A, B, tb=True, prec=ip.BF16X3)
    bound = K * 2.0 ** -13 * A.abs().amax(1, keepdim=True) * B.abs().amax(1, keepdim=True).T
    err = ((out - ref).abs() / bound)
    assert float(err.max()) <= 1.0
    # and it is not secretly the 8-digit product
    assert float((out - ref).abs().max()) > 1e-9 * float(ref.abs().max())
