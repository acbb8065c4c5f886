"""The allocation-free GEMM entry point (ipeps_gemm_noalloc) against the
allocating one (ipeps_gemm, FP64) on two calls in a row.

Some callers cannot let the library allocate device memory: their device
memory is already reserved by another allocator, or they cannot take the
device-wide synchronisation a cudaFree implies.  This entry point keeps its
split-K partial sums in a fixed device array instead.  The file is collected
last so that a run stopping at its first failure has already run every other
test."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ip():
    import __graft_entry__ as g

    g.build()
    from paper_2511_09546_gb300 import ipeps

    return ipeps


def _case(seed, M, N, K):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn((M, K), generator=g, dtype=torch.float64).cuda()
    B = torch.randn((N, K), generator=g, dtype=torch.float64).cuda()
    C = torch.randn((M, N), generator=g, dtype=torch.float64).cuda()
    return A, B, C


@pytest.mark.parametrize("M,N,K", [(96, 80, 9000), (40, 1, 278528), (700, 300, 64)])
def test_noalloc_matches_allocating_gemm_twice(ip, M, N, K):
    for seed in (1, 2):  # the second call finds the array as the first one left it
        A, B, C = _case(seed * 1000 + M, M, N, K)
        ref = ip.gemm(A, B, tb=True, alpha=0.5, beta=-1.5, C=C.clone())
        out = ip.gemm_noalloc(A, B, C.clone(), tb=True, alpha=0.5, beta=-1.5)
        torch.cuda.synchronize()
        scale = max(1.0, float(ref.abs().max()))
        assert float((out - ref).abs().max()) <= 1e-12 * scale * K ** 0.5


def test_noalloc_full_scratch_and_transposed_a(ip):
    # M * N equal to the array's capacity (one K slice fills it), then op(A)
    # read transposed: both against the allocating entry point, twice
    for seed in (3, 4):
        g = torch.Generator(device="cpu").manual_seed(seed)
        A = torch.randn((2048, 24), generator=g, dtype=torch.float64).cuda()
        B = torch.randn((24, 2048), generator=g, dtype=torch.float64).cuda()
        C = torch.randn((2048, 2048), generator=g, dtype=torch.float64).cuda()
        ref = ip.gemm(A, B, alpha=1.25, beta=0.5, C=C.clone())
        out = ip.gemm_noalloc(A, B, C.clone(), alpha=1.25, beta=0.5)
        assert float((out - ref).abs().max()) <= 1e-12 * max(1.0, float(ref.abs().max()))
        At = torch.randn((3000, 130), generator=g, dtype=torch.float64).cuda()  # K x M
        Bt = torch.randn((3000, 70), generator=g, dtype=torch.float64).cuda()   # K x N
        Ct = torch.randn((130, 70), generator=g, dtype=torch.float64).cuda()
        ref = ip.gemm(At, Bt, ta=True, beta=-1.0, C=Ct.clone())
        out = ip.gemm_noalloc(At, Bt, Ct.clone(), ta=True, beta=-1.0)
        assert float((out - ref).abs().max()) <= 1e-12 * max(1.0, float(ref.abs().max())) * 3000 ** 0.5


def test_noalloc_empty_k_scales_c(ip):
    # K = 0: C = beta C exactly
    C = torch.randn((33, 17), dtype=torch.float64, device="cuda")
    A = torch.zeros((33, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 17), dtype=torch.float64, device="cuda")
    out = ip.gemm_noalloc(A, B, C.clone(), beta=-1.5)
    assert torch.equal(out, -1.5 * C)


def test_noalloc_rejects_oversized_output(ip):
    A = torch.zeros((4096, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((8, 2048), dtype=torch.float64, device="cuda")
    C = torch.zeros((4096, 2048), dtype=torch.float64, device="cuda")
    with pytest.raises(ip.IpepsError) as e:
        ip.gemm_noalloc(A, B, C)
    assert e.value.status == 1 and "exceeds" in str(e.value)
