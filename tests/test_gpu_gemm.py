"""tcgen05 BF16 GEMM against a plain PyTorch fp32 reference of the same op."""
import pytest

from paper_2007_07379_gb300 import build, pbits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pbits.load()


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 48), (200, 16, 256), (384, 32, 320),
                                   (128, 512, 64), (4096, 256, 256), (130, 40, 24)])
def test_gemm_matches_fp32_reference(M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    pbits.gemm_bf16(A, B, D)
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T
    err = (D - ref).abs().max().item()
    assert err <= 1e-3 * max(1.0, ref.abs().max().item()), err


def test_gemm_epilogues():
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    M, N, K = 256, 256, 96
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    ref = A.float() @ B.float().T
    out = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    pbits.gemm_bf16(A, B, out, bias=bias, flags=pbits.EPI_RELU | pbits.EPI_OUT_BF16)
    want = torch.relu(ref + bias)
    assert torch.allclose(out.float(), want, rtol=1e-2, atol=1e-2)
    mask = torch.randn(M, N, device="cuda", generator=g).to(torch.bfloat16)
    acc = torch.randn(M, N, device="cuda", generator=g)
    acc0 = acc.clone()
    pbits.gemm_bf16(A, B, acc, mask=mask, flags=pbits.EPI_MASK | pbits.EPI_ACCUM, alpha=0.5)
    want = acc0 + 0.5 * ref * (mask.float() > 0)
    assert torch.allclose(acc, want, rtol=1e-4, atol=1e-3)
