"""tcgen05 BF16 GEMM core against a plain FP32 matmul of the same BF16 inputs (needs a B300)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 16, 128), (384, 128, 576), (128, 256, 64), (128, 48, 192)])
def test_tc_gemm_matches_matmul(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    v.vlbm_tc_gemm_bf16(A, B, D, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.double() @ B.double().T           # products of BF16 values are exact in FP32
    scale = (A.double().abs() @ B.double().abs().T).max().item()
    assert torch.isfinite(D).all()
    assert (D.double() - ref).abs().max().item() <= 1e-6 * scale
