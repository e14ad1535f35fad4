"""The tcgen05 BF16 GEMM (TMEM accumulator) against torch's float32 product of
the same BF16 inputs.  Tolerance: FP32 accumulation in another order,
|err| <= 1e-3 * (1 + |ref|) element-wise."""
import pytest
import torch

import paper_1806_08384_b300 as sel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,splits", [(128, 256, 64, 1), (128, 256, 144, 1), (300, 256, 256, 1),
                                          (4096, 256, 256, 1), (256, 256, 4096, 8), (77, 40, 24, 1),
                                          (256, 512, 192, 3)])
def test_gemm_matches_torch(dev, M, N, K, splits):
    g = torch.Generator(device=dev).manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device=dev, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device=dev, generator=g).to(torch.bfloat16)
    C = sel.debug_gemm_bf16(A, B, splits)
    ref = A.float() @ B.float().T
    assert torch.all((C - ref).abs() <= 1e-3 * (1 + ref.abs())), float((C - ref).abs().max())


def test_gemm_identity_layout(dev):
    """A = I picks rows of B: checks the swizzled row/column placement exactly."""
    A = torch.eye(128, 64, device=dev).to(torch.bfloat16)
    B = torch.arange(256 * 64, device=dev, dtype=torch.float32).reshape(256, 64).remainder(251).to(torch.bfloat16)
    C = sel.debug_gemm_bf16(A, B)
    assert torch.equal(C, (A.float() @ B.float().T))
