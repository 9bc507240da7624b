"""Numerics of the tcgen05 BF16 GEMM (gmt_gemm_bf16) against a plain PyTorch
FP32 reference of the same operation on the same BF16-rounded operands."""
import pytest
import torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def ref(A, B, bias=None):
    C = A.float() @ B.float().T
    return C + bias if bias is not None else C


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (256, 512, 1024, 1), (130, 70, 200, 1),
                                          (1, 4096, 528, 1), (256, 512, 32768, 16), (512, 4096, 528, 3),
                                          (300, 200, 4096, 7), (512, 32768, 256, 1), (1024, 512, 32768, 4),
                                          (77, 1000, 96, 1)])
def test_gemm_matches_fp32_reference(M, N, K, splits):
    from paper_1705_02403_gb300 import _native as N_
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C, err = N_.gmt_gemm_bf16(A, B, 0, splits=splits)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    R = ref(A, B)
    scale = R.abs().max().item() + 1e-6
    assert (C - R).abs().max().item() <= 2e-5 * K ** 0.5 * scale + 1e-4


def test_gemm_epilogues():
    from paper_1705_02403_gb300 import _native as N_
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(200, 512, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(300, 512, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(300, device="cuda", generator=g)
    C2, err = N_.gmt_gemm_bf16(A, B, 2, bias=bias)
    R = ref(A, B, bias)
    assert int(err.item()) == 0
    assert (C2 - R).abs().max().item() <= 1e-3 * R.abs().max().item()
    C1, err = N_.gmt_gemm_bf16(A, B, 1, bias=bias)
    assert C1.dtype == torch.bfloat16 and int(err.item()) == 0
    R1 = torch.relu(R).to(torch.bfloat16).float()
    assert (C1.float() - R1).abs().max().item() <= 1e-2 * R.abs().max().item()
    C1s, err = N_.gmt_gemm_bf16(A, B, 1, bias=bias, splits=4)
    assert (C1s.float() - R1).abs().max().item() <= 1e-2 * R.abs().max().item()
