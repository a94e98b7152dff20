"""Numerics of the tcgen05 BF16 GEMM (nqs_gemm_bf16, the kernel the backflow layers use)
against a plain PyTorch reference of the same op (bf16 inputs, products summed in FP64):
ragged M/N/K, tiles narrower than the box, and split-K."""
import pytest
import torch

from gpu_common import need_gpu, nqs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (64, 32, 64), (300, 100, 200), (1000, 256, 256),
                                   (16384, 256, 256), (256, 256, 16384), (720, 512, 4104),
                                   (130, 250, 72)])
def test_gemm_bf16_matches_torch(M, N, K):
    need_gpu()
    N_ = nqs()
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = N_.gemm_bf16(A, B)
    ref = A.double() @ B.double().T
    bound = (A.double().abs() @ B.double().abs().T) * 2e-6 + 1e-6
    err = (C.double() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


def test_gemm_rejects_unaligned_stride():
    need_gpu()
    N_ = nqs()
    A = torch.randn(64, 100, device="cuda").to(torch.bfloat16)  # 200-byte rows
    B = torch.randn(64, 100, device="cuda").to(torch.bfloat16)
    with pytest.raises(N_.NQSError, match="unsupported"):
        N_.gemm_bf16(A, B)
