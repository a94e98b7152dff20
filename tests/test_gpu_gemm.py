"""Numerics of the tcgen05 BF16 GEMM (nqs_gemm_bf16, the kernel the backflow layers use)
against a plain PyTorch reference of the same op (bf16 inputs, products summed in FP64):
ragged M/N/K, tiles narrower than the box, and split-K."""
import pytest
import torch

from gpu_common import need_gpu, nqs

pytestmark = pytest.mark.gpu


@pytest.fixture(params=[True, False], ids=["paired", "single"])
def pairing(request):
    """Both forms of the 256-column tiles: paired (two SMs, cta_group::2) and single-SM."""
    need_gpu()
    N_ = nqs()
    N_.set_gemm_pairing(request.param)
    yield request.param
    N_.set_gemm_pairing(True)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (64, 32, 64), (300, 100, 200), (1000, 256, 256),
                                   (16384, 256, 256), (256, 256, 16384), (720, 512, 4104),
                                   (130, 250, 72), (200, 2016, 136), (4096 + 77, 1000, 1024)])
def test_gemm_bf16_matches_torch(M, N, K, pairing):
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


def test_gemm_paired_and_single_agree():
    """The paired (M = 256 over two SMs) and single-SM forms give the same FP32 results on a
    shape with ragged rows and columns, a multi-wave one and a split-K one, up to the bound of
    the FP32 accumulation (the two forms sum each output over k in the same order)."""
    need_gpu()
    N_ = nqs()
    try:
        for (M, N, K) in [(1000, 300, 200), (40000, 1024, 256), (512, 512, 65536)]:
            g = torch.Generator(device="cuda").manual_seed(M + N + K)
            A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
            B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
            N_.set_gemm_pairing(True)
            Cp = N_.gemm_bf16(A, B)
            N_.set_gemm_pairing(False)
            Cs = N_.gemm_bf16(A, B)
            bound = (A.float().abs() @ B.float().abs().T) * 2e-6 + 1e-6
            assert bool(((Cp - Cs).abs() <= bound).all())
    finally:
        N_.set_gemm_pairing(True)


def test_gemm_rejects_unaligned_stride():
    need_gpu()
    N_ = nqs()
    A = torch.randn(64, 100, device="cuda").to(torch.bfloat16)  # 200-byte rows
    B = torch.randn(64, 100, device="cuda").to(torch.bfloat16)
    with pytest.raises(N_.NQSError, match="unsupported"):
        N_.gemm_bf16(A, B)


@pytest.mark.parametrize("M,N,K,ldb", [(1000, 296, 200, 296), (304, 84, 5000, 88),
                                       (2016, 1024, 16384, 1024), (136, 250, 72, 256),
                                       (1024, 256, 4104, 256)])
@pytest.mark.parametrize("a_mn,b_mn", [(1, 1), (1, 0), (0, 1)])
def test_gemm_bf16_mn_major_operands(M, N, K, ldb, a_mn, b_mn, pairing):
    """MN-major operands (A stored [K][M], B stored [K][ldb] with N <= ldb: the row-major
    activations a weight gradient reads) against the PyTorch reference of the same product,
    for ragged M / N / K, a row pitch wider than N, and split-K."""
    need_gpu()
    N_ = nqs()
    g = torch.Generator(device="cuda").manual_seed(M * 5 + N * 3 + K + a_mn + 2 * b_mn)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bfull = torch.randn(ldb, K, device="cuda", generator=g).to(torch.bfloat16)
    B = Bfull[:N]
    Aop = A.T.contiguous() if a_mn else A
    Bop = Bfull.T.contiguous() if b_mn else B.contiguous()
    C = N_.gemm_bf16_ex(Aop, bool(a_mn), Bop, bool(b_mn), M=M, N=N)
    ref = A.double() @ B.double().T
    bound = (A.double().abs() @ B.double().abs().T) * 2e-6 + 1e-6
    err = (C.double() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
