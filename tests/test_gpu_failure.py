"""Failure detection without a GPU fault: a bounded device wait on a barrier that nothing
completes gives up after a short limit and returns NQS_ERR_TIMEOUT with the CUDA context still
usable; a capped scratch pool turns an allocation into NQS_ERR_OOM and every block the failed
call took is returned."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    # about 1 ms of SM clocks: the wait runs out, the error word is read and cleared
    for _ in range(2):
        assert N.wait_probe(P, 2_000_000) == N.NQS_ERR_TIMEOUT
    # the context and the problem still work, and the next call sees no stale error
    dets = to_dev(p.S)
    rp, col, val = N.connections(P, dets).host()
    ref = O.hss(10, p.h, p.eri, p.S)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    assert np.array_equal(val, ref.val)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
    csr = N.connections(P, dets)
    out, _, _ = N.energy_grad(P, net, csr, dets, o=N.opts(validate=1))
    assert np.isfinite(out[0].item())
    # out-of-range limits are argument errors
    assert N.wait_probe(P, 0) == N.NQS_ERR_ARG
    assert N.wait_probe(P, 5_000_000_000) == N.NQS_ERR_ARG


def test_scratch_cap_gives_oom_and_leaks_nothing():
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    dets = to_dev(p.S)
    ref = N.connections(P, dets)
    rp0, col0, val0 = ref.host()
    ref.free()
    torch.cuda.synchronize()
    used0, _ = N.pool_usage(P)
    for cap in (4096, 1 << 20):
        N.set_scratch_limit(P, cap)
        with pytest.raises(N.NQSError, match=r"\(-5\)"):
            N.connections(P, dets)
        psi = torch.ones(len(p.S), dtype=torch.float64, device="cuda")
        with pytest.raises(N.NQSError, match=r"\(-5\)"):
            N.pt2(P, dets, psi, -20.0)
        torch.cuda.synchronize()
        assert N.pool_usage(P)[0] == used0  # every block of the failed calls came back
    N.set_scratch_limit(P, 0)
    rp, col, val = N.connections(P, dets).host()
    assert np.array_equal(rp, rp0) and np.array_equal(col, col0) and np.array_equal(val, val0)
