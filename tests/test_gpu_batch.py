"""Batched evaluation of independent problems of uneven shape (concurrent streams, then one
CUDA graph): every problem's E_S and gradient equal its own nqs_energy_grad result."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, to_dev
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _make(N, wl):
    p = synth.make_problem(wl)
    P = N.Problem(wl.norb, wl.nalpha, wl.nbeta, p.h, p.eri)
    dets = to_dev(p.S)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    csr = N.connections(P, dets)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    grad = torch.zeros(net.num_params(), dtype=torch.float32, device="cuda")
    return (P, net, csr, dets, out, grad)


def test_batch_graph_matches_individual_calls():
    need_gpu()
    N = nqs()
    wls = synth.batched_workloads(count=64)[:6]
    items = [_make(N, wl) for wl in wls]
    N.set_autotune(True)
    refs = []
    for P, net, csr, dets, _, _ in items:   # tunes every GEMM shape, then reference results
        N.energy_grad(P, net, csr, dets)
        o, g, _ = N.energy_grad(P, net, csr, dets)
        refs.append((o.clone(), g.clone()))
    N.set_autotune(False)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    b = N.Batch(items, nstreams=4)
    with torch.cuda.stream(stream):
        b.run(stream)
        stream.synchronize()
        for (o_ref, g_ref), it in zip(refs, items):
            assert torch.equal(it[4], o_ref) and torch.equal(it[5], g_ref)
            it[4].zero_()
            it[5].zero_()
        b.capture(stream)
        for _ in range(2):
            b.launch(stream)
        stream.synchronize()
    for (o_ref, g_ref), it in zip(refs, items):
        assert torch.equal(it[4], o_ref)
        assert torch.equal(it[5], g_ref)
    assert len(N.autotune_entries()) > 0
