"""Batched evaluation of independent problems of uneven shape (concurrent streams, then one
CUDA graph): every problem's E_S and gradient equal its own nqs_energy_grad result, and members
of the batch match the oracle's quantisation-matched evaluation."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, to_dev
from oracle import oracle as O
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


def test_batch_streams_graph_matches_individual_calls():
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
    b = N.Batch(items, nstreams=4, mode=N.BATCH_STREAMS)
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


def test_batch_grouped_matches_individual_calls():
    """The grouped mode (one launch per stage over all problems; grouped tensor-core GEMMs over
    a (problem, tile) work list), eager and as a CUDA graph, on sixteen problems of uneven shape:
    E_S, N, D and max log|psi| equal the problems' own nqs_energy_grad results to 1e-12
    relative, and the gradients to 1e-6 relative L2 (the weight gradients' FP32 split-K sums are
    the only reordered arithmetic)."""
    need_gpu()
    N = nqs()
    wls = synth.batched_workloads(count=64)[:16]
    items = [_make(N, wl) for wl in wls]
    refs = []
    for P, net, csr, dets, _, _ in items:
        o, g, _ = N.energy_grad(P, net, csr, dets)
        refs.append((o.clone(), g.clone()))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    b = N.Batch(items, nstreams=4)
    assert b.mode == N.BATCH_GROUPED

    def check():
        for (o_ref, g_ref), it in zip(refs, items):
            o, g = it[4].cpu().numpy(), it[5].cpu().numpy().astype(np.float64)
            oref = o_ref.cpu().numpy()
            assert np.all(np.abs(o - oref) <= 1e-12 * np.abs(oref)), (o, oref)
            gr = g_ref.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(g - gr) <= 1e-6 * np.linalg.norm(gr)
            it[4].zero_()
            it[5].zero_()

    with torch.cuda.stream(stream):
        b.run(stream)
        stream.synchronize()
        check()
        b.capture(stream)
        for _ in range(2):
            b.launch(stream)
        stream.synchronize()
        check()


def test_batch_grouped_energy_only_and_modes():
    """Energy only (no gradients) in the grouped mode; switching to the streams mode and back
    gives the same energies."""
    need_gpu()
    N = nqs()
    wls = synth.batched_workloads(count=64)[:5]
    items = []
    for wl in wls:
        P, net, csr, dets, out, _ = _make(N, wl)
        items.append((P, net, csr, dets, out, None))
    refs = [N.energy_grad(P, net, csr, dets, with_grad=False)[0].clone()
            for P, net, csr, dets, _, _ in items]
    b = N.Batch(items, nstreams=2)
    assert b.mode == N.BATCH_GROUPED
    b.run()
    torch.cuda.synchronize()
    got = [it[4].clone() for it in items]
    b.set_mode(N.BATCH_STREAMS)
    b.run()
    torch.cuda.synchronize()
    for r, g, it in zip(refs, got, items):
        assert torch.equal(r, g) and torch.equal(r, it[4])


def test_batch_members_match_quantised_oracle():
    """Three members of a graph-launched batch in the grouped mode (the smallest |S| of the
    first eight problems), each against the oracle's quantisation-matched E_S and gradient of
    its own problem: E_S within 1e-6 Ha, gradient within 1e-2 relative L2."""
    need_gpu()
    N = nqs()
    wls = synth.batched_workloads(count=64)[:8]
    items = [_make(N, wl) for wl in wls]
    stream = torch.cuda.Stream()
    b = N.Batch(items, nstreams=4)
    assert b.mode == N.BATCH_GROUPED
    with torch.cuda.stream(stream):
        b.run(stream)
        b.capture(stream)
        for it in items:
            it[4].zero_()
            it[5].zero_()
        b.launch(stream)
        stream.synchronize()
    order = np.argsort([wl.nS for wl in wls])[:3]
    for i in order:
        p = synth.make_problem(wls[i])
        ref = O.energy_grad(O.Net(p.net, quant=True), p.S, O.hss(p.wl.norb, p.h, p.eri, p.S))
        E = items[i][4][0].item()
        g = items[i][5].cpu().numpy().astype(np.float64)
        assert abs(E - ref["E"]) < 1e-6, (wls[i].name, E - ref["E"])
        rel = np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"])
        assert rel < 1e-2, (wls[i].name, rel)
