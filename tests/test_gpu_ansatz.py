"""GPU parity of amplitudes, E_S and its gradient against the oracle (FP64 form: 1e-8 Ha and
tight gradient agreement; mixed form: 1e-6 Ha against the quantisation-matched oracle), and the
adjoint against central finite differences, through the C ABI and the autograd wrapper."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, small_problem, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _setup(name, mixed):
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    dt = N.NQS_MIXED if mixed else N.NQS_FP64
    net = N.Net(P, N.net_tensors(p.net, dt), dt)
    return N, p, P, net


def test_amplitudes_fp64():
    need_gpu()
    N, p, P, net = _setup("tiny_n10", False)
    la, sg, st = N.amplitudes(P, net, to_dev(p.S))
    rla, rsg = O.amplitudes(O.Net(p.net), p.S)
    assert st == 0
    assert np.array_equal(sg.cpu().numpy(), rsg)
    assert np.abs(la.cpu().numpy() - rla).max() < 1e-11


def test_amplitudes_mixed_vs_quantised_oracle():
    need_gpu()
    N, p, P, net = _setup("small_n16", True)
    la, sg, _ = N.amplitudes(P, net, to_dev(p.S))
    rla, rsg = O.amplitudes(O.Net(p.net, quant=True), p.S)
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    # Compare amplitudes on the scale of the wavefunction (largest |psi| = 1). The GPU forms
    # each pre-activation in FP32 and the oracle in FP64; when a value lies within FP32 rounding
    # of a BF16 rounding boundary the two sides round the activation to neighbouring BF16
    # values (0.4% apart), which moves small amplitudes by up to ~1e-3 relative. A nearly
    # singular block also loses relative accuracy in FP32 LU. Neither matters on the
    # wavefunction scale, which is what E_S sees (gated at 1e-6 Ha in the energy test).
    M = rla.max()
    pg = sg * np.exp(la - M)
    pr = rsg * np.exp(rla - M)
    assert np.abs(pg - pr).max() < 2e-5, np.abs(pg - pr).max()
    big = np.abs(pr) > 1e-2
    assert np.array_equal(sg[big], rsg[big])
    assert np.abs(la - rla)[big].max() < 1e-3
    d = np.abs(la - rla)
    assert np.median(d) < 1e-5 and np.quantile(d, 0.99) < 5e-3


@pytest.mark.parametrize("name", ["tiny_n10"])
def test_energy_grad_fp64(name):
    need_gpu()
    N, p, P, net = _setup(name, False)
    dets = to_dev(p.S)
    csr = N.connections(P, dets)
    out, grad, psi = N.energy_grad(P, net, csr, dets)
    ref_csr = O.hss(p.wl.norb, p.h, p.eri, p.S)
    ref = O.energy_grad(O.Net(p.net), p.S, ref_csr)
    out = out.cpu().numpy()
    assert abs(out[0] - ref["E"]) < 1e-8
    assert abs(out[2] - ref["D"]) < 1e-10 * ref["D"]
    assert out[3] == pytest.approx(ref["maxlog"], abs=1e-11)
    assert np.abs(psi.cpu().numpy() - ref["psi"]).max() < 1e-10
    g = grad.cpu().numpy()
    rel = np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"])
    assert rel < 1e-9, rel


def test_energy_grad_mixed_vs_quantised_oracle():
    need_gpu()
    N, p, P, net = _setup("small_n16", True)
    dets = to_dev(p.S)
    csr = N.connections(P, dets)
    out, grad, psi = N.energy_grad(P, net, csr, dets)
    ref_csr = O.hss(16, p.h, p.eri, p.S)
    refq = O.energy_grad(O.Net(p.net, quant=True), p.S, ref_csr)
    out = out.cpu().numpy()
    assert abs(out[0] - refq["E"]) < 1e-6, out[0] - refq["E"]
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - refq["grad"]) / np.linalg.norm(refq["grad"])
    assert rel < 1e-2, rel


def test_energy_from_psi_eigenvector():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    csr = N.connections(P, to_dev(p.S))
    ref = O.hss(10, p.h, p.eri, p.S)
    w, V = np.linalg.eigh(ref.to_scipy().toarray())
    out, v = N.energy_from_psi(csr, torch.from_numpy(V[:, 0] * 2.5).cuda())
    out = out.cpu().numpy()
    assert abs(out[0] - w[0]) < 1e-10
    ref_out, ref_v = O.energy_from_psi(ref, V[:, 0] * 2.5)
    assert np.abs(v.cpu().numpy() - ref_v).max() < 1e-12


def test_gradient_central_differences_gpu():
    """GPU adjoint against central differences of the GPU energy (FP64 form, h = 1e-5, 64
    parameters chosen with seed 7)."""
    need_gpu()
    N, p, P, net = _setup("tiny_n10", False)
    dets = to_dev(p.S)
    csr = N.connections(P, dets)
    _, grad, _ = N.energy_grad(P, net, csr, dets)
    g = grad.cpu().numpy()
    flat_views = [t.view(-1) for t in net.params[:6]]
    sizes = [t.numel() for t in flat_views]
    offs = np.cumsum([0] + sizes)
    rng = np.random.default_rng(7)
    pick = rng.choice(offs[-1], size=64, replace=False)
    fd = []
    for k in pick:
        li = int(np.searchsorted(offs, k, side="right") - 1)
        j = int(k - offs[li])
        t = flat_views[li]
        orig = t[j].item()
        t[j] = orig + 1e-5
        ep = N.energy_grad(P, net, csr, dets, with_grad=False)[0][0].item()
        t[j] = orig - 1e-5
        em = N.energy_grad(P, net, csr, dets, with_grad=False)[0][0].item()
        t[j] = orig
        fd.append((ep - em) / 2e-5)
    fd = np.array(fd)
    rel = np.linalg.norm(fd - g[pick]) / np.linalg.norm(g[pick])
    assert rel < 1e-6, rel


def test_autograd_function():
    need_gpu()
    N, p, P, net = _setup("tiny_n10", False)
    dets = to_dev(p.S)
    csr = N.connections(P, dets)
    for t in net.params[:6]:
        t.requires_grad_(True)
    E = N.energy(P, net, csr, dets)
    E.backward()
    _, grad, _ = N.energy_grad(P, net, csr, dets)
    got = torch.cat([t.grad.reshape(-1) for t in net.params[:6]])
    assert torch.equal(got, grad)


def test_amplitudes_other_shapes():
    need_gpu()
    N = nqs()
    for norb, na, nb, nS in [(12, 5, 4, 300), (20, 7, 7, 513)]:
        p, nb = small_problem(norb, na, nS, 50 + norb, hidden=(48, 40), nb=nb)
        P = N.Problem(norb, na, nb, p.h, p.eri)
        net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
        la, sg, _ = N.amplitudes(P, net, to_dev(p.S))
        rla, rsg = O.amplitudes(O.Net(p.net), p.S)
        assert np.array_equal(sg.cpu().numpy(), rsg)
        assert np.abs(la.cpu().numpy() - rla).max() < 1e-10


@pytest.mark.parametrize("mixed", [False, True])
def test_micro_batched_gradient_recomputation(mixed):
    """Sets larger than the micro-batch: amplitudes batch by batch, the gradient recomputes each
    batch's activations and accumulates. The energy is identical to the one-batch evaluation;
    the gradient agrees to the rounding of the different reduction split."""
    need_gpu()
    N, p, P, net = _setup("small_n16" if mixed else "tiny_n10", mixed)
    dets = to_dev(p.S)
    csr = N.connections(P, dets)
    dt = N.NQS_MIXED if mixed else N.NQS_FP64
    o1, g1, _ = N.energy_grad(P, net, csr, dets, o=N.opts(precision=dt, validate=0))
    ob, gb, _ = N.energy_grad(P, net, csr, dets, o=N.opts(precision=dt, validate=0,
                                                          batch_log2=8))
    assert ob[0].item() == o1[0].item()
    rel = (torch.linalg.norm(gb.double() - g1.double()) / torch.linalg.norm(g1.double())).item()
    assert rel < (1e-5 if mixed else 1e-12), rel


@pytest.mark.parametrize("norb,n", [(18, 13), (20, 16), (22, 20), (26, 24), (31, 28)])
def test_mixed_blocks_of_13_to_32_rows_vs_quantised_oracle(norb, n):
    """Spin blocks of 13..32 rows in the mixed form: the FP32 LU with four blocks per warp and
    up to three rows per lane at 13..24 rows (scalar loads at 13, a partial third row at 20,
    16-byte loads at 16, 20 and 24), one lane per row at 28. Amplitudes, E_S and the gradient,
    which goes through the block inverses, against the quantisation-matched oracle."""
    need_gpu()
    N = nqs()
    p, _ = small_problem(norb, n, 400, 70 + norb, hidden=(64, 64))
    P = N.Problem(norb, n, n, p.h, p.eri)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    dets = to_dev(p.S)
    la, sg, _ = N.amplitudes(P, net, dets)
    onet = O.Net(p.net, quant=True)
    rla, rsg = O.amplitudes(onet, p.S)
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    M = rla.max()
    assert np.abs(sg * np.exp(la - M) - rsg * np.exp(rla - M)).max() < 2e-5
    csr = N.connections(P, dets)
    out, grad, _ = N.energy_grad(P, net, csr, dets)
    ref = O.energy_grad(onet, p.S, O.hss(norb, p.h, p.eri, p.S))
    assert abs(out[0].item() - ref["E"]) < 1e-6
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) < 1e-2


def test_mixed_singular_blocks_of_24_rows():
    """Output layer zero: Phi = Phi0 (identity columns), so every configuration other than the
    reference has a singular block. Those get sign 0 and log|psi| = -inf, the reference gets
    psi = 1, E_S = H_00 and the gradient stays finite."""
    need_gpu()
    N = nqs()
    norb, n = 30, 24
    h, eri, _ = synth.integrals(norb, 2 * norb, 9, 3.0)
    S = synth.select_S(norb, n, 300)
    netp = synth.net_params(norb, n, n, (64, 64), 9, out_scale=0.0)
    P = N.Problem(norb, n, n, h, eri)
    net = N.Net(P, N.net_tensors(netp, N.NQS_MIXED), N.NQS_MIXED)
    dets = to_dev(S)
    la, sg, _ = N.amplitudes(P, net, dets)
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    hf = (S[:, 0] == (1 << n) - 1) & (S[:, 1] == (1 << n) - 1)
    assert hf.sum() == 1
    assert sg[hf][0] == 1 and abs(la[hf][0]) < 1e-12
    assert np.all(sg[~hf] == 0) and np.all(np.isneginf(la[~hf]))
    csr = N.connections(P, dets)
    out, grad, _ = N.energy_grad(P, net, csr, dets)
    H00 = O.hss_rows(norb, h, eri, S, int(np.argmax(hf)), int(np.argmax(hf)) + 1)[2][0]
    assert abs(out[0].item() - H00) < 1e-10 * abs(H00)
    assert bool(torch.isfinite(grad).all())
