"""Parity at the shape of Cr2 CAS(24e,30o) (30 orbitals, 12a+12b): the full-size workload
(|S| = 131072, 67284 excitations per determinant, 8.8e9 connections) on sampled outputs the
oracle computes one by one, PT2 invariants at full size, and full parity on a 30-orbital
problem with a smaller S."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr2():
    need_gpu()
    N = nqs()
    p = synth.make_problem("cr2_24e30o")
    P = problem_for(N, p)
    dets = to_dev(p.S)
    return N, p, P, dets


def test_full_size_hss_sampled_rows(cr2):
    N, p, P, dets = cr2
    csr = N.connections(P, dets)
    assert csr.n_enumerated == len(p.S) * 67284
    rp, col, val = csr.host()
    for r0 in (0, 65536, len(p.S) - 64):
        r1 = r0 + 64
        orp, ocol, oval = O.hss_rows(30, p.h, p.eri, p.S, r0, r1)
        a, b = rp[r0], rp[r1]
        assert np.array_equal(rp[r0:r1 + 1] - a, orp)
        assert np.array_equal(col[a:b], ocol)
        assert np.array_equal(val[a:b], oval)


def test_full_size_mixed_amplitudes_sampled(cr2):
    N, p, P, dets = cr2
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    la, sg, _ = N.amplitudes(P, net, dets)
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    pick = np.sort(np.random.default_rng(3).choice(len(p.S), 1024, replace=False))
    rla, rsg = O.amplitudes(O.Net(p.net, quant=True), p.S[pick])
    M = la.max()
    pg = sg[pick] * np.exp(la[pick] - M)
    pr = rsg * np.exp(rla - M)
    assert np.abs(pg - pr).max() < 2e-5
    d = np.abs(la[pick] - rla)
    assert np.median(d) < 1e-5 and np.quantile(d, 0.99) < 5e-3


def test_full_size_mixed_energy_grad_vs_quantised_oracle(cr2):
    """Mixed form at the full cr2_24e30o size (|S| = 131072): E_S within 1e-6 Ha and the
    gradient within 1e-2 relative L2 of the oracle's quantisation-matched evaluation (weights and
    activations rounded to BF16, FP64 arithmetic). The oracle evaluates the network, the
    determinants, E_S and the adjoint itself; it takes H_SS from the library's CSR copied to the
    host (its own H_SS would need 8.8e9 host lookups), whose rows equal the oracle's Slater-Condon
    rows bit for bit on the three row blocks checked here."""
    N, p, P, dets = cr2
    csr = N.connections(P, dets)
    rp, col, val = csr.host()
    for r0 in (0, 70001, len(p.S) - 32):
        orp, ocol, oval = O.hss_rows(30, p.h, p.eri, p.S, r0, r0 + 32)
        a, b = rp[r0], rp[r0 + 32]
        assert np.array_equal(rp[r0:r0 + 33] - a, orp)
        assert np.array_equal(col[a:b], ocol) and np.array_equal(val[a:b], oval)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    out, grad, _ = N.energy_grad(P, net, csr, dets)
    E = out[0].item()
    g = grad.cpu().numpy().astype(np.float64)
    csr.free()
    refq = O.energy_grad(O.Net(p.net, quant=True), p.S, O.CSR(rp, col, val, 0))
    assert abs(E - refq["E"]) < 1e-6, E - refq["E"]
    rel = np.linalg.norm(g - refq["grad"]) / np.linalg.norm(refq["grad"])
    assert rel < 1e-2, rel


def test_full_size_pt2_independent_of_bucketing(cr2):
    """PT2 over the 8.8e9-connection space: the sums and the unique count do not depend on how
    the connected space is split into hash buckets."""
    N, p, P, dets = cr2
    psi = torch.from_numpy(np.random.default_rng(9).normal(size=len(p.S))).cuda()
    r1 = N.pt2(P, dets, psi, -40.0, buckets=12)
    r2 = N.pt2(P, dets, psi, -40.0, buckets=16)
    assert r1["n_emitted"] == r2["n_emitted"] == len(p.S) * 67284
    assert r1["n_unique"] == r2["n_unique"] > 0
    assert abs(r1["ext"] - r2["ext"]) < 1e-11 * abs(r1["ext"])
    assert abs(r1["int"] - r2["int"]) < 1e-11 * abs(r1["int"])
    assert abs(r1["partials"][:, 0].sum() - r1["ext"]) < 1e-11 * abs(r1["ext"])


def test_norb30_smaller_S_full_parity():
    """30 orbitals, 12a+12b, |S| = 1500: H_SS, E_S + gradient (FP64 form) and one PT2 bucket of
    four against the oracle."""
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(30, 60, 2, 5.0)
    S = synth.select_S(30, 12, 1500)
    params = synth.net_params(30, 12, 12, (64, 48), 102)
    P = N.Problem(30, 12, 12, h, eri)
    dets = to_dev(S)
    csr = N.connections(P, dets)
    ref = O.hss(30, h, eri, S)
    rp, col, val = csr.host()
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    assert np.array_equal(val, ref.val)
    net = N.Net(P, N.net_tensors(params, N.NQS_FP64), N.NQS_FP64)
    out, grad, psi = N.energy_grad(P, net, csr, dets)
    r = O.energy_grad(O.Net(params), S, ref)
    assert abs(out[0].item() - r["E"]) < 1e-8
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - r["grad"]) < 1e-9 * np.linalg.norm(r["grad"])
    got = N.pt2(P, dets, psi, out[0].item(), buckets=4)
    rb = O.pt2(30, h, eri, S, r["psi"], r["E"], 4, 0)
    assert abs(got["partials"][0, 0] - rb["ext"]) < 1e-10 * abs(rb["ext"])
    assert abs(got["partials"][0, 1] - rb["int"]) < 1e-10 * max(1e-30, abs(rb["int"]))


@pytest.fixture(scope="module")
def cr2_48():
    need_gpu()
    N = nqs()
    p = synth.make_problem("cr2_48e42o")
    P = problem_for(N, p)
    dets = to_dev(p.S)
    return N, p, P, dets


def test_cr2_48e42o_full_size_hss_amplitudes_energy(cr2_48):
    """42 orbitals, 24a+24b, |S| = 2^20 (2.85e11 connections): H_SS on sampled rows bit-exactly,
    mixed-form amplitudes on sampled determinants, and E_S consistent with the matrix."""
    N, p, P, dets = cr2_48
    csr = N.connections(P, dets)
    assert csr.n_enumerated == len(p.S) * 271944
    for r0 in (0, 500000, len(p.S) - 8):
        rp, col, val = csr.host_rows(r0, r0 + 8)
        orp, ocol, oval = O.hss_rows(42, p.h, p.eri, p.S, r0, r0 + 8)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
        assert np.array_equal(val, oval)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    out, grad, psi = N.energy_grad(P, net, csr, dets)
    la, sg, _ = N.amplitudes(P, net, dets)
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    pick = np.sort(np.random.default_rng(5).choice(len(p.S), 128, replace=False))
    rla, rsg = O.amplitudes(O.Net(p.net, quant=True), p.S[pick])
    M = la.max()
    assert np.abs(sg[pick] * np.exp(la[pick] - M) - rsg * np.exp(rla - M)).max() < 2e-5
    e2, _ = N.energy_from_psi(csr, psi)
    assert abs(e2[0].item() - out[0].item()) < 1e-12 * abs(out[0].item())
    assert bool(torch.isfinite(grad).all())
    csr.free()


def test_norb42_pt2_two_word_keys():
    """42 orbitals, 24a+24b (84-bit PT2 keys), |S| = 150: one PT2 bucket of four against the
    oracle, and the unique count over all buckets."""
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(42, 84, 3, 3.0)
    S = synth.select_S(42, 24, 150)
    P = N.Problem(42, 24, 24, h, eri)
    psi = np.random.default_rng(2).normal(size=len(S))
    got = N.pt2(P, to_dev(S), torch.from_numpy(psi).cuda(), -60.0, buckets=4)
    ref = O.pt2(42, h, eri, S, psi, -60.0, 4, 1)
    assert abs(got["partials"][1, 0] - ref["ext"]) < 1e-10 * abs(ref["ext"])
    assert abs(got["partials"][1, 1] - ref["int"]) < 1e-10 * max(1e-300, abs(ref["int"]))
    assert got["n_emitted"] == len(S) * 271944


def test_amplitudes_beyond_one_micro_batch():
    """nqs_amplitudes on 1.2 million configurations (two micro-batches of 2^20): sampled rows on
    both sides of the batch boundary equal the oracle's FP64 amplitudes."""
    need_gpu()
    N = nqs()
    norb, n = 16, 8
    h, eri, _ = synth.integrals(norb, 2 * norb, 1, 3.0)
    T = synth.select_S(norb, n, 1_200_000)
    T = T[np.random.default_rng(0).permutation(len(T))]  # amplitudes need no ordering
    net = synth.net_params(norb, n, n, (64, 64), 21)
    P = N.Problem(norb, n, n, h, eri)
    gnet = N.Net(P, N.net_tensors(net, N.NQS_FP64), N.NQS_FP64)
    la, sg, _ = N.amplitudes(P, gnet, to_dev(T), o=N.opts(validate=0))
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    B = 1 << 20
    rows = np.r_[0:500, B - 500:B + 500, len(T) - 500:len(T)]
    rla, rsg = O.amplitudes(O.Net(net), T[rows])
    assert np.array_equal(sg[rows], rsg)
    assert np.abs(la[rows] - rla).max() < 1e-9


def test_cr2_48e42o_full_size_pt2_unique_sampled(cr2_48):
    """42 orbitals, |S| = 2^20: one hash bucket of 4096 of the deduplicated external set of Eq.
    (pt2_correction) at full size, checked on samples the oracle computes one by one: for sampled
    x' of the GPU's set, x' is outside S, in the bucket, and c(x') = sum over the members y of S
    connected to x' of H_x'y psi_y (oracle elements); and sampled excitations x' of members of S
    that are outside S and in the bucket appear in the GPU's set."""
    N, p, P, dets = cr2_48
    S = p.S
    rng = np.random.default_rng(21)
    psi = rng.normal(size=len(S))
    B, b = 4096, 0
    keys, c = N.pt2_unique(P, dets, torch.from_numpy(psi).cuda(), B, b)
    keys, c = keys.cpu().numpy(), c.cpu().numpy()
    assert len(keys) > 1000
    # ascending by (a, b), unique
    assert np.all((keys[1:, 0] > keys[:-1, 0]) |
                  ((keys[1:, 0] == keys[:-1, 0]) & (keys[1:, 1] > keys[:-1, 1])))
    sh = 42
    index = {int(a) << sh | int(bb): i for i, (a, bb) in enumerate(S.tolist())}

    def in_set(ya, yb):  # keys ascending by (a, b)
        lo = np.searchsorted(keys[:, 0], np.uint64(ya), "left")
        hi = np.searchsorted(keys[:, 0], np.uint64(ya), "right")
        return bool(np.any(keys[lo:hi, 1] == np.uint64(yb)))

    for k in rng.choice(len(keys), 24, replace=False):
        xa, xb = int(keys[k, 0]), int(keys[k, 1])
        assert (xa << sh | xb) not in index
        assert O.bucket(xa, xb, B) == b
        ref, scale = 0.0, 0.0
        for ya, yb in O.excitations(42, xa, xb).tolist():
            j = index.get(int(ya) << sh | int(yb))
            if j is None:
                continue
            v, _ = O.element(42, p.h, p.eri, (ya, yb), (xa, xb))
            ref += v * psi[j]
            scale += abs(v * psi[j])
        assert abs(c[k] - ref) <= 1e-12 * scale + 1e-300, (k, c[k], ref)
    # completeness: outside-S excitations of sampled members of S, in the bucket, are present
    found = 0
    for r in rng.choice(len(S), 64, replace=False):
        ex = O.excitations(42, int(S[r, 0]), int(S[r, 1]))
        for ya, yb in ex[rng.choice(len(ex), 2000, replace=False)].tolist():
            key = int(ya) << sh | int(yb)
            if key in index or O.bucket(ya, yb, B) != b:
                continue
            assert in_set(ya, yb), (ya, yb)
            found += 1
    assert found > 0


def test_cr2_48e42o_full_size_screened_pt2_unique_sampled(cr2_48):
    """The screened form at 42 orbitals, |S| = 2^20, eps = 1e-6 on normalised amplitudes: one
    hash bucket of 4096, checked on samples. For sampled x' of the GPU's set: outside S, in the
    bucket, and c(x') = the sum over members y of S connected to x' of the contributions
    H_x'y psi_y with |H_x'y| |psi_y| >= eps (oracle elements), at least one of them kept; and
    kept contributions to sampled excitations of members of S land on x' in the set."""
    N, p, P, dets = cr2_48
    S = p.S
    rng = np.random.default_rng(23)
    psi = rng.normal(size=len(S))
    psi /= np.linalg.norm(psi)
    eps, B, b = 1e-6, 4096, 0
    keys, c = N.pt2_unique(P, dets, torch.from_numpy(psi).cuda(), B, b, eps=eps)
    keys, c = keys.cpu().numpy(), c.cpu().numpy()
    assert len(keys) > 100
    sh = 42
    index = {int(a) << sh | int(bb): i for i, (a, bb) in enumerate(S.tolist())}

    def in_set(ya, yb):  # keys ascending by (a, b)
        lo = np.searchsorted(keys[:, 0], np.uint64(ya), "left")
        hi = np.searchsorted(keys[:, 0], np.uint64(ya), "right")
        return bool(np.any(keys[lo:hi, 1] == np.uint64(yb)))

    for k in rng.choice(len(keys), 24, replace=False):
        xa, xb = int(keys[k, 0]), int(keys[k, 1])
        assert (xa << sh | xb) not in index
        assert O.bucket(xa, xb, B) == b
        ref, scale, kept = 0.0, 0.0, 0
        for ya, yb in O.excitations(42, xa, xb).tolist():
            j = index.get(int(ya) << sh | int(yb))
            if j is None:
                continue
            v, _ = O.element(42, p.h, p.eri, (ya, yb), (xa, xb))
            if abs(v) * abs(psi[j]) >= eps:
                ref += v * psi[j]
                scale += abs(v * psi[j])
                kept += 1
        assert kept > 0
        assert abs(c[k] - ref) <= 1e-12 * scale, (k, c[k], ref)
    found = 0
    for r in rng.choice(len(S), 256, replace=False):
        ya, yb = int(S[r, 0]), int(S[r, 1])
        ex = O.excitations(42, ya, yb)
        for xa, xb in ex[rng.choice(len(ex), 2000, replace=False)].tolist():
            if (int(xa) << sh | int(xb)) in index or O.bucket(xa, xb, B) != b:
                continue
            v, _ = O.element(42, p.h, p.eri, (ya, yb), (xa, xb))
            if abs(v) * abs(psi[r]) >= eps:
                assert in_set(xa, xb), (xa, xb)
                found += 1
    assert found > 0
