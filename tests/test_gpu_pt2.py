"""GPU parity of the Epstein-Nesbet PT2 pipeline (emission, radix sort, dedup, segmented
reduction) against the oracle, through the C ABI: the unique set bit-exact key by key, c(x')
element by element, energies within 1e-8 Ha (FP64); the mixed form's external term within
1e-6 Ha of the quantisation-matched oracle."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, small_problem, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _psi_E(p):
    csr = O.hss(p.wl.norb, p.h, p.eri, p.S)
    r = O.energy_grad(O.Net(p.net), p.S, csr, with_grad=False)
    return r["psi"], r["E"]


def test_pt2_tiny_all_buckets():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    psi, E = _psi_E(p)
    ref = O.pt2(10, p.h, p.eri, p.S, psi, E)
    got = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), E)
    assert got["n_unique"] == ref["n_unique"]
    assert got["n_emitted"] == len(p.S) * O.n_excitations(10, 5, 5)
    assert abs(got["ext"] - ref["ext"]) < 1e-12
    assert abs(got["int"] - ref["int"]) < 1e-12


@pytest.mark.parametrize("B", [3, 8])
def test_pt2_buckets_match_oracle(B):
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    psi, E = _psi_E(p)
    got = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), E, buckets=B)
    tot_u = 0
    for b in range(B):
        ref = O.pt2(10, p.h, p.eri, p.S, psi, E, B, b)
        assert abs(got["partials"][b, 0] - ref["ext"]) < 1e-12
        assert abs(got["partials"][b, 1] - ref["int"]) < 1e-12
        tot_u += ref["n_unique"]
    assert got["n_unique"] == tot_u


def test_pt2_small_bucket_sample():
    """Full-size small_n16 problem: one bucket of eight, compared with the oracle restricted to
    the same bucket (the oracle finishes it in seconds)."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    rng = np.random.default_rng(5)
    psi = rng.normal(size=len(p.S))
    E = -20.0
    got = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), E, buckets=8)
    for b in (0, 5):
        ref = O.pt2(16, p.h, p.eri, p.S, psi, E, 8, b)
        assert abs(got["partials"][b, 0] - ref["ext"]) < 1e-9 * max(1, abs(ref["ext"]))
        assert abs(got["partials"][b, 1] - ref["int"]) < 1e-9 * max(1, abs(ref["int"]))


def test_pt2_full_space_is_zero():
    need_gpu()
    N = nqs()
    norb, n = 6, 3
    h, eri, _ = synth.integrals(norb, 12, 2, 3.0)
    F = synth.full_space(norb, n)
    P = N.Problem(norb, n, n, h, eri)
    psi = np.random.default_rng(1).normal(size=len(F))
    got = N.pt2(P, to_dev(F), torch.from_numpy(psi).cuda(), -5.0)
    assert got["ext"] == 0.0 and got["n_unique"] == 0
    ref = O.pt2(norb, h, eri, F, psi, -5.0)
    assert abs(got["int"] - ref["int"]) < 1e-10 * abs(ref["int"])


def test_pt2_ragged_shapes():
    need_gpu()
    N = nqs()
    for norb, na, nb, nS in [(9, 4, 3, 37), (13, 5, 5, 1001)]:
        p, nb = small_problem(norb, na, nS, 70 + norb, nb=nb)
        P = N.Problem(norb, na, nb, p.h, p.eri)
        psi = np.random.default_rng(norb).normal(size=len(p.S))
        got = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), -3.0, buckets=2)
        ref = O.pt2(norb, p.h, p.eri, p.S, psi, -3.0)
        assert got["n_unique"] == ref["n_unique"]
        assert abs(got["ext"] - ref["ext"]) < 1e-11 * max(1, abs(ref["ext"]))
        assert abs(got["int"] - ref["int"]) < 1e-11 * max(1, abs(ref["int"]))


def _norm_psi_E(p):
    psi, E = _psi_E(p)
    return psi / np.linalg.norm(psi), E


@pytest.mark.parametrize("eps", [1e-5, 1e-4, 1e-3])
def test_screened_pt2_tiny_matches_oracle(eps):
    """External sum over the screened perturbative set (contributions |H_x'y psi_y| >= eps):
    the set (its size) exactly, energies within 1e-12 Ha; the internal term stays exact."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    psi, E = _norm_psi_E(p)
    ref = O.pt2(10, p.h, p.eri, p.S, psi, E, eps=eps)
    full = O.pt2(10, p.h, p.eri, p.S, psi, E)
    got = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), E, o=N.opts(eps_pt2=eps))
    assert got["n_unique"] == ref["n_unique"] < full["n_unique"]
    assert abs(got["ext"] - ref["ext"]) < 1e-12
    assert abs(got["int"] - ref["int"]) < 1e-12
    assert abs(got["int"] - full["int"]) < 1e-12
    for B in (3, 8):
        gb = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), E,
                   o=N.opts(eps_pt2=eps, buckets=B))
        assert gb["n_unique"] == ref["n_unique"]
        assert abs(gb["ext"] - ref["ext"]) < 1e-12 and abs(gb["int"] - ref["int"]) < 1e-12


@pytest.mark.parametrize("norb,n,nS,eps", [(16, 8, 2000, 1e-5), (30, 12, 400, 1e-5),
                                           (42, 24, 80, 1e-5)])
def test_screened_pt2_key_widths_match_oracle(norb, n, nS, eps):
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(norb, 2 * norb, norb, 3.0)
    S = synth.select_S(norb, n, nS)
    rng = np.random.default_rng(norb)
    psi = rng.standard_normal(len(S)) * np.exp(-rng.uniform(0, 6, len(S)))
    psi /= np.linalg.norm(psi)
    E = -30.0  # below every H_xx of these integrals: every denominator has the same sign
    P = N.Problem(norb, n, n, h, eri)
    ref = O.pt2(norb, h, eri, S, psi, E, eps=eps)
    got = N.pt2(P, to_dev(S), torch.from_numpy(psi).cuda(), E, o=N.opts(eps_pt2=eps))
    assert got["n_unique"] == ref["n_unique"]
    assert abs(got["ext"] - ref["ext"]) <= 1e-10 * abs(ref["ext"])
    assert abs(got["int"] - ref["int"]) <= 1e-10 * abs(ref["int"])


def test_screened_pt2_full_size_bucket_invariance():
    """cr2_24e30o, all 131072 configurations, eps = 1e-6 on the normalised amplitudes: one
    bucket and five buckets give the same screened set and the same energies."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("cr2_24e30o")
    P = problem_for(N, p)
    la, sg = O.amplitudes(O.Net(p.net), p.S)
    psi = sg * np.exp(la - la.max())
    psi /= np.linalg.norm(psi)
    E = -60.0
    d, ps = to_dev(p.S), torch.from_numpy(psi).cuda()
    a = N.pt2(P, d, ps, E, o=N.opts(eps_pt2=1e-6, validate=0))
    b = N.pt2(P, d, ps, E, o=N.opts(eps_pt2=1e-6, buckets=5, validate=0))
    assert a["n_unique"] == b["n_unique"] > 0
    assert abs(a["ext"] - b["ext"]) <= 1e-10 * abs(a["ext"])
    assert abs(a["int"] - b["int"]) <= 1e-10 * abs(a["int"])


def test_automatic_bucket_count():
    """opts.buckets = 0: the library picks the bucket count (here one: the tiny case fits) and
    reports it; partials are not available then."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    psi, E = _norm_psi_E(p)
    d, ps = to_dev(p.S), torch.from_numpy(psi).cuda()
    for eps in (0.0, 1e-4):
        one = N.pt2(P, d, ps, E, o=N.opts(eps_pt2=eps, buckets=1))
        auto = N.pt2(P, d, ps, E, o=N.opts(eps_pt2=eps, buckets=0))
        assert auto["buckets"] == 1 and auto["partials"] is None
        assert auto["n_unique"] == one["n_unique"]
        assert auto["ext"] == one["ext"] and auto["int"] == one["int"]


@pytest.mark.parametrize("norb,n,nS,eps", [(10, 5, 1000, 1e-4), (16, 8, 2000, 1e-5),
                                           (42, 24, 80, 1e-5)])
def test_screened_pt2_with_hss_matches_oracle(norb, n, nS, eps):
    """nqs_pt2_hss: the screened internal term from the caller's H_SS (one SpMV without the
    diagonal) equals the oracle's and nqs_pt2's; the external sum is the same computation."""
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(norb, 2 * norb, norb + 1, 3.0)
    S = synth.select_S(norb, n, nS)
    rng = np.random.default_rng(norb + 1)
    psi = rng.standard_normal(len(S)) * np.exp(-rng.uniform(0, 6, len(S)))
    psi /= np.linalg.norm(psi)
    E = -30.0
    P = N.Problem(norb, n, n, h, eri)
    d, ps = to_dev(S), torch.from_numpy(psi).cuda()
    csr = N.connections(P, d)
    ref = O.pt2(norb, h, eri, S, psi, E, eps=eps)
    got = N.pt2(P, d, ps, E, o=N.opts(eps_pt2=eps), hss=csr)
    plain = N.pt2(P, d, ps, E, o=N.opts(eps_pt2=eps))
    assert got["n_unique"] == ref["n_unique"] == plain["n_unique"]
    assert got["ext"] == plain["ext"]
    assert abs(got["ext"] - ref["ext"]) <= 1e-10 * abs(ref["ext"])
    assert abs(got["int"] - ref["int"]) <= 1e-10 * abs(ref["int"])
    assert abs(got["int"] - plain["int"]) <= 1e-12 * abs(plain["int"])
    # unscreened: H_SS is not needed and the result is nqs_pt2's
    a = N.pt2(P, d, ps, E, hss=csr)
    b = N.pt2(P, d, ps, E)
    assert a["ext"] == b["ext"] and a["int"] == b["int"]
    # a matrix over other configurations is rejected
    with pytest.raises(N.NQSError):
        N.pt2(P, d[:-1], ps[:-1], E, o=N.opts(eps_pt2=eps), hss=csr)
    csr.free()


def test_pt2_per_bucket_passes_match_single_pass():
    """More buckets than one counting pass covers (1030 > 1024): every bucket is counted and
    emitted by its own pass over S. The unique count and the energies equal those of the
    single-bucket pipeline and of the all-buckets-resident pipeline (B = 5)."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    psi, E = _psi_E(p)
    d, ps = to_dev(p.S), torch.from_numpy(psi).cuda()
    one = N.pt2(P, d, ps, E, buckets=1)
    many = N.pt2(P, d, ps, E, buckets=1030)
    five = N.pt2(P, d, ps, E, buckets=5)
    for r in (many, five):
        assert r["n_unique"] == one["n_unique"]
        assert r["n_emitted"] == one["n_emitted"]
        assert abs(r["ext"] - one["ext"]) < 1e-12 and abs(r["int"] - one["int"]) < 1e-12
    assert abs(many["partials"][:, 0].sum() - many["ext"]) < 1e-12


def _unique_tol(c_ref):
    """The oracle adds a run's terms one by one in FP64 in emission order, the library in FP64
    in the same order but grouped by lanes of eight elements (each sum has error at most
    k 2^-53 sum|terms|, k the run length); 1e-12 of the largest |c| covers k <= 5792 terms of
    at most that size with margin."""
    return 1e-12 * max(1.0, float(np.abs(c_ref).max(initial=0.0)))


@pytest.mark.parametrize("name,B,b", [("tiny_n10", 1, 0), ("tiny_n10", 3, 1),
                                      ("small_n16", 8, 3)])
def test_pt2_unique_set_matches_oracle(name, B, b):
    """The deduplicated external set of Eq. (pt2_correction) key by key: every x' of C minus S
    (of one hash bucket) in ascending order equals the oracle's bit for bit, and c(x') element
    by element."""
    need_gpu()
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    if name == "tiny_n10":
        psi, E = _psi_E(p)
    else:
        psi = np.random.default_rng(9).normal(size=len(p.S))
        E = -20.0
    keys, c = N.pt2_unique(P, to_dev(p.S), torch.from_numpy(psi).cuda(), B, b)
    rk, rc, info = O.pt2_unique(p.wl.norb, p.h, p.eri, p.S, psi, E, B, b if B > 1 else -1)
    keys = keys.cpu().numpy()
    assert keys.shape == rk.shape and len(rk) > 0
    assert np.array_equal(keys, rk)
    c = c.cpu().numpy()
    assert np.abs(c - rc).max() <= _unique_tol(rc), np.abs(c - rc).max()
    got = N.pt2(P, to_dev(p.S), torch.from_numpy(psi).cuda(), E, buckets=B)
    assert abs(got["partials"][b, 0] - info["ext"]) <= 1e-11 * max(1.0, abs(info["ext"]))


@pytest.mark.parametrize("name,B,b,eps", [("tiny_n10", 1, 0, 1e-3), ("tiny_n10", 3, 1, 1e-4),
                                          ("small_n16", 8, 3, 1e-5)])
def test_pt2_unique_screened_set_matches_oracle(name, B, b, eps):
    """The screened external set (Sec. 3.3) key by key: the x' of C minus S (of one hash bucket)
    reached by at least one contribution |H_x'y psi_y| >= eps equal the oracle's bit for bit, and
    c(x'), the sum of the kept contributions, element by element."""
    need_gpu()
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    psi = np.random.default_rng(13).normal(size=len(p.S))
    psi /= np.linalg.norm(psi)
    keys, c = N.pt2_unique(P, to_dev(p.S), torch.from_numpy(psi).cuda(), B, b, eps=eps)
    rk, rc, _ = O.pt2_unique(p.wl.norb, p.h, p.eri, p.S, psi, -20.0, B, b if B > 1 else -1,
                             eps=eps)
    full, _, _ = O.pt2_unique(p.wl.norb, p.h, p.eri, p.S, psi, -20.0, B, b if B > 1 else -1)
    assert 0 < len(rk) < len(full)  # the cut removes some x' entirely
    keys = keys.cpu().numpy()
    assert np.array_equal(keys, rk)
    c = c.cpu().numpy()
    assert np.abs(c - rc).max() <= _unique_tol(rc), np.abs(c - rc).max()


def test_pt2_unique_reports_size_and_rejects_bad_bucket():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    psi, _ = _psi_E(p)
    d, ps = to_dev(p.S), torch.from_numpy(psi).cuda()
    import ctypes as C
    n = C.c_int64(0)
    L = N.lib()
    st = L.nqs_pt2_unique(P.handle, d.data_ptr(), ps.data_ptr(), len(p.S), 1, 0, None, None, 0,
                          C.byref(n), None)
    assert st == N.NQS_ERR_ARG and n.value > 0
    assert L.nqs_pt2_unique(P.handle, d.data_ptr(), ps.data_ptr(), len(p.S), 2, 2, None, None, 0,
                            C.byref(n), None) == N.NQS_ERR_ARG


def test_pt2_mixed_form_vs_quantised_oracle():
    """The mixed-precision form end to end at small_n16 (BF16 network on the tensor cores, FP32
    LU, FP64 Hamiltonian side): GPU amplitudes -> E_S -> nqs_pt2, against the oracle's
    quantisation-matched pipeline (BF16-rounded weights and activations, FP64 arithmetic).
    E_S and the external term of Eq. (pt2_correction) are gated at 1e-6 Ha. The internal term
    divides by E - H_xx over S, which for this random network comes within 1.2e-3 Ha of zero:
    there a 1e-6 change of psi moves the term by ~1e-2 Ha, so no amplitude-level agreement can
    gate it at 1e-6 Ha. It is compared instead with the oracle evaluated on the GPU's own psi
    and E_S (one hash bucket of eight), to 1e-9 relative."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    dets = to_dev(p.S)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    csr = N.connections(P, dets)
    out, _, psi = N.energy_grad(P, net, csr, dets, with_grad=False)
    E = out[0].item()
    got = N.pt2(P, dets, psi, E, buckets=8)
    ref_csr = O.hss(16, p.h, p.eri, p.S)
    refq = O.energy_grad(O.Net(p.net, quant=True), p.S, ref_csr, with_grad=False)
    ref = O.pt2(16, p.h, p.eri, p.S, refq["psi"], refq["E"])
    assert abs(E - refq["E"]) < 1e-6, E - refq["E"]
    assert abs(got["ext"] - ref["ext"]) < 1e-6, got["ext"] - ref["ext"]
    psi_g = psi.cpu().numpy()
    r0 = O.pt2(16, p.h, p.eri, p.S, psi_g, E, 8, 0)
    assert abs(got["partials"][0, 1] - r0["int"]) <= 1e-9 * abs(r0["int"])
    assert abs(got["partials"][0, 0] - r0["ext"]) <= 1e-10 * abs(r0["ext"])


@pytest.mark.parametrize("name,chunk", [("tiny_n10", 8192), ("small_n16", 4_000_000)])
def test_pt2_hashed_passes_match(name, chunk):
    """PT2 over all of C minus S in hashed passes: with opts.buckets = 0 and a pair cap small
    enough that sorted buckets would traverse the connected space more than eight times, each
    pass accumulates the emissions of a range of fine buckets into a hash table of
    configurations in exact fixed point (several passes here). The unique count, the emitted
    count and both terms equal the single-bucket pipeline's, and the oracle's on tiny_n10."""
    need_gpu()
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    if name == "tiny_n10":
        psi, E = _psi_E(p)
    else:
        psi = np.random.default_rng(11).normal(size=len(p.S))
        E = -20.0
    d, ps = to_dev(p.S), torch.from_numpy(psi).cuda()
    one = N.pt2(P, d, ps, E, buckets=1)
    hashed = N.pt2(P, d, ps, E, o=N.opts(buckets=0, chunk=chunk))
    assert hashed["buckets"] > 1 and hashed["partials"] is None
    assert hashed["n_unique"] == one["n_unique"]
    assert hashed["n_emitted"] == one["n_emitted"] == len(p.S) * O.n_excitations(
        p.wl.norb, p.wl.nalpha, p.wl.nbeta)
    assert abs(hashed["ext"] - one["ext"]) <= 1e-12 * max(1.0, abs(one["ext"]))
    assert abs(hashed["int"] - one["int"]) <= 1e-12 * max(1.0, abs(one["int"]))
    if name == "tiny_n10":
        ref = O.pt2(10, p.h, p.eri, p.S, psi, E)
        assert hashed["n_unique"] == ref["n_unique"]
        assert abs(hashed["ext"] - ref["ext"]) < 1e-12 and abs(hashed["int"] - ref["int"]) < 1e-12
    again = N.pt2(P, d, ps, E, o=N.opts(buckets=0, chunk=chunk))
    assert again["ext"] == hashed["ext"] and again["int"] == hashed["int"]  # deterministic
