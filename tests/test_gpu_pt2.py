"""GPU parity of the Epstein-Nesbet PT2 pipeline (emission, radix sort, dedup, segmented
reduction) against the oracle, through the C ABI: unique counts bit-exact, energies within
1e-8 Ha (FP64)."""
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
