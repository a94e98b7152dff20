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
