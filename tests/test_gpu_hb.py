"""GPU parity of the heat-bath screened perturbative set (Eq. hb_screen, Sec. 3.3) against the
oracle, through the C ABI: the selected configurations and their couplings
max_x |H_x'x psi_x| bit-exact (the sorted-table early exit on the GPU keeps exactly what the
definition keeps), for 32-bit, 64-bit and two-word keys, with edge cases."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _normalised_net_psi(p):
    la, sg = O.amplitudes(O.Net(p.net), p.S)
    psi = sg * np.exp(la - la.max())
    return psi / np.linalg.norm(psi)


def _compare(N, P, p_norb, h, eri, S, psi, eps):
    got = N.hb_select(P, to_dev(S), torch.from_numpy(psi).cuda(), eps)
    keys, mx = O.hb_select(p_norb, h, eri, S, psi, eps)
    gd = got["dets"].cpu().view(torch.int64).numpy().view(np.uint64)
    gc = got["coupling"].cpu().numpy()
    assert gd.shape[0] == keys.shape[0], (gd.shape, keys.shape, eps)
    assert np.array_equal(gd, keys)
    assert np.array_equal(gc, mx)
    assert got["n_emitted"] >= gd.shape[0]
    return got


@pytest.mark.parametrize("eps", [0.0, 1e-5, 1e-4, 1e-3, 1e-2])
def test_hb_tiny_matches_oracle(eps):
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    _compare(N, P, 10, p.h, p.eri, p.S, _normalised_net_psi(p), eps)


def test_hb_random_psi_with_zeros_and_spread():
    """Amplitudes over many decades, some exactly zero (those parents contribute nothing)."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(len(p.S)) * 10.0 ** rng.uniform(-6, 0, len(p.S))
    psi[::7] = 0.0
    for eps in (1e-6, 3e-4):
        _compare(N, P, 10, p.h, p.eri, p.S, psi, eps)


def test_hb_small_n16_subset():
    """32-bit keys, 16 orbitals, 4096 parents (the first of the level-major S)."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    S = p.S[:4096]
    psi = _normalised_net_psi(p)[:4096]
    for eps in (1e-5, 1e-4):
        _compare(N, P, 16, p.h, p.eri, S, psi, eps)


def test_hb_norb30_64bit_keys():
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(30, 60, 2, 3.0)
    S = synth.select_S(30, 12, 600)
    P = N.Problem(30, 12, 12, h, eri)
    rng = np.random.default_rng(2)
    psi = rng.standard_normal(len(S)) * np.exp(-rng.uniform(0, 8, len(S)))
    psi /= np.linalg.norm(psi)
    for eps in (1e-6, 1e-4):
        _compare(N, P, 30, h, eri, S, psi, eps)


def test_hb_norb42_two_word_keys():
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(42, 84, 3, 3.0)
    S = synth.select_S(42, 24, 160)
    P = N.Problem(42, 24, 24, h, eri)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(len(S))
    psi /= np.linalg.norm(psi)
    _compare(N, P, 42, h, eri, S, psi, 1e-5)


def test_hb_edge_cases():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    dets = to_dev(p.S)
    zero = torch.zeros(len(p.S), dtype=torch.float64, device="cuda")
    # all amplitudes zero: nothing reaches a positive cutoff; eps = 0 keeps every neighbour
    assert N.hb_select(P, dets, zero, 1e-12)["dets"].shape[0] == 0
    _compare(N, P, 10, p.h, p.eri, p.S, np.zeros(len(p.S)), 0.0)
    # a cutoff above every coupling keeps nothing
    psi = _normalised_net_psi(p)
    assert N.hb_select(P, dets, torch.from_numpy(psi).cuda(), 1e6)["dets"].shape[0] == 0
    # one parent
    _compare(N, P, 10, p.h, p.eri, p.S[:1], psi[:1] * 0 + 1.0, 1e-3)
    # invalid cutoffs are rejected
    for bad in (-1e-9, float("nan")):
        with pytest.raises(N.NQSError):
            N.hb_select(P, dets, torch.from_numpy(psi).cuda(), bad)
    # unsorted S is rejected with validation on
    rev = to_dev(p.S[::-1].copy())
    with pytest.raises(N.NQSError):
        N.hb_select(P, rev, torch.from_numpy(psi).cuda(), 1e-3, o=N.opts(validate=1))


def test_hb_full_size_cr2_24e30o_sampled():
    """Full 30-orbital S (131072 dets), eps = 1e-6 on normalised network amplitudes (the
    paper's threshold). Checked at any size: sorted, unique, outside S, couplings >= eps. Checked
    against the oracle on three blocks of parents: every configuration a block selects is in the
    GPU set with a GPU coupling >= the block's (a maximum over more parents)."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("cr2_24e30o")
    P = problem_for(N, p)
    psi = _normalised_net_psi(p)
    eps = 1e-6
    got = N.hb_select(P, to_dev(p.S), torch.from_numpy(psi).cuda(), eps)
    gd = got["dets"].cpu().view(torch.int64).numpy().view(np.uint64)
    gc = got["coupling"].cpu().numpy()
    assert gd.shape[0] > 0 and np.all(gc >= eps)

    def packed(d):  # 60-bit key (a << 30) | b, numeric order = (a, b) order
        return (d[:, 0] << np.uint64(30)) | d[:, 1]

    gk = packed(gd)
    assert np.all(gk[1:] > gk[:-1])
    sk = packed(p.S)
    pos = np.minimum(np.searchsorted(gk, sk), len(gk) - 1)
    assert not np.any(gk[pos] == sk)
    nS = len(p.S)
    for r0, r1 in [(0, 64), (nS // 2, nS // 2 + 64), (nS - 64, nS)]:
        bk, bm = O.hb_select(30, p.h, p.eri, p.S, psi, eps, rows=(r0, r1))
        if len(bk) == 0:
            continue
        q = packed(bk)
        pos = np.minimum(np.searchsorted(gk, q), len(gk) - 1)
        assert np.all(gk[pos] == q), r0
        assert np.all(gc[pos] >= bm), r0
