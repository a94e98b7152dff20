"""The seeded input generator: structure of integrals, S and parameters."""
import numpy as np
import pytest

from paper_2601_21310_b300 import synth


@pytest.mark.parametrize("norb,K,seed,ell", [(6, 12, 0, 3.0), (10, 20, 0, 3.0), (16, 32, 1, 3.0)])
def test_integrals_symmetry_bit_exact(norb, K, seed, ell):
    h, eri, ecore = synth.integrals(norb, K, seed, ell)
    assert ecore == 0.0
    assert np.array_equal(h, h.T)
    assert np.array_equal(np.diag(h), np.linspace(-2, 1, norb))
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0),
                 (3, 2, 1, 0)]:
        assert np.array_equal(eri, eri.transpose(perm)), perm


def test_integrals_decay_and_scale():
    h, eri, _ = synth.integrals(16, 32, 1, 3.0)
    # off-diagonal one-body elements decay with |p-q|
    near = np.mean([abs(h[p, p + 1]) for p in range(15)])
    far = np.mean([abs(h[p, p + 8]) for p in range(8)])
    assert far < near
    # (pp|pp) = sum_k (L^k_pp)^2 > 0
    assert all(eri[p, p, p, p] > 0 for p in range(16))


def test_selected_set_tiny_composition():
    wl = synth.WORKLOADS["tiny_n10"]
    S = synth.select_S(wl.norb, wl.nalpha, wl.nS)
    assert S.shape == (1000, 2)
    keys = [(int(a), int(b)) for a, b in S]
    assert keys == sorted(set(keys))
    pc = np.bitwise_count(S)
    assert (pc == 5).all()
    hf = (1 << 5) - 1
    lv = [(bin(a ^ hf).count("1") + bin(b ^ hf).count("1")) // 2 for a, b in keys]
    counts = np.bincount(lv)
    # HF, then all 50 singles and 825 doubles, then 124 triples
    assert counts.tolist() == [1, 50, 825, 124]


def test_selected_set_small_sizes():
    wl = synth.WORKLOADS["small_n16"]
    S = synth.select_S(wl.norb, wl.nalpha, wl.nS)
    assert S.shape == (16384, 2)
    hf = (1 << 8) - 1
    lv = [(bin(int(a) ^ hf).count("1") + bin(int(b) ^ hf).count("1")) // 2 for a, b in S]
    assert np.bincount(lv).tolist() == [1, 128, 5664, 10591]


def test_full_space_and_params():
    F = synth.full_space(6, 3)
    assert F.shape == (400, 2)
    net = synth.net_params(10, 5, 5, (64, 64), 100)
    assert net.W1.shape == (64, 20) and net.W3.shape == (100, 64)
    assert (net.b3 == 0).all()
    assert net.Phi0[3, 3] == 1 and net.Phi0[3, 8] == 1 and net.Phi0.sum() == 10
    assert net.n_params == 64 * 20 + 64 + 64 * 64 + 64 + 100 * 64 + 100


def test_batched_workloads():
    ws = synth.batched_workloads()
    assert len(ws) == 64
    for w in ws:
        assert 12 <= w.norb <= 28 and w.nalpha == w.norb // 2 - 2
        assert 512 <= w.nS <= 32768
