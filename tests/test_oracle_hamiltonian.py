"""Pins of the oracle's Hamiltonian pieces against definitions that do not share its logic:
brute-force second quantisation (Jordan-Wigner), exhaustive search of the connected set, and a
textbook full-CI example."""
import itertools
import os

import numpy as np
import pytest

from oracle import bruteforce as BF
from paper_2601_21310_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("norb,na,nb", [(3, 1, 2), (4, 2, 2), (5, 2, 3), (6, 3, 3), (6, 2, 4)])
def test_slater_condon_equals_second_quantisation(olib, norb, na, nb):
    """Every <y|H|x> of the oracle equals the Jordan-Wigner operator sum: same pattern, same
    sign, value within 1e-13."""
    h, eri, _ = synth.integrals(norb, 2 * norb, 17 + norb, 3.0)
    dets, H = BF.dense_hamiltonian(norb, na, nb, h, eri)
    N = len(dets)
    for x in range(N):
        for y in range(N):
            v, lv = olib.element(norb, h, eri, dets[x], dets[y])
            ref = H[y, x]
            assert (v != 0.0) == (ref != 0.0), (x, y)
            assert abs(v - ref) <= 1e-13 * max(1.0, abs(ref)), (x, y, v, ref)
            if lv == 3:
                assert v == 0.0


def test_diag_equals_second_quantisation(olib):
    norb, na, nb = 6, 3, 2
    h, eri, _ = synth.integrals(norb, 12, 5, 3.0)
    dets, H = BF.dense_hamiltonian(norb, na, nb, h, eri)
    for k, (a, b) in enumerate(dets):
        assert abs(olib.diag(norb, h, eri, a, b) - H[k, k]) < 1e-13


@pytest.mark.parametrize("norb,na,nb", [(5, 2, 2), (6, 3, 2), (7, 3, 3)])
def test_connected_set_is_all_singles_and_doubles(olib, norb, na, nb):
    """Eq. (connected_set): the enumerated excitations of x are exactly the configurations of
    the sector at excitation level 1 or 2 from x, each once."""
    dets, _ = BF.sector_basis(norb, na, nb)
    n_expected = olib.n_excitations(norb, na, nb)
    for x in dets[:: max(1, len(dets) // 25)]:
        exc = olib.excitations(norb, x[0], x[1])
        got = {(int(a), int(b)) for a, b in exc}
        assert len(got) == len(exc) == n_expected
        want = set()
        for a, b in dets:
            lv = (bin(int(a) ^ int(x[0])).count("1") + bin(int(b) ^ int(x[1])).count("1")) // 2
            if lv in (1, 2):
                want.add((int(a), int(b)))
        assert got == want


def test_excitation_count_formula(olib):
    # singles + same-spin doubles + opposite-spin doubles
    for norb, n, total in [(10, 5, 875), (16, 8, 5792), (30, 12, 67284), (42, 24, 271944)]:
        assert olib.n_excitations(norb, n, n) == total


def test_canonical_order_head(olib):
    """Alpha singles (i asc, a asc) come first, then beta singles, then alpha-alpha doubles."""
    norb, n = 5, 2
    exc = olib.excitations(norb, 0b00011, 0b00011)
    assert (int(exc[0][0]), int(exc[0][1])) == (0b00110, 0b00011)   # alpha 0 -> 2
    assert (int(exc[1][0]), int(exc[1][1])) == (0b01010, 0b00011)   # alpha 0 -> 3
    assert (int(exc[6][0]), int(exc[6][1])) == (0b00011, 0b00110)   # beta 0 -> 2
    assert (int(exc[12][0]), int(exc[12][1])) == (0b01100, 0b00011)  # alpha 0,1 -> 2,3


def test_hss_matches_dense_restriction(olib):
    """H_SS from the oracle equals the brute-force H restricted to S, and the CSR row layout is
    [diagonal, hits in canonical order]."""
    norb, na, nb = 6, 3, 3
    h, eri, _ = synth.integrals(norb, 12, 3, 3.0)
    dets, H = BF.dense_hamiltonian(norb, na, nb, h, eri)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(dets), size=120, replace=False))
    S = dets[pick]
    csr = olib.hss(norb, h, eri, S)
    dense = csr.to_scipy().toarray()
    ref = H[np.ix_(pick, pick)].T  # row x holds <y|H|x>
    assert np.abs(dense - ref).max() < 1e-13
    assert np.array_equal(dense != 0, ref != 0)
    for r in range(len(S)):
        assert csr.col[csr.row_ptr[r]] == r
    assert csr.n_enumerated == len(S) * olib.n_excitations(norb, na, nb)


def test_hss_bit_exact_symmetric_tiny_workload(olib):
    """The canonical summation order makes H_SS symmetric bit for bit."""
    p = synth.make_problem("tiny_n10")
    csr = olib.hss(p.wl.norb, p.h, p.eri, p.S)
    A = csr.to_scipy()
    assert (A != A.T).nnz == 0
    assert csr.n_enumerated == 1000 * 875


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_h2_minimal_basis_textbook(olib):
    """Textbook H2/STO-3G: HF energy and full-CI correlation energy from the printed integrals."""
    g = _read_golden("h2_sto3g.txt")
    norb = 2
    h = np.array([[g["h11"], 0.0], [0.0, g["h22"]]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = g["J11"]
    eri[1, 1, 1, 1] = g["J22"]
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = g["J12"]
    for p, q, r, s in itertools.product(range(2), repeat=4):
        if sorted((p, q)) == [0, 1] and sorted((r, s)) == [0, 1]:
            eri[p, q, r, s] = g["K12"]
    S = synth.full_space(norb, 1)
    csr = olib.hss(norb, h, eri, S)
    Hd = csr.to_scipy().toarray()
    e_hf = olib.diag(norb, h, eri, 1, 1)
    assert abs(e_hf - g["E_HF"]) < 2e-4
    w, V = np.linalg.eigh(Hd)
    assert abs((w[0] - e_hf) - g["E_corr"]) < 2e-4
    # the Rayleigh quotient of the eigenvector reproduces the eigenvalue
    out, _ = olib.energy_from_psi(csr, V[:, 0])
    assert abs(out[0] - w[0]) < 1e-12


def test_hss_rows_equals_slices_of_full(olib):
    """The row-range H_SS used for sampled checks of large problems equals the same rows of the
    full matrix."""
    p = synth.make_problem("tiny_n10")
    full = olib.hss(10, p.h, p.eri, p.S)
    for r0, r1 in [(0, 1), (100, 250), (990, 1000)]:
        rp, col, val = olib.hss_rows(10, p.h, p.eri, p.S, r0, r1)
        a, b = full.row_ptr[r0], full.row_ptr[r1]
        assert np.array_equal(rp, full.row_ptr[r0:r1 + 1] - a)
        assert np.array_equal(col, full.col[a:b]) and np.array_equal(val, full.val[a:b])
