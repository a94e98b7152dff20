"""Membership of the connected set in S resolved through runs of S (CPU).

The H_SS count pass decides, for every canonical excitation of x = (A, B), whether x' is in S.
Besides one hash lookup per excitation it uses two groupings of the sorted S: the run of
members that share an alpha string and the group of members that share a beta string. A member
y of x's own alpha run is a beta single of x when B ^ b_y has 2 bits and a beta-beta double
when it has 4, and its canonical index follows from the occupied / virtual ranks of the
differing bits (pairs in lexicographic order); likewise for x's own beta group and the alpha
excitations, and for the run of each alpha single a' of A and the alpha-beta doubles.

This test restates that resolution in NumPy, independently of the CUDA code, and checks that it
marks exactly the canonical indices whose x' the oracle's connected set (Eq. connected_set)
places in S: the same hit set, index for index.
"""
import numpy as np
import pytest

from paper_2601_21310_b300 import synth


def _bits(w, norb):
    return [p for p in range(norb) if (w >> p) & 1]


def _rank(w, bit):
    """number of set bits of w below position bit"""
    return bin(w & ((1 << bit) - 1)).count("1")


def _pair_pos(r1, r2, n):
    return r1 * (2 * n - r1 - 1) // 2 + (r2 - r1 - 1)


def _index_hits(norb, na, nb, S):
    """canonical hit indices of every member of S, through the alpha runs and beta groups"""
    ma, mb = norb - na, norb - nb
    sA, sB = na * ma, nb * mb
    dAA = (na * (na - 1) // 2) * (ma * (ma - 1) // 2)
    dBB = (nb * (nb - 1) // 2) * (mb * (mb - 1) // 2)
    o1, o2 = sA, sA + sB
    o3, o4 = o2 + dAA, o2 + dAA + dBB
    Qa, Qb = ma * (ma - 1) // 2, mb * (mb - 1) // 2
    keys = [(int(a), int(b)) for a, b in S]
    runs, groups = {}, {}
    for a, b in keys:
        runs.setdefault(a, []).append(b)
        groups.setdefault(b, []).append(a)
    full = (1 << norb) - 1
    out = []
    for A, B in keys:
        hits = set()
        # own alpha run: beta singles (2 bits differ) and beta-beta doubles (4 bits)
        for by in runs[A]:
            d = by ^ B
            pc = bin(d).count("1")
            if pc == 2:
                j, b = (B & d).bit_length() - 1, (by & d).bit_length() - 1
                hits.add(o1 + _rank(B, j) * mb + _rank(~B & full, b))
            elif pc == 4:
                j1, j2 = _bits(B & d, norb)
                b1, b2 = _bits(by & d, norb)
                hits.add(o3 + _pair_pos(_rank(B, j1), _rank(B, j2), nb) * Qb +
                         _pair_pos(_rank(~B & full, b1), _rank(~B & full, b2), mb))
        # own beta group: alpha singles and alpha-alpha doubles
        for ay in groups[B]:
            d = ay ^ A
            pc = bin(d).count("1")
            if pc == 2:
                i, a = (A & d).bit_length() - 1, (ay & d).bit_length() - 1
                hits.add(_rank(A, i) * ma + _rank(~A & full, a))
            elif pc == 4:
                i1, i2 = _bits(A & d, norb)
                a1, a2 = _bits(ay & d, norb)
                hits.add(o2 + _pair_pos(_rank(A, i1), _rank(A, i2), na) * Qa +
                         _pair_pos(_rank(~A & full, a1), _rank(~A & full, a2), ma))
        # alpha-beta doubles: the run of each alpha single a' of A
        occ_a, vir_a = _bits(A, norb), [p for p in range(norb) if not (A >> p) & 1]
        for xa, i in enumerate(occ_a):
            for ya, a in enumerate(vir_a):
                ap = A ^ (1 << i) ^ (1 << a)
                for by in runs.get(ap, ()):
                    d = by ^ B
                    if bin(d).count("1") == 2:
                        j, b = (B & d).bit_length() - 1, (by & d).bit_length() - 1
                        lb = _rank(B, j) * mb + _rank(~B & full, b)
                        hits.add(o4 + (xa * ma + ya) * sB + lb)
        out.append(hits)
    return out


def _oracle_hits(olib, norb, S):
    members = {(int(a), int(b)) for a, b in S}
    out = []
    for a, b in S:
        exc = olib.excitations(norb, a, b)
        out.append({k for k, (x, y) in enumerate(exc) if (int(x), int(y)) in members})
    return out


@pytest.mark.parametrize("case", ["tiny_n10", "unequal", "full"])
def test_run_resolution_equals_lookup(olib, case):
    if case == "tiny_n10":
        norb, na, nb = 10, 5, 5
        S = synth.select_S(norb, na, 1000)
    elif case == "unequal":
        norb, na, nb = 9, 4, 3
        F = synth.full_space(norb, na, nb)
        rng = np.random.default_rng(5)
        S = F[np.sort(rng.choice(len(F), size=700, replace=False))]
    else:
        norb, na, nb = 7, 3, 2
        S = synth.full_space(norb, na, nb)
    got = _index_hits(norb, na, nb, S)
    ref = _oracle_hits(olib, norb, S)
    assert all(g == r for g, r in zip(got, ref))
    # every excitation class has hits to find (class offsets of the canonical order)
    ma, mb = norb - na, norb - nb
    o = np.cumsum([0, na * ma, nb * mb, (na * (na - 1) // 2) * (ma * (ma - 1) // 2),
                   (nb * (nb - 1) // 2) * (mb * (mb - 1) // 2)])
    cls = np.searchsorted(o, [k for r in ref for k in r], side="right") - 1
    assert set(cls.tolist()) == {0, 1, 2, 3, 4}
