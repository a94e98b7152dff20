"""Pins of the oracle's heat-bath screened perturbative set, Eq. (hb_screen) of Sec. 3.3,
against computations that share none of its code: the brute-force Jordan-Wigner Hamiltonian
(the definition evaluated on dense H), and the sorted-integral-table traversal with early exit
that Sec. 3.3 describes, written here from that description."""
import itertools

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2601_21310_b300 import synth


def _case(norb, na, nb, nS, seed):
    h, eri, _ = synth.integrals(norb, 2 * norb, seed, 3.0)
    dets, H = BF.dense_hamiltonian(norb, na, nb, h, eri)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(dets), size=nS, replace=False))
    psi = rng.standard_normal(nS) * np.exp(-2.0 * rng.random(nS))
    return h, eri, dets, H, pick, psi


def _definition_on_dense(dets, H, pick, psi, eps):
    """max_x |H_x'x psi_x| over x in S for every x' outside S with a nonzero coupling or a
    coupling of zero at eps = 0 (x' connected to S)."""
    inS = np.zeros(len(dets), bool)
    inS[pick] = True
    out = {}
    for col, x in enumerate(pick):
        for y in range(len(dets)):
            if inS[y]:
                continue
            lv = (bin(int(dets[y][0]) ^ int(dets[x][0])).count("1")
                  + bin(int(dets[y][1]) ^ int(dets[x][1])).count("1")) // 2
            if lv not in (1, 2):
                continue
            m = abs(H[y, x]) * abs(psi[col])
            if m >= eps:
                key = (int(dets[y][0]), int(dets[y][1]))
                out[key] = max(out.get(key, 0.0), m)
    return out


def _as_dict(keys, mx):
    return {(int(a), int(b)): float(m) for (a, b), m in zip(keys, mx)}


def _check_same(got, want, eps):
    """Equal key sets up to configurations whose coupling sits within rounding of eps; the
    maxima agree to rounding (dense H is summed in another order)."""
    for k in set(got) ^ set(want):
        m = got.get(k, want.get(k))
        assert abs(m - eps) <= 1e-12 * max(eps, 1e-300), (k, m, eps)
    for k in set(got) & set(want):
        assert abs(got[k] - want[k]) <= 1e-13 * max(1.0, want[k]), k


@pytest.mark.parametrize("norb,na,nb,nS,seed", [(5, 2, 2, 20, 3), (6, 3, 3, 60, 4),
                                                (6, 2, 3, 40, 5)])
def test_hb_select_equals_definition_on_dense_H(olib, norb, na, nb, nS, seed):
    h, eri, dets, H, pick, psi = _case(norb, na, nb, nS, seed)
    S = dets[pick]
    for eps in (0.0, 1e-3, 1e-2, 5e-2, 0.2):
        keys, mx = O.hb_select(norb, h, eri, S, psi, eps)
        got = _as_dict(keys, mx)
        want = _definition_on_dense(dets, H, pick, psi, eps)
        _check_same(got, want, eps)
        # output order: ascending (a, b)
        assert all(tuple(keys[i]) < tuple(keys[i + 1]) for i in range(len(keys) - 1))


def _sorted_tables(norb, eri):
    """For each hole pair the particle pairs by descending |<ij||ab>|: same spin
    (ia|jb) - (ib|ja) over i<j, a<b; opposite spin (ia|jb)."""
    same, opp = {}, {}
    for i, j in itertools.combinations(range(norb), 2):
        rows = [(abs(eri[i, a, j, b] - eri[i, b, j, a]), a, b)
                for a, b in itertools.combinations(range(norb), 2) if not {a, b} & {i, j}]
        same[(i, j)] = sorted(rows, key=lambda t: -t[0])
    for i in range(norb):
        for j in range(norb):
            rows = [(abs(eri[i, a, j, b]), a, b) for a in range(norb) for b in range(norb)
                    if a != i and b != j]
            opp[(i, j)] = sorted(rows, key=lambda t: -t[0])
    return same, opp


def _early_exit_selection(norb, dets, H, pick, psi, eps, same, opp):
    """Sec. 3.3: per x a cutoff tau = eps / |psi_x|; each hole pair's sorted particle pairs are
    walked until |<ij||ab>| < tau. Singles are taken from the dense H."""
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(dets)}
    inS = {(int(dets[x][0]), int(dets[x][1])) for x in pick}
    out = {}

    def keep(key, m):
        if key not in inS:
            out[key] = max(out.get(key, 0.0), m)

    for col, x in enumerate(pick):
        A, B = int(dets[x][0]), int(dets[x][1])
        ap = abs(psi[col])
        tau = eps / ap
        occ = {0: [p for p in range(norb) if A >> p & 1], 1: [p for p in range(norb) if B >> p & 1]}
        words = {0: A, 1: B}
        for s in (0, 1):  # singles: every one, exact element
            for i in occ[s]:
                for a in range(norb):
                    if words[s] >> a & 1:
                        continue
                    w = words[s] ^ (1 << i) ^ (1 << a)
                    key = (w, B) if s == 0 else (A, w)
                    m = abs(H[index[key], x]) * ap
                    if m >= eps:
                        keep(key, m)
        for s in (0, 1):  # same-spin doubles
            for i, j in itertools.combinations(occ[s], 2):
                for v, a, b in same[(i, j)]:
                    if v < tau:
                        break
                    if words[s] >> a & 1 or words[s] >> b & 1:
                        continue
                    w = words[s] ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << b)
                    keep((w, B) if s == 0 else (A, w), v * ap)
        for i in occ[0]:  # opposite-spin doubles
            for j in occ[1]:
                for v, a, b in opp[(i, j)]:
                    if v < tau:
                        break
                    if A >> a & 1 or B >> b & 1:
                        continue
                    keep((A ^ (1 << i) ^ (1 << a), B ^ (1 << j) ^ (1 << b)), v * ap)
    return out


@pytest.mark.parametrize("norb,na,nb,nS,seed", [(6, 3, 3, 50, 7), (6, 2, 2, 30, 8)])
def test_hb_select_equals_sorted_table_early_exit(olib, norb, na, nb, nS, seed):
    h, eri, dets, H, pick, psi = _case(norb, na, nb, nS, seed)
    same, opp = _sorted_tables(norb, eri)
    for eps in (2e-3, 2e-2, 1e-1):
        keys, mx = O.hb_select(norb, h, eri, dets[pick], psi, eps)
        _check_same(_as_dict(keys, mx),
                    _early_exit_selection(norb, dets, H, pick, psi, eps, same, opp), eps)


def test_hb_select_limits_and_nesting(olib):
    """eps = 0 keeps the whole connected set outside S; eps above every coupling keeps nothing;
    larger eps gives a subset with the same maxima."""
    norb, na, nb = 6, 3, 3
    h, eri, dets, H, pick, psi = _case(norb, na, nb, 40, 9)
    S = dets[pick]
    conn = set()
    for x in S:
        conn |= {(int(a), int(b)) for a, b in O.excitations(norb, x[0], x[1])}
    conn -= {(int(a), int(b)) for a, b in S}
    k0, m0 = O.hb_select(norb, h, eri, S, psi, 0.0)
    assert {(int(a), int(b)) for a, b in k0} == conn
    big = float(np.abs(H).max() * np.abs(psi).max() * 1.01)
    assert len(O.hb_select(norb, h, eri, S, psi, big)[0]) == 0
    full = _as_dict(k0, m0)
    prev = None
    for eps in (1e-4, 1e-3, 1e-2, 1e-1):
        cur = _as_dict(*O.hb_select(norb, h, eri, S, psi, eps))
        assert all(full[k] == v and v >= eps for k, v in cur.items())
        assert set(cur) == {k for k, v in full.items() if v >= eps}
        if prev is not None:
            assert set(cur) <= set(prev)
        prev = cur


def test_hb_select_row_blocks_combine_to_the_whole(olib):
    """Parents split into row blocks: the union of the blocks' sets, with the maximum of their
    couplings, is the set of all parents (what the sampled full-size GPU checks rely on)."""
    norb, na, nb = 6, 3, 3
    h, eri, dets, H, pick, psi = _case(norb, na, nb, 60, 11)
    S = dets[pick]
    eps = 3e-3
    whole = _as_dict(*O.hb_select(norb, h, eri, S, psi, eps))
    merged = {}
    for r0, r1 in [(0, 7), (7, 30), (30, 31), (31, 60)]:
        for k, v in _as_dict(*O.hb_select(norb, h, eri, S, psi, eps, rows=(r0, r1))).items():
            merged[k] = max(merged.get(k, 0.0), v)
    assert merged == whole
    assert len(O.hb_select(norb, h, eri, S, psi, eps, rows=(5, 5))[0]) == 0
