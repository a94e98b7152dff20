"""Brute-force second-quantised Hamiltonian for tiny cases (test infrastructure only).

This applies the electronic Hamiltonian term by term, from its definition

    H = sum_{pq,s} h_pq a+_{ps} a_{qs} + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs},

to every basis configuration of the Fock-space sector of Sec. 2.1, using Jordan-Wigner signs
on spin-orbital bit strings (alpha orbitals 0..norb-1 first, then beta). It knows nothing
about Slater-Condon rules, excitation classes or the oracle's sign bookkeeping, which is the
point: it pins them.
"""
from __future__ import annotations

import itertools

import numpy as np


def _popcount(x: np.ndarray) -> np.ndarray:
    return np.bitwise_count(x.astype(np.uint64)).astype(np.int64)


def sector_basis(norb: int, na: int, nb: int):
    """All (a, b) configurations, sorted by key, and their spin-orbital strings."""
    sa = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(norb), na))
    sb = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(norb), nb))
    dets = np.array([(a, b) for a in sa for b in sb], dtype=np.uint64)
    strings = (dets[:, 0].astype(np.int64)) | (dets[:, 1].astype(np.int64) << norb)
    return dets, strings


def _apply(states, sign, ok, k, create: bool):
    occ = (states >> k) & 1
    if create:
        ok = ok & (occ == 0)
    else:
        ok = ok & (occ == 1)
    below = states & ((1 << k) - 1)
    sign = sign * np.where(_popcount(below) % 2 == 1, -1, 1)
    states = states ^ (1 << k)
    return states, sign, ok


def dense_hamiltonian(norb: int, na: int, nb: int, h: np.ndarray, eri: np.ndarray):
    """Returns (dets [N,2] uint64, H [N,N]) with H[y, x] = <y|H|x>."""
    dets, strings = sector_basis(norb, na, nb)
    N = strings.size
    index = {int(s): i for i, s in enumerate(strings)}
    H = np.zeros((N, N))
    cols = np.arange(N)

    def add(ops, coef):
        # ops applied right to left: ops[-1] acts first
        st = strings.copy()
        sg = np.ones(N, np.int64)
        ok = np.ones(N, bool)
        for k, create in reversed(ops):
            st, sg, ok = _apply(st, sg, ok, k, create)
        if not ok.any():
            return
        rows = np.array([index[int(s)] for s in st[ok]])
        np.add.at(H, (rows, cols[ok]), coef * sg[ok])

    so = lambda p, s: p + s * norb  # noqa: E731
    for s in (0, 1):
        for p in range(norb):
            for q in range(norb):
                if h[p, q] != 0.0:
                    add([(so(p, s), True), (so(q, s), False)], h[p, q])
    for s in (0, 1):
        for t in (0, 1):
            for p, q, r, u in itertools.product(range(norb), repeat=4):
                c = 0.5 * eri[p, q, r, u]
                if c == 0.0:
                    continue
                if so(p, s) == so(r, t) or so(q, s) == so(u, t):
                    continue  # a+ a+ on the same orbital (or a a) vanishes
                add([(so(p, s), True), (so(r, t), True), (so(u, t), False), (so(q, s), False)], c)
    return dets, H
