"""Seeded synthetic inputs: integrals, the selected set S and backflow-network parameters.

This module is the one piece shared by the CUDA path and the oracle. It holds none of the
method's arithmetic: no matrix elements, no signs, no network evaluation. It only draws
random numbers and lists occupation bitstrings.

Conventions (Sec. 2.1 notation; Sec. 2.2 ansatz):
  * a determinant is a pair of uint64 words (alpha string, beta string); bit p of a word set
    means spatial orbital p of that spin is occupied;
  * the key order of determinants is (alpha, beta) lexicographic, alpha in the high word;
  * S is sorted ascending by key and unique.

Integrals follow the shapes of the paper's active spaces (Sec. 4.4: Cr2 CAS(24e,30o) and
CAS(48e,42o)) but are synthetic, since the molecular FCIDUMPs are not available:
  h_pq = h_qp = N(0, 0.3^2) * exp(-|p-q|/ell) for p<q, h_pp = linspace(-2, 1, norb);
  (pq|rs) = sum_k L^k_pq L^k_rs with L^k symmetric, L^k_pq = N(0, 0.1^2) * exp(-|p-q|/ell).
The ERI sum runs over k in a fixed order with separate multiply and add, so the eightfold
permutational symmetry of (pq|rs) holds bit for bit.

The selected set S ("level-major" reading): candidates are the Hartree-Fock determinant
(orbitals 0..n-1 of each spin, where h_pp is lowest) followed by its excitations, ordered by (excitation level, sum of occupied orbital indices, key). With
h_pp = linspace(-2, 1, norb) the index sum orders determinants exactly like the sum of
one-body orbital energies, so the rule is purely combinatorial. The first |S| candidates are
kept and then sorted by key.

Network parameters (Sec. 3.3 initialisation, small output layer so that the ansatz starts near
Hartree-Fock but with Delta Phi = O(0.1) so that amplitudes beyond HF are not vanishingly small):
  W_l ~ N(0, 1/fan_in), b_l ~ N(0, 0.01^2) for the two hidden layers,
  W_3 ~ N(0, 0.1^2/fan_in), b_3 = 0, Phi0 = identity columns.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------------------
# workload table (shapes of the synthetic problems)
# ----------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    norb: int
    nalpha: int
    seed: int
    K: int              # number of Cholesky-like vectors L^k
    ell: float          # off-diagonal decay length
    nS: int             # |S|
    hidden: tuple       # (H1, H2)
    mixed: bool         # True: BF16 GEMMs / FP32 LU; False: plain FP64 form

    @property
    def nbeta(self) -> int:
        return self.nalpha

    @property
    def nelec(self) -> int:
        return self.nalpha + self.nbeta


WORKLOADS = {
    # 10 orbitals, 5a+5b, |S|=1000, MLP 20-64-64-100, plain FP64
    "tiny_n10": Workload("tiny_n10", 10, 5, 0, 20, 3.0, 1000, (64, 64), False),
    # 16 orbitals, 8a+8b, |S|=16384, MLP 32-256-256-256, BF16 GEMMs
    "small_n16": Workload("small_n16", 16, 8, 1, 32, 3.0, 16384, (256, 256), True),
    # 30 orbitals, 12a+12b (shape of Cr2 CAS(24e,30o)), |S|=131072, MLP 60-512-512-720
    "cr2_24e30o": Workload("cr2_24e30o", 30, 12, 2, 60, 5.0, 131072, (512, 512), True),
    # 42 orbitals, 24a+24b (shape of Cr2 CAS(48e,42o)), |S|=2^20, MLP 84-1024-1024-2016
    "cr2_48e42o": Workload("cr2_48e42o", 42, 24, 3, 84, 3.0, 1 << 20, (1024, 1024), True),
    # the same integrals and network with |S| = 2^16 (level-major: HF, its singles and the lowest
    # doubles): a few GB on the device, for single-kernel profiles of the 42-orbital kernels
    "cr2_48e42o_s64k": Workload("cr2_48e42o_s64k", 42, 24, 3, 84, 3.0, 1 << 16, (1024, 1024),
                                True),
}


def batched_workloads(count: int = 64, seed: int = 4, width: int = 128) -> list:
    """The batch of independent problems: norb ~ U[12, 28], n = floor(norb/2) - 2,
    |S| log-uniform in [512, 32768], problem i seeded with 1000 + i, K = 2 norb, ell = 3."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        norb = int(rng.integers(12, 29))
        n = norb // 2 - 2
        nS = int(round(math.exp(rng.uniform(math.log(512), math.log(32768)))))
        out.append(Workload(f"batch_{i}", norb, n, 1000 + i, 2 * norb, 3.0, nS, (width, width), True))
    return out


# ----------------------------------------------------------------------------------------
# integrals
# ----------------------------------------------------------------------------------------
def integrals(norb: int, K: int, seed: int, ell: float = 3.0):
    """Return (h [norb,norb] f64, eri [norb,norb,norb,norb] f64, ecore=0.0)."""
    rng = np.random.default_rng(seed)
    p, q = np.triu_indices(norb, k=1)
    decay = np.exp(-np.abs(p - q) / ell)
    h = np.zeros((norb, norb))
    g = rng.normal(0.0, 0.3, size=p.size) * decay
    h[p, q] = g
    h[q, p] = g
    h[np.arange(norb), np.arange(norb)] = np.linspace(-2.0, 1.0, norb)

    p2, q2 = np.triu_indices(norb, k=0)
    decay2 = np.exp(-np.abs(p2 - q2) / ell)
    eri = np.zeros((norb, norb, norb, norb))
    for _ in range(K):
        L = np.zeros((norb, norb))
        v = rng.normal(0.0, 0.1, size=p2.size) * decay2
        L[p2, q2] = v
        L[q2, p2] = v
        prod = np.multiply.outer(L, L)      # exact products, no fused multiply-add
        eri = eri + prod                    # same k order for every element
    return h, eri, 0.0


# ----------------------------------------------------------------------------------------
# determinants
# ----------------------------------------------------------------------------------------
def hf_string(n: int) -> int:
    return (1 << n) - 1


def _bits_to_int(idx) -> int:
    v = 0
    for i in idx:
        v |= 1 << int(i)
    return v


def level_strings(norb: int, n: int, level: int):
    """All single-spin strings at excitation level `level` from the HF string 0..n-1.

    Returns (words uint64 [N], delta int64 [N]) with delta = (sum of occupied indices) minus
    that of the HF string."""
    occ = list(range(n))
    vir = list(range(n, norb))
    if level > min(n, len(vir)):
        return np.zeros(0, np.uint64), np.zeros(0, np.int64)
    holes = list(itertools.combinations(occ, level))
    parts = list(itertools.combinations(vir, level))
    hf = hf_string(n)
    hw = np.array([_bits_to_int(c) for c in holes], dtype=np.uint64)
    hs = np.array([sum(c) for c in holes], dtype=np.int64)
    pw = np.array([_bits_to_int(c) for c in parts], dtype=np.uint64)
    ps = np.array([sum(c) for c in parts], dtype=np.int64)
    words = (np.uint64(hf) ^ hw[:, None]) | pw[None, :]
    delta = ps[None, :] - hs[:, None]
    return words.reshape(-1), delta.reshape(-1)


def _level_dets(norb: int, n: int, level: int):
    """All determinants at total excitation level `level` from HF: (a, b, delta)."""
    A, B, D = [], [], []
    for la in range(level + 1):
        lb = level - la
        wa, da = level_strings(norb, n, la)
        wb, db = level_strings(norb, n, lb)
        if wa.size == 0 or wb.size == 0:
            continue
        A.append(np.repeat(wa, wb.size))
        B.append(np.tile(wb, wa.size))
        D.append((da[:, None] + db[None, :]).reshape(-1))
    if not A:
        return np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0, np.int64)
    return np.concatenate(A), np.concatenate(B), np.concatenate(D)


def select_S(norb: int, n: int, nS: int) -> np.ndarray:
    """The level-major selected set: returns uint64 [nS, 2] sorted by (alpha, beta)."""
    hf = np.uint64(hf_string(n))
    chosen_a = [np.array([hf], np.uint64)]
    chosen_b = [np.array([hf], np.uint64)]
    left = nS - 1
    level = 1
    while left > 0:
        a, b, d = _level_dets(norb, n, level)
        if a.size == 0:
            raise ValueError(f"only {nS - left} determinants exist; |S|={nS} requested")
        if a.size > left:
            order = np.lexsort((b, a, d))[:left]
            a, b = a[order], b[order]
        chosen_a.append(a)
        chosen_b.append(b)
        left -= a.size
        level += 1
    a = np.concatenate(chosen_a)
    b = np.concatenate(chosen_b)
    order = np.lexsort((b, a))
    S = np.stack([a[order], b[order]], axis=1).astype(np.uint64)
    return np.ascontiguousarray(S)


def full_space(norb: int, na: int, nb: int | None = None) -> np.ndarray:
    """Every determinant of the (na, nb) sector, sorted by key: uint64 [N, 2]."""
    nb = na if nb is None else nb
    sa = sorted(_bits_to_int(c) for c in itertools.combinations(range(norb), na))
    sb = sorted(_bits_to_int(c) for c in itertools.combinations(range(norb), nb))
    a = np.repeat(np.array(sa, np.uint64), len(sb))
    b = np.tile(np.array(sb, np.uint64), len(sa))
    return np.ascontiguousarray(np.stack([a, b], axis=1))


# ----------------------------------------------------------------------------------------
# network parameters
# ----------------------------------------------------------------------------------------
@dataclass
class NetParams:
    """Backflow MLP parameters (row-major, out x in): Phi = Phi0 + reshape(W3 tanh(W2 tanh(W1 x
    + b1) + b2) + b3, [norb][nelec])."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    Phi0: np.ndarray
    norb: int = 0
    nalpha: int = 0
    nbeta: int = 0
    extra: dict = field(default_factory=dict)

    def as_list(self):
        return [self.W1, self.b1, self.W2, self.b2, self.W3, self.b3, self.Phi0]

    @property
    def n_params(self) -> int:
        """Trainable parameter count (Phi0 is fixed)."""
        return sum(x.size for x in self.as_list()[:6])


def identity_phi0(norb: int, na: int, nb: int) -> np.ndarray:
    phi0 = np.zeros((norb, na + nb))
    for k in range(na):
        phi0[k, k] = 1.0
    for k in range(nb):
        phi0[k, na + k] = 1.0
    return phi0


def net_params(norb: int, na: int, nb: int, hidden, seed: int, out_scale: float = 0.1) -> NetParams:
    H1, H2 = hidden
    nin = 2 * norb
    nout = norb * (na + nb)
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, 1.0 / math.sqrt(nin), size=(H1, nin))
    b1 = rng.normal(0.0, 0.01, size=H1)
    W2 = rng.normal(0.0, 1.0 / math.sqrt(H1), size=(H2, H1))
    b2 = rng.normal(0.0, 0.01, size=H2)
    W3 = rng.normal(0.0, out_scale / math.sqrt(H2), size=(nout, H2))
    b3 = np.zeros(nout)
    return NetParams(W1, b1, W2, b2, W3, b3, identity_phi0(norb, na, nb), norb, na, nb)


# ----------------------------------------------------------------------------------------
# one full problem
# ----------------------------------------------------------------------------------------
@dataclass
class Problem:
    wl: Workload
    h: np.ndarray
    eri: np.ndarray
    ecore: float
    S: np.ndarray
    net: NetParams


def make_problem(wl: Workload | str, nS: int | None = None) -> Problem:
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    h, eri, ecore = integrals(wl.norb, wl.K, wl.seed, wl.ell)
    S = select_S(wl.norb, wl.nalpha, nS if nS is not None else wl.nS)
    net = net_params(wl.norb, wl.nalpha, wl.nbeta, wl.hidden, wl.seed + 100)
    return Problem(wl, h, eri, ecore, S, net)


def random_psi(nS: int, seed: int) -> np.ndarray:
    """A seeded amplitude vector (for tests that inject psi directly)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, size=nS)
