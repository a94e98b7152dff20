"""Pins of the oracle's ansatz, energy, gradient and PT2 against independent definitions:
permutation-expansion determinants, torch's own MLP and bf16 cast, dense eigensolvers, central
finite differences, and the brute-force Hamiltonian."""
import itertools
import math

import numpy as np
import pytest
import torch

from oracle import bruteforce as BF
from paper_2601_21310_b300 import synth


def _perm_det(A):
    """det by the Leibniz permutation expansion (n <= 6)."""
    n = A.shape[0]
    tot = 0.0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        prod = 1.0
        for i in range(n):
            prod *= A[i, p[i]]
        tot += (-1) ** inv * prod
    return tot


def _occ(w, norb):
    return [p for p in range(norb) if (int(w) >> p) & 1]


def test_amplitude_constant_phi_is_product_of_minors(olib):
    """With W3 = 0 the orbital matrix is Phi0 + b3 for every x; psi(x) must equal the product of
    the two occupied minors computed by permutation expansion."""
    norb, n = 7, 3
    net = synth.net_params(norb, n, n, (16, 16), 5)
    rng = np.random.default_rng(1)
    net.W3[:] = 0.0
    net.b3[:] = rng.normal(0, 0.5, size=net.b3.size)
    Phi = net.Phi0 + net.b3.reshape(norb, 2 * n)
    S = synth.full_space(norb, n)[::7]
    la, sg = olib.amplitudes(olib.Net(net), S)
    for k, (a, b) in enumerate(S):
        da = _perm_det(Phi[np.ix_(_occ(a, norb), range(n))])
        db = _perm_det(Phi[np.ix_(_occ(b, norb), range(n, 2 * n))])
        ref = da * db
        assert sg[k] == np.sign(ref)
        assert abs(la[k] - math.log(abs(ref))) < 1e-12


def test_amplitude_hf_is_one_when_backflow_vanishes(olib):
    net = synth.net_params(10, 5, 5, (64, 64), 100)
    net.W3[:] = 0.0
    la, sg = olib.amplitudes(olib.Net(net), np.array([[31, 31]], np.uint64))
    assert sg[0] == 1 and la[0] == 0.0


def _torch_logpsi(net, S, quant=False):
    """Independent evaluation of the backflow ansatz with torch (FP64)."""
    t = lambda x: torch.tensor(x, dtype=torch.float64)  # noqa: E731
    W1, b1, W2, b2, W3, b3, Phi0 = [t(x) for x in net.as_list()]
    norb, na, nb = net.norb, net.nalpha, net.nbeta
    if quant:
        q = lambda w: w.to(torch.float32).to(torch.bfloat16).to(torch.float64)  # noqa: E731
        f = lambda w: w.to(torch.float32).to(torch.float64)  # noqa: E731
        W1, W2, W3 = q(W1), q(W2), q(W3)
        b1, b2, b3, Phi0 = f(b1), f(b2), f(b3), f(Phi0)
    else:
        q = lambda w: w  # noqa: E731
    bits = np.array([[(int(a) >> p) & 1 for p in range(norb)] + [(int(b) >> p) & 1 for p in range(norb)]
                     for a, b in S], dtype=np.float64)
    x = torch.tensor(bits)
    h1 = q(torch.tanh(x @ W1.T + b1))
    h2 = q(torch.tanh(h1 @ W2.T + b2))
    phi = (h2 @ W3.T + b3).reshape(-1, norb, na + nb) + Phi0
    out = []
    for k, (a, b) in enumerate(S):
        Aa = phi[k][_occ(a, norb)][:, :na]
        Ab = phi[k][_occ(b, norb)][:, na:]
        sa, la = torch.linalg.slogdet(Aa)
        sb, lb = torch.linalg.slogdet(Ab)
        out.append((float(la + lb), int(sa * sb)))
    return out


@pytest.mark.parametrize("quant", [False, True])
def test_amplitudes_match_torch(olib, quant):
    p = synth.make_problem("tiny_n10")
    la, sg = olib.amplitudes(olib.Net(p.net, quant=quant), p.S)
    ref = _torch_logpsi(p.net, p.S[:200], quant=quant)
    for k, (l, s) in enumerate(ref):
        assert sg[k] == s
        assert abs(la[k] - l) < 1e-11


def test_bf16_rounding_matches_torch(olib):
    rng = np.random.default_rng(3)
    vals = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-3, 2000), rng.uniform(-300, 300, 2000)])
    # exact ties between two bf16 neighbours (round half to even)
    ties = [1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, -(2.0 + 2.0**-7), 0.5 + 2.0**-9 + 2.0**-8]
    vals = np.concatenate([vals, ties])
    ref = torch.tensor(vals, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([olib.bf16_round(v) for v in vals])
    assert np.array_equal(got, ref)


@pytest.fixture(scope="module")
def tiny(olib):
    p = synth.make_problem("tiny_n10")
    csr = olib.hss(p.wl.norb, p.h, p.eri, p.S)
    return p, csr


def test_energy_eigenvector_and_lower_bound(olib, tiny):
    """E_S = lambda for an eigenvector of H_SS; E_S >= lambda_min(H_SS) for the network psi."""
    p, csr = tiny
    Hd = csr.to_scipy().toarray()
    w, V = np.linalg.eigh(Hd)
    for k in (0, 5, 999):
        out, _ = olib.energy_from_psi(csr, V[:, k] * 3.7)
        assert abs(out[0] - w[k]) < 1e-10
    r = olib.energy_grad(olib.Net(p.net), p.S, csr, with_grad=False)
    assert r["E"] >= w[0] - 1e-12
    assert r["E"] <= w[-1] + 1e-12
    # N and D are psi^T H psi and psi^T psi
    psi = r["psi"]
    assert abs(r["N"] - psi @ Hd @ psi) < 1e-10 * abs(r["N"])
    assert abs(r["D"] - psi @ psi) < 1e-12 * r["D"]


def test_full_space_fci_tiny(olib):
    """S = full space and psi = the ground state of the brute-force H: E_S = E_FCI, and PT2
    vanishes (no external set; zero residual)."""
    norb, n = 5, 2
    h, eri, _ = synth.integrals(norb, 10, 9, 3.0)
    dets, H = BF.dense_hamiltonian(norb, n, n, h, eri)
    w, V = np.linalg.eigh(H)
    csr = olib.hss(norb, h, eri, dets)
    out, _ = olib.energy_from_psi(csr, V[:, 0])
    assert abs(out[0] - w[0]) < 1e-11
    r = olib.pt2(norb, h, eri, dets, V[:, 0], out[0])
    assert r["ext"] == 0.0 and r["n_unique"] == 0
    assert abs(r["int"]) < 1e-20


def test_gradient_central_differences(olib, tiny):
    """Adjoint gradient (Eq. variational_gradient) vs central differences, h = 1e-5, on 64
    parameters chosen with seed 7 (FP64 form)."""
    p, csr = tiny
    net = p.net
    base = olib.Net(net)
    g = olib.energy_grad(base, p.S, csr)["grad"]
    flat = np.concatenate([x.ravel() for x in net.as_list()[:6]])
    rng = np.random.default_rng(7)
    pick = rng.choice(flat.size, size=64, replace=False)
    hstep = 1e-5

    def energy_at(vec):
        arrs, k = [], 0
        for x in net.as_list()[:6]:
            arrs.append(vec[k:k + x.size].reshape(x.shape))
            k += x.size
        q = synth.NetParams(*arrs, net.Phi0, net.norb, net.nalpha, net.nbeta)
        return olib.energy_grad(olib.Net(q), p.S, csr, with_grad=False)["E"]

    fd = []
    for k in pick:
        vp, vm = flat.copy(), flat.copy()
        vp[k] += hstep
        vm[k] -= hstep
        fd.append((energy_at(vp) - energy_at(vm)) / (2 * hstep))
    fd = np.array(fd)
    err = np.linalg.norm(fd - g[pick]) / np.linalg.norm(g[pick])
    assert err < 1e-6, err
    # directional derivative along a random direction
    d = rng.normal(size=flat.size)
    dd = (energy_at(flat + 1e-6 * d) - energy_at(flat - 1e-6 * d)) / 2e-6
    assert abs(dd - g @ d) < 1e-6 * abs(g @ d) + 1e-10


def test_pt2_matches_dense_bruteforce(olib):
    """Eq. (pt2_correction) on a tiny case, against the dense brute-force H: external term over
    the complement of S and internal term over S, both with psi normalised by D."""
    norb, n = 6, 3
    h, eri, _ = synth.integrals(norb, 12, 21, 3.0)
    dets, H = BF.dense_hamiltonian(norb, n, n, h, eri)
    rng = np.random.default_rng(4)
    pick = np.sort(rng.choice(len(dets), size=60, replace=False))
    S = dets[pick]
    psi = rng.normal(size=60)
    csr = olib.hss(norb, h, eri, S)
    out, _ = olib.energy_from_psi(csr, psi)
    E, D = out[0], out[2]
    full = np.zeros(len(dets))
    full[pick] = psi
    c = H @ full
    inS = np.zeros(len(dets), bool)
    inS[pick] = True
    dH = np.diag(H)
    ext_mask = (~inS) & (np.abs(c) > 0)
    ext = np.sum(c[ext_mask] ** 2 / (D * (E - dH[ext_mask])))
    r = c[pick] - E * psi
    intl = np.sum(r**2 / (D * (E - dH[pick])))
    got = olib.pt2(norb, h, eri, S, psi, E)
    assert abs(got["ext"] - ext) < 1e-12 * abs(ext)
    assert abs(got["int"] - intl) < 1e-12 * abs(intl)
    # configurations reachable from S but outside it; an accidental zero c is not expected here
    assert got["n_unique"] == int(ext_mask.sum())


@pytest.mark.parametrize("nbuckets,bucket_id", [(1, -1), (3, 1)])
def test_pt2_unique_set_matches_dense_bruteforce(olib, nbuckets, bucket_id):
    """The deduplicated external set of Eq. (pt2_correction): every configuration outside S
    within two excitations of some member of S (found by counting differing occupation bits,
    not by enumerating excitations), ascending by (a, b), with c(x') = (H psi)_x' from the
    dense brute-force H; with buckets, the members of that hash bucket only."""
    norb, n = 6, 3
    h, eri, _ = synth.integrals(norb, 12, 22, 3.0)
    dets, H = BF.dense_hamiltonian(norb, n, n, h, eri)
    rng = np.random.default_rng(5)
    pick = np.sort(rng.choice(len(dets), size=40, replace=False))
    S = dets[pick]
    psi = rng.normal(size=40)
    full = np.zeros(len(dets))
    full[pick] = psi
    c = H @ full
    inS = np.zeros(len(dets), bool)
    inS[pick] = True
    diff = (np.bitwise_count(dets[:, None, 0] ^ S[None, :, 0]) +
            np.bitwise_count(dets[:, None, 1] ^ S[None, :, 1]))
    reach = ((diff > 0) & (diff <= 4)).any(axis=1) & ~inS
    if bucket_id >= 0:
        reach &= np.array([olib.bucket(a, b, nbuckets) == bucket_id for a, b in dets])
    keys, cu, info = olib.pt2_unique(norb, h, eri, S, psi, -1.0, nbuckets, bucket_id)
    order = np.lexsort((dets[reach, 1], dets[reach, 0]))
    assert np.array_equal(keys, dets[reach][order])
    assert np.abs(cu - c[reach][order]).max() < 1e-13
    assert info["n_unique"] == int(reach.sum())
    assert info["ext"] == olib.pt2(norb, h, eri, S, psi, -1.0, nbuckets, bucket_id)["ext"]


def test_pt2_buckets_partition(olib, tiny):
    p, csr = tiny
    r = olib.energy_grad(olib.Net(p.net), p.S, csr, with_grad=False)
    whole = olib.pt2(p.wl.norb, p.h, p.eri, p.S, r["psi"], r["E"])
    parts = [olib.pt2(p.wl.norb, p.h, p.eri, p.S, r["psi"], r["E"], 4, b) for b in range(4)]
    assert abs(sum(x["ext"] for x in parts) - whole["ext"]) < 1e-12 * abs(whole["ext"])
    assert abs(sum(x["int"] for x in parts) - whole["int"]) < 1e-12 * abs(whole["int"])
    assert sum(x["n_unique"] for x in parts) == whole["n_unique"]
    assert whole["ext"] < 0 and whole["int"] < 0


def test_pt2_internal_vanishes_at_eigenvector(olib, tiny):
    p, csr = tiny
    w, V = np.linalg.eigh(csr.to_scipy().toarray())
    r = olib.pt2(p.wl.norb, p.h, p.eri, p.S, V[:, 0], w[0])
    assert abs(r["int"]) < 1e-18


@pytest.mark.parametrize("eps", [1e-3, 1e-2, 5e-2])
def test_screened_pt2_matches_dense_bruteforce(olib, eps):
    """Screened external term (Sec. 3.3 applied to each contribution): c(x') keeps the terms
    H_x'y psi_y with |H_x'y psi_y| >= eps; x' outside S with at least one kept term form P.
    Against the dense brute-force H; the internal term stays exact."""
    norb, n = 6, 3
    h, eri, _ = synth.integrals(norb, 12, 23, 3.0)
    dets, H = BF.dense_hamiltonian(norb, n, n, h, eri)
    rng = np.random.default_rng(6)
    pick = np.sort(rng.choice(len(dets), size=70, replace=False))
    S = dets[pick]
    psi = rng.normal(size=70) * np.exp(-3 * rng.random(70))
    csr = olib.hss(norb, h, eri, S)
    out, _ = olib.energy_from_psi(csr, psi)
    E, D = out[0], out[2]
    inS = np.zeros(len(dets), bool)
    inS[pick] = True
    dH = np.diag(H)
    Hc = H[:, pick] * psi[None, :]          # contributions H_x'y psi_y
    Hc[np.arange(len(dets))[:, None] == pick[None, :]] = 0.0  # no diagonal contribution
    keep = np.abs(Hc) >= eps
    c = np.where(keep, Hc, 0.0).sum(axis=1)
    in_P = (~inS) & keep.any(axis=1)
    ext = np.sum(c[in_P] ** 2 / (D * (E - dH[in_P])))
    full = np.zeros(len(dets))
    full[pick] = psi
    r = (H @ full)[pick] - E * psi
    intl = np.sum(r ** 2 / (D * (E - dH[pick])))
    got = olib.pt2(norb, h, eri, S, psi, E, eps=eps)
    assert got["n_unique"] == int(in_P.sum())
    assert abs(got["ext"] - ext) <= 1e-12 * abs(ext)
    assert abs(got["int"] - intl) <= 1e-12 * abs(intl)
    # eps = 0 is the unscreened correction
    z = olib.pt2(norb, h, eri, S, psi, E, eps=0.0)
    u = olib.pt2(norb, h, eri, S, psi, E)
    assert z == u


def test_pt2_unique_screened_matches_dense_bruteforce(olib):
    """The screened external set of Sec. 3.3: the configurations outside S with at least one
    contribution |H_x'y psi_y| >= eps, ascending by (a, b), and c(x') the sum of the kept
    contributions, from the dense brute-force H (eps placed away from every contribution, so
    the last-bit difference between the two forms of H decides nothing)."""
    norb, n = 6, 3
    h, eri, _ = synth.integrals(norb, 12, 22, 3.0)
    dets, H = BF.dense_hamiltonian(norb, n, n, h, eri)
    rng = np.random.default_rng(7)
    pick = np.sort(rng.choice(len(dets), size=40, replace=False))
    S = dets[pick]
    psi = rng.normal(size=40)
    inS = np.zeros(len(dets), bool)
    inS[pick] = True
    contrib = H[:, pick] * psi[None, :]
    mags = np.sort(np.abs(contrib[~inS][np.abs(contrib[~inS]) > 0]))
    k = (9 * len(mags)) // 10  # a cut that drops most contributions and some x' entirely
    while mags[k + 1] <= mags[k] * (1 + 1e-6):  # a gap between two neighbouring magnitudes
        k += 1
    eps = float(np.sqrt(mags[k] * mags[k + 1]))
    assert mags[k] < eps * (1 - 1e-9) and mags[k + 1] > eps * (1 + 1e-9)
    kept = np.abs(contrib) >= eps
    reach = kept.any(axis=1) & ~inS
    c = np.where(kept, contrib, 0.0).sum(axis=1)
    keys, cu, info = olib.pt2_unique(norb, h, eri, S, psi, -1.0, eps=eps)
    order = np.lexsort((dets[reach, 1], dets[reach, 0]))
    assert 0 < len(keys) < int((np.abs(contrib[~inS]) > 0).any(axis=1).sum())
    assert np.array_equal(keys, dets[reach][order])
    assert np.abs(cu - c[reach][order]).max() < 1e-13
    assert info["ext"] == olib.pt2(norb, h, eri, S, psi, -1.0, eps=eps)["ext"]
