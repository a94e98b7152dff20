"""Pins of the oracle's Proxy-mode Hamiltonian (Eq. proxy_hamiltonian, Sec. 2.4.1): against the
dense brute-force H with its P-P block reduced to the diagonal, the variational limit (P
empty), symmetry, and E_proxy (Eq. proxy_energy) with its gradient (Eq. proxy_gradient) by
central differences."""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2601_21310_b300 import synth


def _sets(norb, na, nb, nV, nP, seed):
    h, eri, _ = synth.integrals(norb, 2 * norb, seed, 3.0)
    dets, H = BF.dense_hamiltonian(norb, na, nb, h, eri)
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(dets), size=nV + nP, replace=False)
    iv, ip = np.sort(pick[:nV]), np.sort(pick[nV:])
    return h, eri, dets, H, iv, ip


@pytest.mark.parametrize("norb,na,nb,nV,nP,seed", [(5, 2, 2, 20, 40, 1), (6, 3, 3, 60, 120, 2),
                                                   (6, 2, 3, 30, 90, 3)])
def test_proxy_csr_equals_dense_definition(olib, norb, na, nb, nV, nP, seed):
    h, eri, dets, H, iv, ip = _sets(norb, na, nb, nV, nP, seed)
    csr = O.proxy_csr(norb, h, eri, dets[iv], dets[ip])
    t = np.concatenate([iv, ip])
    want = H[np.ix_(t, t)].copy()
    pp = np.ix_(np.arange(nV, nV + nP), np.arange(nV, nV + nP))
    want[pp] = np.diag(np.diag(want[pp]))
    got = csr.to_scipy().toarray().T  # row x holds <y|H~|x>
    assert np.abs(got - want).max() < 1e-13
    A = csr.to_scipy()
    assert (A != A.T).nnz == 0  # symmetric bit for bit
    # every row starts with its diagonal
    assert all(csr.col[csr.row_ptr[r]] == r for r in range(nV + nP))
    # rows of P reach V only
    for r in range(nV, nV + nP):
        assert np.all(csr.col[csr.row_ptr[r] + 1:csr.row_ptr[r + 1]] < nV)


def test_proxy_without_P_is_hss(olib):
    p = synth.make_problem("tiny_n10")
    a = O.proxy_csr(10, p.h, p.eri, p.S, np.zeros((0, 2), np.uint64))
    b = O.hss(10, p.h, p.eri, p.S)
    assert np.array_equal(a.row_ptr, b.row_ptr)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)


def test_proxy_energy_and_gradient(olib):
    """E_proxy is the Rayleigh quotient of H~ on T (dense check); its gradient is the
    variational formula over T with H~, checked by central differences."""
    p = synth.make_problem("tiny_n10")
    V = p.S[:150]
    la, sg = O.amplitudes(O.Net(p.net), V)
    psi = sg * np.exp(la - la.max())
    Pk, _ = O.hb_select(10, p.h, p.eri, V, psi / np.linalg.norm(psi), 3e-3)
    T = np.concatenate([V, Pk])
    csr = O.proxy_csr(10, p.h, p.eri, V, Pk)
    r = O.energy_grad(O.Net(p.net), T, csr)
    lt, st = O.amplitudes(O.Net(p.net), T)
    pt = st * np.exp(lt - lt.max())
    Hd = csr.to_scipy().toarray()
    assert abs(r["E"] - pt @ Hd @ pt / (pt @ pt)) < 1e-12
    flat = np.concatenate([x.ravel() for x in p.net.as_list()[:6]])
    pick = np.random.default_rng(9).choice(flat.size, size=24, replace=False)
    hs = 1e-5

    def e_at(vec):
        arrs, k = [], 0
        for x in p.net.as_list()[:6]:
            arrs.append(vec[k:k + x.size].reshape(x.shape))
            k += x.size
        q = synth.NetParams(*arrs, p.net.Phi0, p.net.norb, p.net.nalpha, p.net.nbeta)
        return O.energy_grad(O.Net(q), T, csr, with_grad=False)["E"]

    fd = []
    for k in pick:
        a, b = flat.copy(), flat.copy()
        a[k] += hs
        b[k] -= hs
        fd.append((e_at(a) - e_at(b)) / (2 * hs))
    g = r["grad"][pick]
    assert np.abs(g - np.array(fd)).max() <= 1e-6 * max(1.0, np.abs(g).max())
