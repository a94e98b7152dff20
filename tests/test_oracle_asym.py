"""Pins of the oracle's Asymmetric mode (Sec. 2.4.1, Eqs. asymmetric_energy,
asymmetric_gradient): E_asym, the log-derivative estimator and the exact gradient against an
independent torch evaluation with automatic differentiation on the dense brute-force H."""
import numpy as np
import pytest
import torch

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2601_21310_b300 import synth


def _occ(w, norb):
    return [p for p in range(norb) if (int(w) >> p) & 1]


def _torch_psi(params, net, dets):
    W1, b1, W2, b2, W3, b3, Phi0 = params
    norb, na, nb = net.norb, net.nalpha, net.nbeta
    bits = np.array([[(int(a) >> p) & 1 for p in range(norb)] + [(int(b) >> p) & 1 for p in range(norb)]
                     for a, b in dets], dtype=np.float64)
    x = torch.tensor(bits)
    h1 = torch.tanh(x @ W1.T + b1)
    h2 = torch.tanh(h1 @ W2.T + b2)
    phi = (h2 @ W3.T + b3).reshape(-1, norb, na + nb) + Phi0
    out = []
    for k, (a, b) in enumerate(dets):
        out.append(torch.linalg.det(phi[k][_occ(a, norb)][:, :na]) *
                   torch.linalg.det(phi[k][_occ(b, norb)][:, na:]))
    return torch.stack(out)


@pytest.mark.parametrize("seed", [1, 2])
def test_asymmetric_energy_and_gradients_vs_autograd(olib, seed):
    norb, n = 6, 3
    h, eri, _ = synth.integrals(norb, 12, 30 + seed, 3.0)
    dets, H = BF.dense_hamiltonian(norb, n, n, h, eri)
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(dets), size=120, replace=False)
    iv, ip = np.sort(pick[:40]), np.sort(pick[40:])
    V, P = dets[iv], dets[ip]
    net = synth.net_params(norb, n, n, (16, 16), 200 + seed)
    csr = O.proxy_csr(norb, h, eri, V, P)
    onet = O.Net(net)
    ex = O.asym_energy_grad(onet, V, P, csr, exact=True)
    ap = O.asym_energy_grad(onet, V, P, csr, exact=False)

    params = [torch.tensor(x, dtype=torch.float64, requires_grad=(k < 6))
              for k, x in enumerate(net.as_list())]
    t = np.concatenate([iv, ip])
    HT = torch.tensor(H[np.ix_(iv, t)])  # rows V, columns T: <x|H|y>
    psi = _torch_psi(params, net, np.concatenate([V, P]))
    pv = psi[:len(iv)]
    D = (pv * pv).sum()
    N = (pv * (HT @ psi)).sum()
    E = N / D
    assert abs(E.item() - ex["E"]) < 1e-12 * max(1.0, abs(ex["E"]))
    g_exact = torch.autograd.grad(E, params[:6], retain_graph=True)
    g_exact = torch.cat([g.reshape(-1) for g in g_exact]).numpy()
    # the log-derivative estimator: 2 sum_V p(x) (E_loc(x) - E) d ln|psi(x)|
    eloc = (HT @ psi) / pv
    coef = (2.0 * (pv * pv / D) * (eloc - E)).detach()
    surrogate = (coef * torch.log(torch.abs(pv))).sum()
    g_est = torch.autograd.grad(surrogate, params[:6])
    g_est = torch.cat([g.reshape(-1) for g in g_est]).numpy()
    for got, want in ((ex["grad"], g_exact), (ap["grad"], g_est)):
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    # the estimator is not the gradient of E_asym (Sec. 2.4.1)
    assert np.linalg.norm(g_exact - g_est) > 1e-6 * np.linalg.norm(g_exact)
    assert ex["E"] == ap["E"]


def test_asymmetric_without_P_is_variational(olib):
    p = synth.make_problem("tiny_n10")
    V = p.S
    empty = np.zeros((0, 2), np.uint64)
    csr = O.proxy_csr(10, p.h, p.eri, V, empty)
    onet = O.Net(p.net)
    var = O.energy_grad(onet, V, O.hss(10, p.h, p.eri, V))
    for exact in (True, False):
        a = O.asym_energy_grad(onet, V, empty, csr, exact=exact)
        assert abs(a["E"] - var["E"]) < 1e-12
        assert np.linalg.norm(a["grad"] - var["grad"]) <= 1e-10 * np.linalg.norm(var["grad"])
