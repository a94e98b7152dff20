"""GPU parity of the Proxy mode (Sec. 2.4.1): the proxy Hamiltonian H~ of Eq.
(proxy_hamiltonian) over T = V + P bit-exact against the oracle (structure and values), and
E_proxy (Eq. proxy_energy) with its gradient (Eq. proxy_gradient) through nqs_energy_grad over T
(FP64 form 1e-8 Ha; mixed form 1e-6 Ha against the quantisation-matched oracle)."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _VP(p, nV, eps):
    V = p.S[:nV]
    la, sg = O.amplitudes(O.Net(p.net), V)
    psi = sg * np.exp(la - la.max())
    Pk, _ = O.hb_select(p.wl.norb, p.h, p.eri, V, psi / np.linalg.norm(psi), eps)
    return V, Pk


def _compare_csr(g, ref):
    rp, col, val = g.host()
    assert np.array_equal(rp, ref.row_ptr)
    assert np.array_equal(col, ref.col)
    assert np.array_equal(val, ref.val)


@pytest.mark.parametrize("name,nV,eps", [("tiny_n10", 300, 1e-3), ("tiny_n10", 1000, 1e-4),
                                         ("small_n16", 2000, 1e-4)])
def test_proxy_hamiltonian_bit_exact(name, nV, eps):
    need_gpu()
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    V, Pk = _VP(p, nV, eps)
    T = np.concatenate([V, Pk])
    g = N.proxy_hamiltonian(P, to_dev(T), len(V))
    _compare_csr(g, O.proxy_csr(p.wl.norb, p.h, p.eri, V, Pk))


def test_proxy_hamiltonian_30_orbitals():
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(30, 60, 2, 3.0)
    V = synth.select_S(30, 12, 300)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(len(V))
    Pk, _ = O.hb_select(30, h, eri, V, psi / np.linalg.norm(psi), 1e-3)
    P = N.Problem(30, 12, 12, h, eri)
    g = N.proxy_hamiltonian(P, to_dev(np.concatenate([V, Pk])), len(V))
    _compare_csr(g, O.proxy_csr(30, h, eri, V, Pk))


def test_proxy_without_P_is_hss():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    d = to_dev(p.S)
    a = N.proxy_hamiltonian(P, d, len(p.S)).host()
    b = N.connections(P, d).host()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_proxy_energy_grad_fp64():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    V, Pk = _VP(p, 400, 1e-3)
    T = np.concatenate([V, Pk])
    net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
    dT = to_dev(T)
    csr = N.proxy_hamiltonian(P, dT, len(V))
    out, grad, psi = N.energy_grad(P, net, csr, dT)
    ref = O.energy_grad(O.Net(p.net), T, O.proxy_csr(10, p.h, p.eri, V, Pk))
    out = out.cpu().numpy()
    assert abs(out[0] - ref["E"]) < 1e-8
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) < 1e-9
    # the proxy energy lies between the variational energy on V and the bottom of H~'s spectrum
    Ev = O.energy_grad(O.Net(p.net), V, O.hss(10, p.h, p.eri, V), with_grad=False)["E"]
    assert out[0] != Ev


def test_proxy_energy_grad_mixed_vs_quantised_oracle():
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    V, Pk = _VP(p, 2000, 1e-4)
    T = np.concatenate([V, Pk])
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    dT = to_dev(T)
    csr = N.proxy_hamiltonian(P, dT, len(V))
    out, grad, _ = N.energy_grad(P, net, csr, dT)
    ref = O.energy_grad(O.Net(p.net, quant=True), T, O.proxy_csr(16, p.h, p.eri, V, Pk))
    assert abs(out[0].item() - ref["E"]) < 1e-6
    g = grad.double().cpu().numpy()
    assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) < 1e-2


def test_proxy_rejects_overlapping_sets():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    V = p.S[:100]
    Pk = p.S[50:150]  # shares 50 configurations with V
    with pytest.raises(N.NQSError):
        N.proxy_hamiltonian(P, to_dev(np.concatenate([V, Pk])), len(V), o=N.opts(validate=1))
