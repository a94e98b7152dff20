"""GPU parity of the Asymmetric mode (Sec. 2.4.1, Eqs. asymmetric_energy, asymmetric_gradient)
over T = V + P with the proxy CSR: E_asym, the log-derivative estimator and the exact gradient
against the oracle (FP64 form 1e-8 Ha and 1e-9 relative; mixed form against the
quantisation-matched oracle)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("exact", [False, True])
def test_asym_fp64(exact):
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    V, Pk = _VP(p, 400, 1e-3)
    T = np.concatenate([V, Pk])
    dT = to_dev(T)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
    csr = N.proxy_hamiltonian(P, dT, len(V))
    out, grad, _ = N.asym_energy_grad(P, net, csr, dT, len(V), exact)
    ref = O.asym_energy_grad(O.Net(p.net), V, Pk, O.proxy_csr(10, p.h, p.eri, V, Pk), exact)
    assert abs(out[0].item() - ref["E"]) < 1e-8
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) < 1e-9


def test_asym_mixed_vs_quantised_oracle():
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    V, Pk = _VP(p, 2000, 1e-4)
    T = np.concatenate([V, Pk])
    dT = to_dev(T)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED), N.NQS_MIXED)
    csr = N.proxy_hamiltonian(P, dT, len(V))
    ref_csr = O.proxy_csr(16, p.h, p.eri, V, Pk)
    for exact in (False, True):
        out, grad, _ = N.asym_energy_grad(P, net, csr, dT, len(V), exact)
        ref = O.asym_energy_grad(O.Net(p.net, quant=True), V, Pk, ref_csr, exact)
        assert abs(out[0].item() - ref["E"]) < 1e-6
        g = grad.double().cpu().numpy()
        assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) < 1e-2


def test_asym_without_P_is_variational():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    d = to_dev(p.S)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
    csr = N.connections(P, d)
    ov, gv, _ = N.energy_grad(P, net, csr, d)
    for exact in (False, True):
        oa, ga, _ = N.asym_energy_grad(P, net, csr, d, len(p.S), exact)
        assert abs(oa[0].item() - ov[0].item()) < 1e-12
        assert (np.linalg.norm((ga - gv).cpu().numpy()) <=
                1e-10 * np.linalg.norm(gv.cpu().numpy()))
