"""GPU parity of the post-hoc diagonalisation diagnostic E_diag = lambda_min(H_VV) (Sec. 3.5):
Lanczos with full reorthogonalisation on the device against the oracle's dense / iterative
eigensolver, and Delta_opt = E_var - E_diag >= 0."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nS", [("tiny_n10", 1000), ("small_n16", 16384)])
def test_lanczos_min_matches_oracle(name, nS):
    need_gpu()
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    S = p.S[:nS]
    csr = N.connections(P, to_dev(S))
    lam, iters = N.lanczos_min(csr, max_iters=400, tol=1e-14)
    ref = O.e_diag(O.hss(p.wl.norb, p.h, p.eri, S))
    assert abs(lam - ref) < 1e-9 * max(1.0, abs(ref)), (lam, ref, iters)
    assert iters <= 400


def test_delta_opt_nonnegative_and_start_vector():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    d = to_dev(p.S)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
    csr = N.connections(P, d)
    out, _, psi = N.energy_grad(P, net, csr, d, with_grad=False)
    lam, _ = N.lanczos_min(csr)
    lam_psi, _ = N.lanczos_min(csr, start=psi)  # starting from the network's amplitudes
    assert abs(lam - lam_psi) < 1e-9 * abs(lam)
    assert out[0].item() - lam >= -1e-12  # Delta_opt = E_var - E_diag >= 0
