"""Shared helpers of the GPU parity tests (inputs from the seeded generator; expected values
from the oracle only)."""
import numpy as np
import pytest
import torch

from paper_2601_21310_b300 import synth


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def nqs():
    from paper_2601_21310_b300 import build, nqs as N
    build.build()
    return N


def to_dev(S):
    return torch.from_numpy(np.ascontiguousarray(S).view(np.int64)).cuda().view(torch.uint64)


def problem_for(N, p):
    return N.Problem(p.wl.norb, p.wl.nalpha, p.wl.nbeta, p.h, p.eri)


def small_problem(norb, n, nS, seed, hidden=(32, 32), nb=None):
    """A synthetic problem of arbitrary shape (level-major S)."""
    nb = n if nb is None else nb
    h, eri, _ = synth.integrals(norb, 2 * norb, seed, 3.0)
    if nb == n:
        S = synth.select_S(norb, n, nS)
    else:
        F = synth.full_space(norb, n, nb)
        rng = np.random.default_rng(seed)
        S = F[np.sort(rng.choice(len(F), size=min(nS, len(F)), replace=False))]
    net = synth.net_params(norb, n, nb, hidden, seed + 100)
    wl = synth.Workload(f"custom_{norb}_{n}", norb, n, seed, 2 * norb, 3.0, len(S), hidden, False)
    return synth.Problem(wl, h, eri, 0.0, S, net), nb
