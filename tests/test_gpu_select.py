"""GPU parity of the outer-loop subspace selector (Sec. 2.4.2: Top-K, cumulative mass, absolute
threshold) against the oracle, through the C ABI. Top-K is compared bit for bit; the mass and
threshold protocols compare exactly except for configurations whose running mass or weight sits
within rounding of the cutoff (the device sums in another fixed order than the oracle)."""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _T_and_logabs(n, norb, nel, seed, ties=False, zeros=0):
    """n distinct configurations of the (norb, nel, nel) sector in shuffled order, log|psi|
    spread over many decades."""
    rng = np.random.default_rng(seed)
    T = synth.select_S(norb, nel, n)
    T = T[rng.permutation(len(T))]
    lg = rng.normal(0.0, 3.0, len(T))
    if ties:
        lg = np.round(lg)
    if zeros:
        lg[rng.choice(len(T), zeros, replace=False)] = -np.inf
    return T, lg


def _gpu(N, P, T, lg, mode, K=0, param=0.0):
    r = N.select(P, to_dev(T), torch.from_numpy(lg).cuda(), mode, K=K, param=param)
    d = r["dets"].cpu().view(torch.int64).numpy().view(np.uint64)
    return d, r["logabs"].cpu().numpy(), r["index"].cpu().numpy()


def _check_output(T, lg, d, v, ix):
    assert np.array_equal(d, T[ix])
    assert np.array_equal(v, lg[ix])
    if len(d) > 1:
        a, b = d[:, 0], d[:, 1]
        assert np.all((a[1:] > a[:-1]) | ((a[1:] == a[:-1]) & (b[1:] > b[:-1])))


@pytest.mark.parametrize("norb,nel,n", [(10, 5, 3000), (16, 8, 50000), (30, 12, 40000),
                                        (42, 24, 20000)])
@pytest.mark.parametrize("ties", [False, True])
def test_topk_bit_exact(norb, nel, n, ties):
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(norb, 2 * norb, 1, 3.0)
    P = N.Problem(norb, nel, nel, h, eri)
    T, lg = _T_and_logabs(n, norb, nel, norb + n, ties=ties, zeros=n // 10)
    for K in (0, 1, 777, n // 2, n, 10 * n):
        d, v, ix = _gpu(N, P, T, lg, N.SELECT_TOPK, K=K)
        assert np.array_equal(ix, O.select(T, lg, O.SELECT_TOPK, K=K)), K
        _check_output(T, lg, d, v, ix)


def _weights(lg):
    return np.exp(2 * (lg - lg.max()))


def _rank(T, lg):
    return np.lexsort((T[:, 1], T[:, 0], -lg))


@pytest.mark.parametrize("gamma", [0.0, 0.5, 0.9, 0.999, 1.0])
def test_mass_matches_oracle(gamma):
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    T, lg = _T_and_logabs(60000, 16, 8, 3, zeros=100)
    d, v, ix = _gpu(N, P, T, lg, N.SELECT_MASS, param=gamma)
    ref = O.select(T, lg, O.SELECT_MASS, param=gamma)
    _check_output(T, lg, d, v, ix)
    if len(ix) != len(ref):
        w = _weights(lg)[_rank(T, lg)]
        cums = np.cumsum(w)
        target = gamma * w.sum()
        for c in (len(ix), len(ref)):
            # both counts sit where the running mass is within rounding of the target
            assert abs(cums[c - 1] - target) <= 1e-12 * w.sum() or (
                c > 1 and abs(cums[c - 2] - target) <= 1e-12 * w.sum())
    else:
        assert np.array_equal(ix, ref)


@pytest.mark.parametrize("eps", [0.0, 1e-9, 1e-6, 1e-3, 0.5])
def test_threshold_matches_oracle(eps):
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    T, lg = _T_and_logabs(60000, 16, 8, 4, ties=True, zeros=500)
    d, v, ix = _gpu(N, P, T, lg, N.SELECT_THRESHOLD, param=eps)
    ref = O.select(T, lg, O.SELECT_THRESHOLD, param=eps)
    _check_output(T, lg, d, v, ix)
    diff = set(ix.tolist()) ^ set(ref.tolist())
    if diff:
        w = _weights(lg)
        D = w.sum()
        for q in diff:
            assert abs(w[q] / D - eps) <= 1e-12 * max(eps, 1e-300), q


def test_select_edge_cases():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    T, lg = _T_and_logabs(500, 10, 5, 9)
    # one configuration
    d, v, ix = _gpu(N, P, T[:1], lg[:1], N.SELECT_TOPK, K=5)
    assert list(ix) == [0]
    # every amplitude zero: Top-K still ranks by key; threshold keeps nothing
    z = np.full(len(T), -np.inf)
    d, v, ix = _gpu(N, P, T, z, N.SELECT_TOPK, K=10)
    assert np.array_equal(ix, O.select(T, z, O.SELECT_TOPK, K=10))
    # invalid inputs
    bad = lg.copy()
    bad[3] = np.nan
    with pytest.raises(N.NQSError):
        N.select(P, to_dev(T), torch.from_numpy(bad).cuda(), N.SELECT_TOPK, K=3)
    with pytest.raises(N.NQSError):
        N.select(P, to_dev(T), torch.from_numpy(lg).cuda(), N.SELECT_MASS, param=1.5)
    with pytest.raises(N.NQSError):
        N.select(P, to_dev(T), torch.from_numpy(lg).cuda(), 7)
    dup = np.concatenate([T[:10], T[:1]])
    with pytest.raises(N.NQSError):
        N.select(P, to_dev(dup), torch.from_numpy(lg[:11]).cuda(), N.SELECT_TOPK, K=3,
                 o=N.opts(validate=1))


def test_outer_loop_round_trip():
    """Algorithm 1 steps 1 and 3 on the device: screened P from S, amplitudes on T = S + P,
    Top-K back to |S| configurations; the result matches the oracle's selection on the same
    amplitudes."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    S = to_dev(p.S)
    net = N.Net(P, N.net_tensors(p.net, N.NQS_FP64), N.NQS_FP64)
    la, sg, _ = N.amplitudes(P, net, S, o=N.opts(precision=N.NQS_FP64, validate=0))
    psi = (sg.double() * torch.exp(la - la.max()))
    psi = psi / torch.linalg.norm(psi)
    hb = N.hb_select(P, S, psi, 1e-4)
    T = torch.cat([S.view(torch.int64), hb["dets"].view(torch.int64)]).view(torch.uint64)
    laT, _, _ = N.amplitudes(P, net, T, o=N.opts(precision=N.NQS_FP64, validate=0))
    r = N.select(P, T, laT, N.SELECT_TOPK, K=len(p.S))
    Th = T.cpu().view(torch.int64).numpy().view(np.uint64)
    ref = O.select(Th, laT.cpu().numpy(), O.SELECT_TOPK, K=len(p.S))
    assert np.array_equal(r["index"].cpu().numpy(), ref)
    assert r["dets"].shape[0] == len(p.S)
