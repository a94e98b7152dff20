"""Pins of the oracle's outer-loop subspace selector (Sec. 2.4.2: Top-K, cumulative mass,
absolute threshold) against a NumPy ranking written independently (lexsort on (key, -|psi|))
and against the protocols' limiting cases. Amplitudes enter as log|psi| (-inf for zero)."""
import numpy as np
import pytest

from oracle import oracle as O


def _rank(T, psi):
    """Positions ordered by |psi| descending, ties by ascending (a, b)."""
    return np.lexsort((T[:, 1], T[:, 0], -np.abs(psi)))


def _log(psi):
    with np.errstate(divide="ignore"):
        return np.log(np.abs(psi))


def _by_key(T, pos):
    pos = np.asarray(pos, np.int64)
    return pos[np.lexsort((T[pos, 1], T[pos, 0]))]


def _random_T(n, seed, ties=False):
    rng = np.random.default_rng(seed)
    keys = set()
    while len(keys) < n:
        keys.add((int(rng.integers(0, 1 << 40)), int(rng.integers(0, 1 << 40))))
    T = np.array(sorted(keys), np.uint64)
    T = T[rng.permutation(n)]  # the selector does not need T sorted
    psi = rng.standard_normal(n) * np.exp(-rng.uniform(0, 10, n))
    if ties:
        psi = np.round(psi * 4) / 4  # many equal |psi|, including zeros
    return T, psi


@pytest.mark.parametrize("ties", [False, True])
@pytest.mark.parametrize("K", [0, 1, 17, 500, 1000, 5000])
def test_topk_equals_numpy_ranking(ties, K):
    T, psi = _random_T(1000, 3 + K, ties)
    want = _by_key(T, _rank(T, psi)[:K])
    assert np.array_equal(O.select(T, _log(psi), O.SELECT_TOPK, K=K), want)


@pytest.mark.parametrize("gamma", [0.0, 0.3, 0.9, 0.999, 1.0])
def test_cumulative_mass_equals_numpy(gamma):
    T, psi = _random_T(800, 7)
    order = _rank(T, psi)
    lg = _log(psi)
    wall = np.exp(2 * (lg - lg.max()))
    w = wall[order]
    D = np.sum(wall)
    cums = np.cumsum(w)
    c = int(np.searchsorted(cums >= gamma * D, True)) + 1 if np.any(cums >= gamma * D) else len(T)
    got = O.select(T, lg, O.SELECT_MASS, param=gamma)
    # the oracle sums in rank order like cumsum; D is compensated there, pairwise here: the count
    # may differ only where the running mass sits within rounding of gamma * D
    if len(got) != c:
        lo, hi = sorted((len(got), c))
        assert abs(cums[hi - 1] - gamma * D) <= 1e-12 * D or abs(cums[lo - 1] - gamma * D) <= 1e-12 * D
    else:
        assert np.array_equal(got, _by_key(T, order[:c]))
    # the kept mass reaches gamma and no shorter prefix does
    kept = np.sum(wall[got])
    assert kept >= gamma * D * (1 - 1e-12)
    assert len(got) == 1 or gamma == 0.0 or cums[len(got) - 2] < gamma * D * (1 + 1e-12)


@pytest.mark.parametrize("eps", [0.0, 1e-6, 1e-3, 0.05, 2.0])
def test_threshold_equals_numpy(eps):
    T, psi = _random_T(600, 11, ties=True)
    lg = _log(psi)
    w = np.exp(2 * (lg - lg.max()))
    p = w / np.sum(w)
    want = _by_key(T, np.nonzero(p > eps)[0])
    assert np.array_equal(O.select(T, lg, O.SELECT_THRESHOLD, param=eps), want)


def test_limits():
    T, psi = _random_T(300, 5)
    psi[:40] = 0.0
    # Top-K with K >= n keeps everything; threshold 0 keeps exactly the nonzero amplitudes;
    # mass 0 keeps one configuration (the largest)
    lg = _log(psi)
    assert len(O.select(T, lg, O.SELECT_TOPK, K=10 ** 9)) == 300
    assert set(O.select(T, lg, O.SELECT_THRESHOLD, param=0.0)) == set(range(40, 300))
    top = O.select(T, lg, O.SELECT_MASS, param=0.0)
    assert list(top) == [int(np.argmax(np.abs(psi)))]
    # a common shift of log|psi| (a normalisation) changes no selection
    for mode, kw in ((O.SELECT_TOPK, dict(K=50)), (O.SELECT_MASS, dict(param=0.7)),
                     (O.SELECT_THRESHOLD, dict(param=1e-3))):
        assert np.array_equal(O.select(T, lg + 3.0, mode, **kw), O.select(T, lg, mode, **kw))
