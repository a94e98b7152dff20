"""GPU parity of the combinatorial kernels (diagonal, enumeration + lookup -> CSR H_SS) against
the oracle, through the C ABI. Pattern and columns bit-exact; values compared exactly where the
summation order is shared, with a 1e-12 guard."""
import numpy as np
import pytest

from gpu_common import need_gpu, nqs, problem_for, small_problem, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _compare_csr(gpu, ref, exact_values=True):
    rp, col, val = gpu.host()
    assert np.array_equal(rp, ref.row_ptr)
    assert np.array_equal(col, ref.col)
    if exact_values:
        assert np.array_equal(val, ref.val), np.abs(val - ref.val).max()
    else:
        assert np.abs(val - ref.val).max() < 1e-12
    assert gpu.n_enumerated == ref.n_enumerated


@pytest.mark.parametrize("name", ["tiny_n10", "small_n16"])
def test_hss_matches_oracle(name):
    need_gpu()
    N = nqs()
    p = synth.make_problem(name)
    P = problem_for(N, p)
    gpu = N.connections(P, to_dev(p.S))
    ref = O.hss(p.wl.norb, p.h, p.eri, p.S)
    _compare_csr(gpu, ref)


@pytest.mark.parametrize("norb,na,nb,nS", [(6, 3, 2, 150), (12, 5, 4, 777), (9, 1, 2, 50)])
def test_hss_unequal_spins_ragged(norb, na, nb, nS):
    need_gpu()
    N = nqs()
    p, nb = small_problem(norb, na, nS, 31 + norb, nb=nb)
    P = N.Problem(norb, na, nb, p.h, p.eri)
    gpu = N.connections(P, to_dev(p.S))
    ref = O.hss(norb, p.h, p.eri, p.S)
    _compare_csr(gpu, ref)


def test_hss_single_det_and_full_space():
    need_gpu()
    N = nqs()
    norb, n = 7, 3
    h, eri, _ = synth.integrals(norb, 14, 8, 3.0)
    P = N.Problem(norb, n, n, h, eri)
    hf = np.array([[7, 7]], np.uint64)
    g = N.connections(P, to_dev(hf))
    rp, col, val = g.host()
    assert rp.tolist() == [0, 1] and col.tolist() == [0]
    assert val[0] == O.diag(norb, h, eri, 7, 7)
    F = synth.full_space(norb, n)
    g = N.connections(P, to_dev(F))
    ref = O.hss(norb, h, eri, F)
    _compare_csr(g, ref)
    assert g.nnz == len(F) * (1 + O.n_excitations(norb, n, n))


def test_hss_symmetric_bit_exact():
    need_gpu()
    import scipy.sparse as sp
    N = nqs()
    p = synth.make_problem("small_n16")
    g = N.connections(N.Problem(16, 8, 8, p.h, p.eri), to_dev(p.S))
    rp, col, val = g.host()
    A = sp.csr_matrix((val, col, rp), shape=(len(p.S),) * 2)
    assert (A != A.T).nnz == 0


def test_diag_matches_oracle():
    need_gpu()
    N = nqs()
    p = synth.make_problem("small_n16")
    P = problem_for(N, p)
    d = N.diag(P, to_dev(p.S)).cpu().numpy()
    ref = np.array([O.diag(16, p.h, p.eri, a, b) for a, b in p.S[:4000]])
    assert np.array_equal(d[:4000], ref)


def test_invalid_inputs_are_rejected():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    bad = p.S[::-1].copy()
    with pytest.raises(N.NQSError, match="sorted"):
        N.connections(P, to_dev(bad))
    bad = p.S.copy()
    bad[3, 0] = np.uint64(0b111)  # three alpha electrons
    with pytest.raises(N.NQSError, match="electron count"):
        N.connections(P, to_dev(bad))
    dup = np.concatenate([p.S[:5], p.S[4:6]])
    with pytest.raises(N.NQSError, match="sorted"):
        N.connections(P, to_dev(dup))
