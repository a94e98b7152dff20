"""nqs_connections_noalloc: the H_SS build for callers that cannot allocate device memory.

Such callers (a host framework that owns every device allocation and gives the library none,
or an embedded solver on a fixed device budget) pass every input and output buffer themselves;
the library keeps its own scratch in a fixed static device array. This file is collected last
so that a run stopping at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from gpu_common import need_gpu, nqs, problem_for, to_dev
from oracle import oracle as O
from paper_2601_21310_b300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(N, P, dets, capacity):
    n = dets.shape[0]
    rp = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
    col = torch.full((max(capacity, 1),), -7, dtype=torch.int32, device="cuda")
    val = torch.full((max(capacity, 1),), np.nan, dtype=torch.float64, device="cuda")
    st, nnz, nen = N.connections_noalloc(P, dets, rp, col, val)
    torch.cuda.synchronize()
    return st, nnz, nen, rp.cpu().numpy(), col.cpu().numpy()[:nnz], val.cpu().numpy()[:nnz]


def test_noalloc_matches_connections_two_calls_in_a_row():
    need_gpu()
    N = nqs()
    cases = []
    for name in ("small_n16", "tiny_n10"):
        p = synth.make_problem(name)
        P = problem_for(N, p)
        dets = to_dev(p.S)
        ref = N.connections(P, dets)
        cases.append((P, dets, ref.host(), ref.n_enumerated))
    # two consecutive calls with different problems share (and must clear) the static scratch
    for P, dets, (rp_ref, col_ref, val_ref), nen_ref in cases:
        st, nnz, nen, rp, col, val = _noalloc(N, P, dets, len(col_ref))
        assert st == 0, N.lib().nqs_last_error()
        assert nnz == len(col_ref) and nen == nen_ref
        assert np.array_equal(rp, rp_ref)
        assert np.array_equal(col, col_ref)
        assert np.abs(val - val_ref).max() <= 1e-12


def test_noalloc_at_the_maximum_size():
    """65536 determinants, the largest input the static scratch accepts; the problem's
    stream-ordered pool is the same before and after the call (nothing allocated from it)."""
    need_gpu()
    N = nqs()
    h, eri, _ = synth.integrals(16, 32, 1, 3.0)
    S = synth.select_S(16, 8, 65536)
    P = N.Problem(16, 8, 8, h, eri)
    dets = to_dev(S)
    ref = N.connections(P, dets)
    rp_ref, col_ref, val_ref = ref.host()
    ref.free()
    torch.cuda.synchronize()
    pool0 = N.pool_usage(P)
    st, nnz, _, rp, col, val = _noalloc(N, P, dets, len(col_ref))
    assert st == 0, N.lib().nqs_last_error()
    assert N.pool_usage(P) == pool0
    assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref)
    assert np.abs(val - val_ref).max() <= 1e-12


def test_noalloc_validation_then_valid_input_matches_oracle():
    """With validation on, an unsorted S and a configuration with the wrong electron count are
    rejected (their flags land in the shared static array); the next valid call still equals
    the oracle's H_SS bit for bit, so nothing left over from the rejected calls leaks into it."""
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    ref = O.hss(10, p.h, p.eri, p.S)
    bad = p.S.copy()
    bad[[3, 4]] = bad[[4, 3]]
    st, *_ = _noalloc(N, P, to_dev(bad), ref.nnz)
    assert st == -2  # NQS_ERR_UNSORTED
    bad = p.S.copy()
    bad[7, 0] |= np.uint64(1 << 9) if not (int(bad[7, 0]) >> 9) & 1 else np.uint64(1 << 8)
    bad = bad[np.lexsort((bad[:, 1], bad[:, 0]))]
    st, *_ = _noalloc(N, P, to_dev(bad), ref.nnz)
    assert st == -3  # NQS_ERR_POPCOUNT
    for _ in range(2):
        st, nnz, _, rp, col, val = _noalloc(N, P, to_dev(p.S), ref.nnz)
        assert st == 0, N.lib().nqs_last_error()
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
        assert np.array_equal(val, ref.val)


def test_noalloc_reports_size_limits():
    need_gpu()
    N = nqs()
    p = synth.make_problem("tiny_n10")
    P = problem_for(N, p)
    dets = to_dev(p.S)
    st, nnz, _, _, _, _ = _noalloc(N, P, dets, 10)
    assert st == -1 and nnz > 10  # capacity too small: nothing written, size reported
    big = synth.select_S(16, 8, 70000)
    P16 = N.Problem(16, 8, 8, *synth.integrals(16, 32, 1, 3.0)[:2])
    st, _, _, _, _, _ = _noalloc(N, P16, to_dev(big), 1)
    assert st == -1
    assert b"65536" in N.lib().nqs_last_error()
