"""The C ABI's documented argument errors, on CPU: invalid arguments are rejected with the
status codes include/nqs.h states before any device work, so these calls need no GPU; no
exception crosses the boundary."""
import ctypes as C

import numpy as np
import pytest

from paper_2601_21310_b300 import nqs as N

NQS_ERR_ARG, NQS_ERR_NORB = -1, -4


@pytest.fixture(scope="module")
def L():
    return N.lib()


def test_problem_create_rejects_bad_shapes(L):
    h = np.zeros(4, np.float64)
    eri = np.zeros(16, np.float64)
    out = C.c_void_p()
    hp, ep = h.ctypes.data_as(C.c_void_p), eri.ctypes.data_as(C.c_void_p)
    assert L.nqs_problem_create(65, 5, 5, hp, ep, 0.0, C.byref(out)) == NQS_ERR_NORB
    assert L.nqs_problem_create(0, 1, 1, hp, ep, 0.0, C.byref(out)) == NQS_ERR_NORB
    # every spin needs an electron and an empty orbital
    for na, nb in ((0, 1), (1, 0), (2, 1), (1, 2)):
        assert L.nqs_problem_create(2, na, nb, hp, ep, 0.0, C.byref(out)) == NQS_ERR_ARG
    assert out.value is None
    assert L.nqs_problem_create(2, 1, 1, None, ep, 0.0, C.byref(out)) == NQS_ERR_ARG
    assert L.nqs_problem_create(2, 1, 1, hp, ep, 0.0, None) == NQS_ERR_ARG


def test_null_handles_are_rejected(L):
    buf = np.zeros(8, np.float64)
    p = buf.ctypes.data_as(C.c_void_p)
    assert L.nqs_connections(None, p, 1, None, p, None, None) == NQS_ERR_ARG
    assert L.nqs_diag(None, p, 1, p, None) == NQS_ERR_ARG
    assert L.nqs_net_create(None, 8, 8, 0, p, p) == NQS_ERR_ARG
    assert L.nqs_proxy_hamiltonian(None, p, 1, 1, None, p, None) == NQS_ERR_ARG
    assert L.nqs_hb_select(None, p, p, 1, 1e-6, None, p, None) == NQS_ERR_ARG
    assert L.nqs_select(None, p, p, 1, 0, 1, 0.0, None, p, None) == NQS_ERR_ARG
    assert L.nqs_energy_from_psi(None, p, 1, p, None, None) == NQS_ERR_ARG
    assert L.nqs_lanczos_min(None, 10, 1e-12, p, None, None, None) == NQS_ERR_ARG
    assert L.nqs_connections_noalloc(None, p, 1, 0, p, p, p, 1, p, None, None) == NQS_ERR_ARG
    assert L.nqs_gemm_bf16(None, 8, p, 8, 8, 8, 8, p, 8, None, None) == NQS_ERR_ARG
    assert L.nqs_batch_create(0, p, p, p, p, p, p, p, 1, p) == NQS_ERR_ARG
    assert L.nqs_csr_free(None) == NQS_ERR_ARG
    assert L.nqs_pt2_unique(None, p, p, 1, 1, 0, None, None, 0, p, None) == NQS_ERR_ARG


def test_gemm_rejects_empty_shapes(L):
    buf = np.zeros(8, np.float64)
    p = buf.ctypes.data_as(C.c_void_p)
    for M, Nn, K in ((0, 8, 8), (8, 0, 8), (8, 8, 0), (-1, 8, 8)):
        assert L.nqs_gemm_bf16(p, 8, p, 8, M, Nn, K, p, 8, None, None) == NQS_ERR_ARG


def test_every_status_has_a_message(L):
    for code in range(-8, 2):
        msg = L.nqs_status_string(code)
        assert isinstance(msg, bytes) and len(msg) > 0


def test_gemm_ex_rejects_bad_arguments(L):
    """nqs_gemm_bf16_ex: null operands, empty shapes, and leading dimensions shorter than the
    contiguous extent of each operand layout (K for K-major, M or N for MN-major)."""
    buf = np.zeros(64, np.float32)
    p = buf.ctypes.data_as(C.c_void_p)
    ex = L.nqs_gemm_bf16_ex
    assert ex(None, 8, 0, p, 8, 0, 8, 8, 8, p, 8, None, None) == NQS_ERR_ARG
    assert ex(p, 8, 0, None, 8, 0, 8, 8, 8, p, 8, None, None) == NQS_ERR_ARG
    assert ex(p, 8, 0, p, 8, 0, 8, 8, 8, None, 8, None, None) == NQS_ERR_ARG
    for M, Nn, K in ((0, 8, 8), (8, 0, 8), (8, 8, 0)):
        assert ex(p, 8, 1, p, 8, 1, M, Nn, K, p, 8, None, None) == NQS_ERR_ARG
    # K-major needs lda, ldb >= K; MN-major needs lda >= M, ldb >= N
    assert ex(p, 8, 0, p, 16, 0, 8, 8, 16, p, 8, None, None) == NQS_ERR_ARG
    assert ex(p, 16, 0, p, 8, 0, 8, 8, 16, p, 8, None, None) == NQS_ERR_ARG
    assert ex(p, 8, 1, p, 16, 1, 16, 16, 8, p, 16, None, None) == NQS_ERR_ARG
    assert ex(p, 16, 1, p, 8, 1, 16, 16, 8, p, 16, None, None) == NQS_ERR_ARG


def test_gemm_pairing_switch(L):
    """nqs_set_gemm_pairing takes any int (non-zero: on) and leaves the library paired."""
    assert L.nqs_set_gemm_pairing(0) == 0
    assert L.nqs_set_gemm_pairing(7) == 0
    assert L.nqs_set_gemm_pairing(1) == 0
