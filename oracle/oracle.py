"""ctypes front end of the C oracle (oracle.c). Test infrastructure only.

Each function restates which part of the paper it follows; the arithmetic itself lives in
oracle.c and is documented there.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        u64, i64, dp = C.c_uint64, C.c_int64, C.c_void_p
        L.orc_diag.restype = C.c_double
        L.orc_diag.argtypes = [C.c_int, dp, dp, u64, u64]
        L.orc_element.restype = C.c_double
        L.orc_element.argtypes = [C.c_int, dp, dp, u64, u64, u64, u64, dp]
        L.orc_n_excitations.restype = i64
        L.orc_n_excitations.argtypes = [C.c_int, C.c_int, C.c_int]
        L.orc_excitations.restype = i64
        L.orc_excitations.argtypes = [C.c_int, u64, u64, dp]
        L.orc_hss.restype = C.c_int
        L.orc_hss.argtypes = [C.c_int, dp, dp, dp, i64, C.c_int, dp, dp, dp, dp]
        L.orc_hss_rows.restype = C.c_int
        L.orc_hss_rows.argtypes = [C.c_int, dp, dp, dp, i64, i64, i64, C.c_int, dp, dp, dp]
        L.orc_bf16_round.restype = C.c_double
        L.orc_bf16_round.argtypes = [C.c_double]
        L.orc_amplitudes.restype = C.c_int
        L.orc_amplitudes.argtypes = [dp, dp, i64, dp, dp]
        L.orc_energy_from_psi.restype = C.c_int
        L.orc_energy_from_psi.argtypes = [dp, dp, dp, dp, i64, dp, dp]
        L.orc_n_params.restype = i64
        L.orc_n_params.argtypes = [dp]
        L.orc_energy_grad.restype = C.c_int
        L.orc_energy_grad.argtypes = [dp, dp, i64, dp, dp, dp, dp, dp, dp, dp]
        L.orc_bucket.restype = u64
        L.orc_bucket.argtypes = [u64, u64, u64]
        L.orc_pt2.restype = C.c_int
        L.orc_pt2.argtypes = [C.c_int, dp, dp, dp, i64, dp, C.c_double, i64, i64, dp]
        L.orc_hb_select.restype = i64
        L.orc_hb_select.argtypes = [C.c_int, dp, dp, dp, i64, dp, C.c_double, i64, dp, dp]
        L.orc_hb_select_rows.restype = i64
        L.orc_hb_select_rows.argtypes = [C.c_int, dp, dp, dp, i64, i64, i64, dp, C.c_double, i64,
                                         dp, dp]
        L.orc_select.restype = i64
        L.orc_select.argtypes = [dp, dp, i64, C.c_int, i64, C.c_double, dp]
        L.orc_pt2_eps.restype = C.c_int
        L.orc_pt2_eps.argtypes = [C.c_int, dp, dp, dp, i64, dp, C.c_double, C.c_double, i64, i64,
                                  dp]
        L.orc_pt2_unique.restype = C.c_int
        L.orc_pt2_unique.argtypes = [C.c_int, dp, dp, dp, i64, dp, C.c_double, i64, i64, dp,
                                     i64, dp, dp]
        L.orc_pt2_unique_eps.restype = C.c_int
        L.orc_pt2_unique_eps.argtypes = [C.c_int, dp, dp, dp, i64, dp, C.c_double, C.c_double,
                                         i64, i64, dp, i64, dp, dp]
        L.orc_proxy_csr.restype = C.c_int
        L.orc_proxy_csr.argtypes = [C.c_int, dp, dp, dp, i64, i64, C.c_int, dp, dp, dp]
        L.orc_asym_energy_grad.restype = C.c_int
        L.orc_asym_energy_grad.argtypes = [dp, dp, i64, i64, dp, dp, dp, C.c_int, dp, dp]
        L.orc_num_threads.restype = C.c_int
        L.orc_num_threads.argtypes = []
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def num_threads() -> int:
    return lib().orc_num_threads()


# ------------------------------------------------------------------------------------------
# Slater-Condon rules (Sec. 3.1 names them for the combinatorial kernel)
# ------------------------------------------------------------------------------------------
def diag(norb, h, eri, a, b) -> float:
    h, eri = _f64(h), _f64(eri)
    return lib().orc_diag(norb, _p(h), _p(eri), int(a), int(b))


def element(norb, h, eri, x, y):
    """<y|H|x> and the excitation level (3 = more than a double)."""
    h, eri = _f64(h), _f64(eri)
    lv = C.c_int(0)
    v = lib().orc_element(norb, _p(h), _p(eri), int(x[0]), int(x[1]), int(y[0]), int(y[1]),
                          C.addressof(lv))
    return v, lv.value


def n_excitations(norb, na, nb) -> int:
    return lib().orc_n_excitations(norb, na, nb)


def excitations(norb, a, b) -> np.ndarray:
    """Connected set of one configuration, Eq. (connected_set), canonical order: uint64 [N,2]."""
    na, nb = bin(int(a)).count("1"), bin(int(b)).count("1")
    n = n_excitations(norb, na, nb)
    out = np.zeros((n, 2), np.uint64)
    k = lib().orc_excitations(norb, int(a), int(b), _p(out))
    assert k == n
    return out


@dataclass
class CSR:
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    n_enumerated: int

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        n = self.row_ptr.size - 1
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(n, n))


def hss(norb, h, eri, S) -> CSR:
    """H_SS in CSR, rows in S order, each row [diagonal, hits in canonical excitation order]
    (Sec. 3.1, Algorithm 1 step 1: construct the sparse block H_VV)."""
    h, eri, S = _f64(h), _f64(eri), _u64(S)
    nS = S.shape[0]
    row_ptr = np.zeros(nS + 1, np.int64)
    nen = np.zeros(1, np.int64)
    L = lib()
    st = L.orc_hss(norb, _p(h), _p(eri), _p(S), nS, 0, _p(row_ptr), None, None, _p(nen))
    assert st == 0, st
    nnz = int(row_ptr[-1])
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float64)
    st = L.orc_hss(norb, _p(h), _p(eri), _p(S), nS, 1, _p(row_ptr), _p(col), _p(val), _p(nen))
    assert st == 0, st
    return CSR(row_ptr, col[:nnz], val[:nnz], int(nen[0]))


def hss_rows(norb, h, eri, S, r0: int, r1: int):
    """Rows r0..r1-1 of H_SS (same layout as hss), lookups into all of S: (row_ptr, col, val)
    with row_ptr starting at 0."""
    h, eri, S = _f64(h), _f64(eri), _u64(S)
    nS = S.shape[0]
    rp = np.zeros(r1 - r0 + 1, np.int64)
    L = lib()
    st = L.orc_hss_rows(norb, _p(h), _p(eri), _p(S), nS, r0, r1, 0, _p(rp), None, None)
    assert st == 0, st
    nnz = int(rp[-1])
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float64)
    st = L.orc_hss_rows(norb, _p(h), _p(eri), _p(S), nS, r0, r1, 1, _p(rp), _p(col), _p(val))
    assert st == 0, st
    return rp, col[:nnz], val[:nnz]


# ------------------------------------------------------------------------------------------
# backflow network, amplitudes, energy and gradient (Sec. 2.2, Sec. 2.3.3)
# ------------------------------------------------------------------------------------------
class _Net(C.Structure):
    _fields_ = [("norb", C.c_int), ("na", C.c_int), ("nb", C.c_int), ("H1", C.c_int),
                ("H2", C.c_int), ("quant", C.c_int),
                ("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
                ("W3", C.c_void_p), ("b3", C.c_void_p), ("Phi0", C.c_void_p)]


class Net:
    """Holds FP64 copies of the parameters and the C struct that points at them."""

    def __init__(self, params, quant: bool = False):
        self.arrays = [_f64(x) for x in params.as_list()]
        W1 = self.arrays[0]
        self.norb, self.na, self.nb = params.norb, params.nalpha, params.nbeta
        self.H1, self.H2 = W1.shape[0], self.arrays[2].shape[0]
        self.s = _Net(self.norb, self.na, self.nb, self.H1, self.H2, int(quant),
                      *[x.ctypes.data for x in self.arrays])

    @property
    def ref(self):
        return C.byref(self.s)

    def n_params(self) -> int:
        return lib().orc_n_params(self.ref)

    def unflatten(self, g: np.ndarray):
        out, k = [], 0
        for x in self.arrays[:6]:
            out.append(g[k:k + x.size].reshape(x.shape))
            k += x.size
        return out


def bf16_round(x: float) -> float:
    return lib().orc_bf16_round(float(x))


def amplitudes(net: Net, S):
    """(log|psi|, sign) for each x in S, Eq. (backflow_amplitude) in spin-blocked form."""
    S = _u64(S)
    nS = S.shape[0]
    la = np.zeros(nS)
    sg = np.zeros(nS, np.int8)
    st = lib().orc_amplitudes(net.ref, _p(S), nS, _p(la), _p(sg))
    assert st >= 0, st
    return la, sg


def energy_from_psi(csr: CSR, psi):
    """Rayleigh quotient of a given psi on H_SS, Eq. (variational_energy): (E, N, D), v."""
    psi = _f64(psi)
    nS = psi.size
    out = np.zeros(3)
    v = np.zeros(nS)
    lib().orc_energy_from_psi(_p(csr.row_ptr), _p(csr.col), _p(csr.val), _p(psi), nS, _p(out),
                              _p(v))
    return out, v


def energy_grad(net: Net, S, csr: CSR, with_grad: bool = True):
    """E_S and dE/dtheta, Eqs. (variational_energy), (variational_gradient).
    Returns dict(E, N, D, maxlog, grad, psi, v)."""
    S = _u64(S)
    nS = S.shape[0]
    out = np.zeros(4)
    grad = np.zeros(net.n_params()) if with_grad else None
    psi = np.zeros(nS)
    v = np.zeros(nS)
    st = lib().orc_energy_grad(net.ref, _p(S), nS, _p(csr.row_ptr), _p(csr.col), _p(csr.val),
                               _p(out), _p(grad) if with_grad else None, _p(psi), _p(v))
    assert st >= 0, st
    return dict(E=out[0], N=out[1], D=out[2], maxlog=out[3], grad=grad, psi=psi, v=v)


# ------------------------------------------------------------------------------------------
# Epstein-Nesbet PT2 (Eq. pt2_correction)
# ------------------------------------------------------------------------------------------
def bucket(a, b, nbuckets) -> int:
    return int(lib().orc_bucket(int(a), int(b), int(nbuckets)))


def pt2(norb, h, eri, S, psi, E, nbuckets: int = 1, bucket_id: int = -1, eps: float = 0.0):
    """Returns dict(ext, int, n_unique, D, n_emitted). bucket_id >= 0 restricts both terms to the
    configurations of that hash bucket. eps > 0 screens the external contributions
    (|H_x'y psi_y| >= eps, Sec. 3.3); the internal term stays exact."""
    h, eri, S, psi = _f64(h), _f64(eri), _u64(S), _f64(psi)
    out = np.zeros(5)
    st = lib().orc_pt2_eps(norb, _p(h), _p(eri), _p(S), S.shape[0], _p(psi), float(E),
                           float(eps), int(nbuckets), int(bucket_id), _p(out))
    assert st == 0, st
    return dict(ext=out[0], int=out[1], n_unique=int(out[2]), D=out[3], n_emitted=int(out[4]))


def pt2_unique(norb, h, eri, S, psi, E, nbuckets: int = 1, bucket_id: int = -1,
               eps: float = 0.0):
    """The deduplicated external set of pt2 (Eq. pt2_correction): (keys uint64 [n, 2] ascending
    by (a, b), c [n] with c(x') = sum_{y in S} H_x'y psi_y) over C minus S, restricted to one
    hash bucket when bucket_id >= 0, plus pt2's result dict. eps > 0: the screened set, x' with
    at least one contribution |H_x'y psi_y| >= eps and c(x') the sum of those (Sec. 3.3)."""
    h, eri, S, psi = _f64(h), _f64(eri), _u64(S), _f64(psi)
    out = np.zeros(5)
    L = lib()
    args = (norb, _p(h), _p(eri), _p(S), S.shape[0], _p(psi), float(E))
    tail = (int(nbuckets), int(bucket_id), _p(out))

    def call(n, keys, c):
        if eps > 0.0:
            return L.orc_pt2_unique_eps(*args, float(eps), *tail, n, keys, c)
        return L.orc_pt2_unique(*args, *tail, n, keys, c)

    st = call(0, None, None)
    assert st == 0, st
    n = int(out[2])
    keys = np.zeros((max(n, 1), 2), np.uint64)
    c = np.zeros(max(n, 1))
    st = call(n, _p(keys), _p(c))
    assert st == 0, st
    return keys[:n], c[:n], dict(ext=out[0], int=out[1], n_unique=n, D=out[3])


# ------------------------------------------------------------------------------------------
# heat-bath screened perturbative set (Eq. hb_screen, Sec. 3.3)
# ------------------------------------------------------------------------------------------
def hb_select(norb, h, eri, S, psi, eps, rows=None):
    """P = {x' not in S : max_x |H_x'x psi_x| >= eps}: (keys uint64 [n, 2] ascending,
    max coupling [n]). rows=(r0, r1) takes the maximum over the parents S[r0:r1] only."""
    h, eri, S, psi = _f64(h), _f64(eri), _u64(S), _f64(psi)
    nS = S.shape[0]
    r0, r1 = rows if rows is not None else (0, nS)
    L = lib()
    args = (norb, _p(h), _p(eri), _p(S), nS, r0, r1, _p(psi), float(eps))
    n = L.orc_hb_select_rows(*args, 0, None, None)
    assert n >= 0, n
    keys = np.zeros((max(n, 1), 2), np.uint64)
    mx = np.zeros(max(n, 1))
    n2 = L.orc_hb_select_rows(*args, n, _p(keys), _p(mx))
    assert n2 == n
    return keys[:n], mx[:n]


# ------------------------------------------------------------------------------------------
# subspace selection of the outer loop (Sec. 2.4.2, Algorithm 1 step 3)
# ------------------------------------------------------------------------------------------
SELECT_TOPK, SELECT_MASS, SELECT_THRESHOLD = 0, 1, 2


def select(T, logabs, mode, K=0, param=0.0):
    """Positions in T of the kept configurations, ascending by key (amplitudes as log|psi|)."""
    T, logabs = _u64(T), _f64(logabs)
    out = np.zeros(max(T.shape[0], 1), np.int64)
    c = lib().orc_select(_p(T), _p(logabs), T.shape[0], int(mode), int(K), float(param), _p(out))
    assert c >= 0, c
    return out[:c]


# ------------------------------------------------------------------------------------------
# Proxy mode (Sec. 2.4.1): the proxy Hamiltonian of Eq. (proxy_hamiltonian) on T = V + P
# ------------------------------------------------------------------------------------------
def proxy_csr(norb, h, eri, V, P) -> CSR:
    """CSR of H~ over T = [V; P] (V and P each sorted): rows of V hold every connection inside T,
    rows of P the diagonal and their connections to V only. E_proxy and its gradient are
    energy_grad(net, T, proxy_csr(...))."""
    h, eri = _f64(h), _f64(eri)
    T = _u64(np.concatenate([_u64(V).reshape(-1, 2), _u64(P).reshape(-1, 2)]))
    nV, nT = len(V), T.shape[0]
    row_ptr = np.zeros(nT + 1, np.int64)
    L = lib()
    st = L.orc_proxy_csr(norb, _p(h), _p(eri), _p(T), nV, nT, 0, _p(row_ptr), None, None)
    assert st == 0, st
    nnz = int(row_ptr[-1])
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float64)
    st = L.orc_proxy_csr(norb, _p(h), _p(eri), _p(T), nV, nT, 1, _p(row_ptr), _p(col), _p(val))
    assert st == 0, st
    return CSR(row_ptr, col[:nnz], val[:nnz], 0)


def asym_energy_grad(net: Net, V, P, csr: CSR, exact: bool, with_grad: bool = True):
    """Asymmetric mode on T = [V; P] with the proxy CSR over T: dict(E, N, D, maxlog, grad).
    exact=False: the log-derivative estimator (Eq. asymmetric_gradient); exact=True: the
    derivative of E_asym."""
    T = _u64(np.concatenate([_u64(V).reshape(-1, 2), _u64(P).reshape(-1, 2)]))
    out = np.zeros(4)
    grad = np.zeros(net.n_params()) if with_grad else None
    st = lib().orc_asym_energy_grad(net.ref, _p(T), T.shape[0], len(V), _p(csr.row_ptr),
                                    _p(csr.col), _p(csr.val), int(exact), _p(out),
                                    _p(grad) if with_grad else None)
    assert st >= 0, st
    return dict(E=out[0], N=out[1], D=out[2], maxlog=out[3], grad=grad)


# ------------------------------------------------------------------------------------------
# post-hoc diagonalisation diagnostic E_diag = lambda_min(H_VV) (Sec. 3.5)
# ------------------------------------------------------------------------------------------
def e_diag(csr: CSR) -> float:
    """Lowest eigenvalue of the CSR matrix: dense eigvalsh up to 4000 rows, else SciPy's
    implicitly restarted Lanczos (eigsh, smallest algebraic) to 1e-13."""
    A = csr.to_scipy()
    if A.shape[0] <= 4000:
        return float(np.linalg.eigvalsh(A.toarray())[0])
    import scipy.sparse.linalg as sla
    return float(sla.eigsh(A, k=1, which="SA", tol=1e-13, return_eigenvectors=False)[0])
