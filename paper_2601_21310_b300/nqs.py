"""Python binding of the C ABI in include/nqs.h (argument marshalling only).

Every computation runs in libnqs.so on the GPU; this module converts torch tensors to device
pointers, fills the option struct and turns status codes into exceptions. There is no CPU
path: if the library or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnqs.so")

NQS_FP64 = 0
NQS_MIXED = 1
NQS_WARN_SINGULAR = 1
NQS_ERR_ARG = -1
NQS_ERR_OOM = -5
NQS_ERR_TIMEOUT = -7

_lib = None


class NQSError(RuntimeError):
    pass


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("buckets", C.c_int), ("chunk", C.c_int64),
                ("validate", C.c_int), ("internal_pt2", C.c_int), ("eps_pt2", C.c_double),
                ("batch_log2", C.c_int), ("reserved", C.c_int * 5)]


class CSRStruct(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("nnz", C.c_int64), ("n_rows", C.c_int64)]


class DetSetStruct(C.Structure):
    _fields_ = [("dets", C.c_void_p), ("value", C.c_void_p), ("index", C.c_void_p),
                ("n", C.c_int64), ("n_emitted", C.c_int64), ("n_examined", C.c_int64)]


EXPORTS = {
    # name: (restype, argtypes)
    "nqs_opts_default": (None, [C.c_void_p]),
    "nqs_status_string": (C.c_char_p, [C.c_int]),
    "nqs_version": (C.c_char_p, []),
    "nqs_last_error": (C.c_char_p, []),
    "nqs_problem_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_void_p]),
    "nqs_problem_destroy": (C.c_int, [C.c_void_p]),
    "nqs_net_create": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "nqs_net_destroy": (C.c_int, [C.c_void_p]),
    "nqs_net_num_params": (C.c_int64, [C.c_void_p]),
    "nqs_diag": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "nqs_connections": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "nqs_csr_free": (C.c_int, [C.c_void_p]),
    "nqs_csr_free_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nqs_proxy_hamiltonian": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "nqs_amplitudes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_energy_from_psi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "nqs_energy_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_asym_energy_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                       C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "nqs_lanczos_min": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "nqs_pt2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_pt2_hss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_pt2_unique": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                 C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_void_p]),
    "nqs_pt2_unique_screened": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                          C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_int64, C.c_void_p, C.c_void_p]),
    "nqs_hb_select": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_detset_free": (C.c_int, [C.c_void_p]),
    "nqs_select": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int64,
                             C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_wait_probe": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "nqs_set_scratch_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "nqs_pool_usage": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "nqs_profile_enable": (C.c_int, [C.c_int]),
    "nqs_profile_reset": (C.c_int, []),
    "nqs_profile_read": (C.c_int, [C.c_char_p, C.c_void_p, C.c_void_p]),
    "nqs_launch_count": (C.c_int64, []),
    "nqs_batch_create": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "nqs_batch_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nqs_batch_capture": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nqs_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nqs_batch_destroy": (C.c_int, [C.c_void_p]),
    "nqs_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "nqs_batch_get_mode": (C.c_int, [C.c_void_p]),
    "nqs_set_autotune": (C.c_int, [C.c_int]),
    "nqs_set_gemm_pairing": (C.c_int, [C.c_int]),
    "nqs_autotune_entries": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "nqs_gemm_bf16": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                                C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "nqs_gemm_bf16_ex": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                   C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                                   C.c_void_p, C.c_void_p]),
    "nqs_connections_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
}

PROFILED = ["conn_count", "conn_fill", "pt2_count", "pt2_emit", "rs_hist", "rs_scatter",
            "seg_reduce", "gemm", "lu", "spmv", "layer1", "unique_terms", "heads", "scan",
            "hb_select", "select"]


def lib():
    """Load libnqs.so (in-tree build). Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise NQSError(f"{LIB_PATH} is missing: build it with paper_2601_21310_b300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


_cudart_lib = None


def _cudart():
    """The CUDA runtime already loaded by torch (same soname), for raw device-to-host copies."""
    global _cudart_lib
    if _cudart_lib is None:
        torch.cuda.init()
        _cudart_lib = C.CDLL("libcudart.so.13")
        _cudart_lib.cudaMemcpy.restype = C.c_int
        _cudart_lib.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
    return _cudart_lib


def _check(status: int, what: str):
    if status < 0:
        L = lib()
        msg = L.nqs_status_string(status).decode()
        detail = L.nqs_last_error().decode()
        raise NQSError(f"{what}: {msg} ({status}) {detail}")
    return status


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dets(d: torch.Tensor) -> torch.Tensor:
    if not (d.is_cuda and d.dtype == torch.uint64 and d.dim() == 2 and d.shape[1] == 2):
        raise NQSError("dets must be a CUDA uint64 tensor of shape [n, 2]")
    return d.contiguous()


def opts(precision=NQS_FP64, buckets=1, chunk=0, validate=1, internal_pt2=1,
         eps_pt2=0.0, batch_log2=0) -> Opts:
    o = Opts()
    lib().nqs_opts_default(C.byref(o))
    o.precision, o.buckets, o.chunk = precision, buckets, chunk
    o.validate, o.internal_pt2, o.eps_pt2 = validate, internal_pt2, eps_pt2
    o.batch_log2 = batch_log2
    return o


class Problem:
    """nqs_problem: device copies of h and the ERIs (Sec. 3.3 Hamiltonian input)."""

    def __init__(self, norb: int, nalpha: int, nbeta: int, h, eri, ecore: float = 0.0):
        import numpy as np
        h = np.ascontiguousarray(h, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta
        handle = C.c_void_p()
        _check(lib().nqs_problem_create(norb, nalpha, nbeta, h.ctypes.data_as(C.c_void_p),
                                        eri.ctypes.data_as(C.c_void_p), ecore, C.byref(handle)),
               "nqs_problem_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            lib().nqs_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """nqs_net over caller-owned device parameters [W1, b1, W2, b2, W3, b3, Phi0]."""

    def __init__(self, problem: Problem, params: list, dtype: int):
        self.problem = problem
        self.params = [p.contiguous() for p in params]
        self.dtype = dtype
        H1, H2 = self.params[0].shape[0], self.params[2].shape[0]
        arr = (C.c_void_p * 7)(*[p.data_ptr() for p in self.params])
        handle = C.c_void_p()
        _check(lib().nqs_net_create(problem.handle, H1, H2, dtype, arr, C.byref(handle)),
               "nqs_net_create")
        self.handle = handle

    def num_params(self) -> int:
        return lib().nqs_net_num_params(self.handle)

    def grad_dtype(self):
        return torch.float64 if self.dtype == NQS_FP64 else torch.float32

    def split(self, flat: torch.Tensor):
        out, k = [], 0
        for p in self.params[:6]:
            out.append(flat[k:k + p.numel()].view(p.shape))
            k += p.numel()
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().nqs_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_tensors(params, dtype: int, device="cuda") -> list:
    """Device tensors for a synth.NetParams in the requested precision form. The mixed form
    rounds weights to bfloat16 (through float32) and biases / Phi0 to float32."""
    ts = [torch.from_numpy(x.copy()) for x in params.as_list()]
    if dtype == NQS_FP64:
        return [t.to(device=device, dtype=torch.float64).contiguous() for t in ts]
    out = []
    for i, t in enumerate(ts):
        t32 = t.to(torch.float32)
        out.append((t32.to(torch.bfloat16) if i in (0, 2, 4) else t32).to(device).contiguous())
    return out


class CSR:
    """Library-owned H_SS in CSR (freed with nqs_csr_free). Holds a reference to its problem so
    that the problem is never destroyed before the matrix."""

    def __init__(self, st: CSRStruct, n_enumerated: int, problem=None):
        self.s = st
        self.n_enumerated = n_enumerated
        self.problem = problem

    @property
    def nnz(self) -> int:
        return self.s.nnz

    @property
    def n_rows(self) -> int:
        return self.s.n_rows

    def host(self):
        """(row_ptr, col, val) copied to host numpy arrays."""
        import numpy as np
        torch.cuda.synchronize()
        rp = np.zeros(self.n_rows + 1, np.int64)
        col = np.zeros(max(self.nnz, 1), np.int32)
        val = np.zeros(max(self.nnz, 1), np.float64)
        cudart = _cudart()
        for dst, src, nb in ((rp, self.s.row_ptr, rp.nbytes), (col, self.s.col, self.nnz * 4),
                             (val, self.s.val, self.nnz * 8)):
            if nb:
                st = cudart.cudaMemcpy(C.c_void_p(dst.ctypes.data), C.c_void_p(src),
                                       C.c_size_t(nb), 2)
                if st != 0:
                    raise NQSError(f"cudaMemcpy failed ({st})")
        return rp, col[:self.nnz], val[:self.nnz]

    def host_rows(self, r0: int, r1: int):
        """Rows r0..r1-1 copied to host: (row_ptr starting at 0, col, val)."""
        import numpy as np
        torch.cuda.synchronize()
        cudart = _cudart()
        rp = np.zeros(r1 - r0 + 1, np.int64)
        st = cudart.cudaMemcpy(C.c_void_p(rp.ctypes.data), C.c_void_p(self.s.row_ptr + 8 * r0),
                               C.c_size_t(rp.nbytes), 2)
        if st != 0:
            raise NQSError(f"cudaMemcpy failed ({st})")
        a, b = int(rp[0]), int(rp[-1])
        col = np.zeros(max(b - a, 1), np.int32)
        val = np.zeros(max(b - a, 1), np.float64)
        for dst, src, nb in ((col, self.s.col + 4 * a, (b - a) * 4),
                             (val, self.s.val + 8 * a, (b - a) * 8)):
            if nb and cudart.cudaMemcpy(C.c_void_p(dst.ctypes.data), C.c_void_p(src),
                                        C.c_size_t(nb), 2) != 0:
                raise NQSError("cudaMemcpy failed")
        return rp - a, col[:b - a], val[:b - a]

    def free(self):
        """Release the matrix after the whole device is idle."""
        if self.s is not None and self.s.row_ptr:
            lib().nqs_csr_free(C.byref(self.s))

    def free_async(self, stream=None):
        """Release the matrix in the order of `stream` (default: torch's current stream); work on
        other streams that reads it must be ordered before this call."""
        if self.s is not None and self.s.row_ptr:
            _check(lib().nqs_csr_free_async(C.byref(self.s), _stream(stream)),
                   "nqs_csr_free_async")

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def diag(problem: Problem, dets: torch.Tensor, stream=None) -> torch.Tensor:
    dets = _dets(dets)
    out = torch.empty(dets.shape[0], dtype=torch.float64, device=dets.device)
    _check(lib().nqs_diag(problem.handle, _ptr(dets), dets.shape[0], _ptr(out), _stream(stream)),
           "nqs_diag")
    return out


def connections(problem: Problem, dets: torch.Tensor, o: Opts | None = None, stream=None) -> CSR:
    dets = _dets(dets)
    st = CSRStruct()
    nen = C.c_int64(0)
    _check(lib().nqs_connections(problem.handle, _ptr(dets), dets.shape[0],
                                 C.byref(o) if o else None, C.byref(st), C.byref(nen),
                                 _stream(stream)), "nqs_connections")
    return CSR(st, nen.value, problem)


def proxy_hamiltonian(problem: Problem, T: torch.Tensor, nV: int, o: Opts | None = None,
                      stream=None) -> CSR:
    """H~ of the Proxy mode (Eq. proxy_hamiltonian) over T = [V; P] as a library-owned CSR."""
    T = _dets(T)
    st = CSRStruct()
    _check(lib().nqs_proxy_hamiltonian(problem.handle, _ptr(T), int(nV), T.shape[0],
                                       C.byref(o) if o else None, C.byref(st), _stream(stream)),
           "nqs_proxy_hamiltonian")
    return CSR(st, 0, problem)


def connections_noalloc(problem: Problem, dets: torch.Tensor, row_ptr: torch.Tensor,
                        col: torch.Tensor, val: torch.Tensor, validate: bool = True, stream=None):
    """H_SS into caller-owned buffers with the library's static scratch (no device
    allocation). Returns (status, nnz, n_enumerated); a negative status is returned, not
    raised, so that a caller can read the nnz it needs."""
    dets = _dets(dets)
    nnz = C.c_int64(0)
    nen = C.c_int64(0)
    st = lib().nqs_connections_noalloc(problem.handle, _ptr(dets), dets.shape[0], int(validate),
                                       _ptr(row_ptr), _ptr(col), _ptr(val), col.numel(),
                                       C.byref(nnz), C.byref(nen), _stream(stream))
    return st, nnz.value, nen.value


def amplitudes(problem: Problem, net: Net, dets: torch.Tensor, o: Opts | None = None,
               stream=None):
    dets = _dets(dets)
    n = dets.shape[0]
    la = torch.empty(n, dtype=torch.float64, device=dets.device)
    sg = torch.empty(n, dtype=torch.int8, device=dets.device)
    o = o or opts(precision=net.dtype)
    st = _check(lib().nqs_amplitudes(problem.handle, net.handle, _ptr(dets), n, _ptr(la), _ptr(sg),
                                     C.byref(o), _stream(stream)), "nqs_amplitudes")
    return la, sg, st


def energy_from_psi(csr: CSR, psi: torch.Tensor, stream=None):
    psi = psi.contiguous()
    out = torch.empty(3, dtype=torch.float64, device=psi.device)
    v = torch.empty_like(psi)
    _check(lib().nqs_energy_from_psi(C.byref(csr.s), _ptr(psi), psi.shape[0], _ptr(out), _ptr(v),
                                     _stream(stream)), "nqs_energy_from_psi")
    return out, v


def energy_grad(problem: Problem, net: Net, csr: CSR, dets: torch.Tensor, with_grad=True,
                o: Opts | None = None, stream=None, out=None, grad=None, psi=None):
    """Returns (out[4] = E, N, D, max log|psi|, grad or None, psi~), all device tensors."""
    dets = _dets(dets)
    n = dets.shape[0]
    dev = dets.device
    out = out if out is not None else torch.empty(4, dtype=torch.float64, device=dev)
    if with_grad and grad is None:
        grad = torch.empty(net.num_params(), dtype=net.grad_dtype(), device=dev)
    psi = psi if psi is not None else torch.empty(n, dtype=torch.float64, device=dev)
    o = o or opts(precision=net.dtype, validate=0)
    _check(lib().nqs_energy_grad(problem.handle, net.handle, C.byref(csr.s), _ptr(dets), n,
                                 _ptr(out), _ptr(grad) if with_grad else None, _ptr(psi),
                                 C.byref(o), _stream(stream)), "nqs_energy_grad")
    return out, (grad if with_grad else None), psi


def asym_energy_grad(problem: Problem, net: Net, csr: CSR, T: torch.Tensor, nV: int,
                     exact: bool, with_grad=True, o: Opts | None = None, stream=None):
    """Asymmetric mode over T = [V; P] with the proxy CSR: (out[4] = E, N, D, max log|psi|,
    grad or None, psi~ over T)."""
    T = _dets(T)
    n = T.shape[0]
    out = torch.empty(4, dtype=torch.float64, device=T.device)
    grad = torch.empty(net.num_params(), dtype=net.grad_dtype(), device=T.device) \
        if with_grad else None
    psi = torch.empty(n, dtype=torch.float64, device=T.device)
    o = o or opts(precision=net.dtype, validate=0)
    _check(lib().nqs_asym_energy_grad(problem.handle, net.handle, C.byref(csr.s), _ptr(T), n,
                                      int(nV), int(exact), _ptr(out), _ptr(grad), _ptr(psi),
                                      C.byref(o), _stream(stream)), "nqs_asym_energy_grad")
    return out, grad, psi


def lanczos_min(csr: CSR, max_iters: int = 300, tol: float = 1e-13,
                start: torch.Tensor | None = None, stream=None):
    """E_diag = lambda_min of the CSR matrix: (eigenvalue, iterations)."""
    ev = C.c_double(0)
    it = C.c_int(0)
    _check(lib().nqs_lanczos_min(C.byref(csr.s), int(max_iters), float(tol),
                                 _ptr(start.contiguous()) if start is not None else None,
                                 C.byref(ev), C.byref(it), _stream(stream)), "nqs_lanczos_min")
    return ev.value, it.value


def pt2(problem: Problem, dets: torch.Tensor, psi: torch.Tensor, E: float, buckets: int = 1,
        o: Opts | None = None, stream=None, hss: "CSR | None" = None):
    """Epstein-Nesbet PT2. Returns dict(ext, int, n_unique, n_emitted, partials[B,2]). With hss
    (H_SS of the same dets from connections()) the screened internal term uses it."""
    import numpy as np
    dets = _dets(dets)
    psi = psi.contiguous()
    o = o or opts(buckets=buckets)
    out = np.zeros(5)
    parts = np.zeros(2 * max(o.buckets, 1))
    outp = out.ctypes.data_as(C.c_void_p)
    partp = parts.ctypes.data_as(C.c_void_p) if o.buckets > 0 else None
    if hss is None:
        _check(lib().nqs_pt2(problem.handle, _ptr(dets), _ptr(psi), dets.shape[0], float(E),
                             C.byref(o), outp, partp, _stream(stream)), "nqs_pt2")
    else:
        _check(lib().nqs_pt2_hss(problem.handle, _ptr(dets), _ptr(psi), dets.shape[0], float(E),
                                 C.byref(hss.s), C.byref(o), outp, partp, _stream(stream)),
               "nqs_pt2_hss")
    return dict(ext=out[0], int=out[1], n_unique=int(out[2]), n_emitted=int(out[3]),
                buckets=int(out[4]), partials=parts.reshape(-1, 2) if o.buckets > 0 else None)


def pt2_unique(problem: Problem, dets: torch.Tensor, psi: torch.Tensor, buckets: int = 1,
               bucket: int = 0, eps: float = 0.0, stream=None):
    """The deduplicated external set of nqs_pt2 for one hash bucket: (configurations uint64
    [n, 2] ascending by key, c(x') float64 [n]) on the device; with eps > 0 the screened set
    (nqs_pt2_unique_screened). Sizes the output with a first call that reports the set's size."""
    dets = _dets(dets)
    psi = psi.contiguous()
    n = C.c_int64(0)
    L = lib()

    def call(out, c, cap):
        if eps > 0.0:
            return L.nqs_pt2_unique_screened(problem.handle, _ptr(dets), _ptr(psi),
                                             dets.shape[0], float(eps), int(buckets), int(bucket),
                                             out, c, cap, C.byref(n), _stream(stream))
        return L.nqs_pt2_unique(problem.handle, _ptr(dets), _ptr(psi), dets.shape[0],
                                int(buckets), int(bucket), out, c, cap, C.byref(n),
                                _stream(stream))

    st = call(None, None, 0)
    if st != NQS_ERR_ARG or n.value == 0:
        _check(st, "nqs_pt2_unique")
    cap = max(n.value, 1)
    out = torch.empty((cap, 2), dtype=torch.int64, device=dets.device)
    c = torch.empty(cap, dtype=torch.float64, device=dets.device)
    _check(call(_ptr(out), _ptr(c), cap), "nqs_pt2_unique")
    return out[:n.value].view(torch.uint64), c[:n.value]


def hb_select(problem: Problem, dets: torch.Tensor, psi: torch.Tensor, eps: float,
              o: Opts | None = None, stream=None):
    """Heat-bath screened perturbative set (Eq. hb_screen). Returns dict(dets uint64 [n, 2]
    ascending, coupling float64 [n] = max_x |H_x'x psi_x|, n_emitted, n_examined); the library's
    buffers are copied into torch tensors on the same stream and freed."""
    dets = _dets(dets)
    psi = psi.contiguous()
    st = DetSetStruct()
    _check(lib().nqs_hb_select(problem.handle, _ptr(dets), _ptr(psi), dets.shape[0], float(eps),
                               C.byref(o) if o else None, C.byref(st), _stream(stream)),
           "nqs_hb_select")
    out_d, out_c, _ = _take_detset(st, dets.device)
    return dict(dets=out_d, coupling=out_c, n_emitted=st.n_emitted, n_examined=st.n_examined)


SELECT_TOPK, SELECT_MASS, SELECT_THRESHOLD = 0, 1, 2


def _take_detset(st: DetSetStruct, device, with_index=False):
    """Copy a library-owned set into torch tensors and free it."""
    try:
        n = st.n
        d = torch.empty((n, 2), dtype=torch.uint64, device=device)
        v = torch.empty(n, dtype=torch.float64, device=device)
        ix = torch.empty(n, dtype=torch.int64, device=device) if with_index else None
        cudart = _cudart()
        for dst, src, nb in ((d, st.dets, 16 * n), (v, st.value, 8 * n),
                             (ix, st.index, 8 * n)):
            if dst is not None and nb and cudart.cudaMemcpy(
                    C.c_void_p(dst.data_ptr()), C.c_void_p(src), C.c_size_t(nb), 3) != 0:
                raise NQSError("cudaMemcpy failed")
    finally:
        lib().nqs_detset_free(C.byref(st))
    return d, v, ix


def select(problem: Problem, T: torch.Tensor, logabs: torch.Tensor, mode: int, K: int = 0,
           param: float = 0.0, o: Opts | None = None, stream=None):
    """Outer-loop selector (Sec. 2.4.2). Returns dict(dets uint64 [c, 2] ascending by key,
    logabs [c], index [c] = positions in T)."""
    T = _dets(T)
    logabs = logabs.contiguous()
    st = DetSetStruct()
    _check(lib().nqs_select(problem.handle, _ptr(T), _ptr(logabs), T.shape[0], int(mode), int(K),
                            float(param), C.byref(o) if o else None, C.byref(st),
                            _stream(stream)), "nqs_select")
    d, v, ix = _take_detset(st, T.device, with_index=True)
    return dict(dets=d, logabs=v, index=ix)


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """C = A B^T on the tcgen05 tensor-core kernel (A [M][K], B [N][K] bfloat16, C float)."""
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C_ = torch.empty(M, N, dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().nqs_gemm_bf16(_ptr(A), K, _ptr(B), K, M, N, K, _ptr(C_), N, _ptr(err),
                               _stream(stream)), "nqs_gemm_bf16")
    if int(err.item()) != 0:
        raise NQSError("nqs_gemm_bf16: a pipeline wait timed out")
    return C_


def gemm_bf16_ex(A: torch.Tensor, a_mn: bool, B: torch.Tensor, b_mn: bool, M=None, N=None,
                 stream=None) -> torch.Tensor:
    """C = A' B'^T with A' = A^T if a_mn else A (A [K][lda] or [M][K]) and B' = B^T if b_mn
    else B (B [K][ldb] or [N][K]), bfloat16 in, float out (nqs_gemm_bf16_ex). M (N) may be
    given below the row length of an MN-major A (B): the trailing columns are not read."""
    A, B = A.contiguous(), B.contiguous()
    K = A.shape[0] if a_mn else A.shape[1]
    if M is None:
        M = A.shape[1] if a_mn else A.shape[0]
    if N is None:
        N = B.shape[1] if b_mn else B.shape[0]
    C_ = torch.empty(M, N, dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().nqs_gemm_bf16_ex(_ptr(A), A.shape[1], 1 if a_mn else 0, _ptr(B), B.shape[1],
                                  1 if b_mn else 0, M, N, K, _ptr(C_), N, _ptr(err),
                                  _stream(stream)), "nqs_gemm_bf16_ex")
    if int(err.item()) != 0:
        raise NQSError("nqs_gemm_bf16_ex: a pipeline wait timed out")
    return C_


BATCH_STREAMS, BATCH_GROUPED = 0, 1


class Batch:
    """nqs_batch: many independent E_S + gradient evaluations, either one launch per pipeline
    stage over all problems (BATCH_GROUPED, the default when the batch qualifies) or the
    problems' own pipelines on side streams (BATCH_STREAMS), optionally recorded as one CUDA
    graph. items: list of (problem, net, csr, dets, out[4], grad) tuples."""

    def __init__(self, items, nstreams: int = 16, mode: int | None = None):
        self.items = items  # keeps every referenced object alive
        n = len(items)
        P = (C.c_void_p * n)(*[it[0].handle.value for it in items])
        Nt = (C.c_void_p * n)(*[it[1].handle.value for it in items])
        csrs = (CSRStruct * n)(*[it[2].s for it in items])
        D = (C.c_void_p * n)(*[it[3].data_ptr() for it in items])
        nS = (C.c_int64 * n)(*[it[3].shape[0] for it in items])
        O = (C.c_void_p * n)(*[it[4].data_ptr() for it in items])
        G = (C.c_void_p * n)(*[(it[5].data_ptr() if it[5] is not None else 0) for it in items])
        h = C.c_void_p()
        _check(lib().nqs_batch_create(n, P, Nt, csrs, D, nS, O, G, nstreams, C.byref(h)),
               "nqs_batch_create")
        self.handle = h
        if mode is not None:
            self.set_mode(mode)

    def set_mode(self, mode: int):
        _check(lib().nqs_batch_set_mode(self.handle, int(mode)), "nqs_batch_set_mode")

    @property
    def mode(self) -> int:
        return lib().nqs_batch_get_mode(self.handle)

    def run(self, stream=None):
        _check(lib().nqs_batch_run(self.handle, _stream(stream)), "nqs_batch_run")

    def capture(self, stream):
        _check(lib().nqs_batch_capture(self.handle, _stream(stream)), "nqs_batch_capture")

    def launch(self, stream):
        _check(lib().nqs_batch_launch(self.handle, _stream(stream)), "nqs_batch_launch")

    def close(self):
        if getattr(self, "handle", None):
            lib().nqs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_autotune(on: bool):
    lib().nqs_set_autotune(1 if on else 0)


def set_gemm_pairing(on: bool):
    """Paired (two-SM, cta_group::2) tensor-core GEMMs for 256-column tiles on or off."""
    lib().nqs_set_gemm_pairing(1 if on else 0)


def autotune_entries():
    n = lib().nqs_autotune_entries(None, None, None, None, 0)
    arrs = [(C.c_int * max(n, 1))() for _ in range(4)]
    lib().nqs_autotune_entries(*arrs, n)
    return [(arrs[0][i], arrs[1][i], arrs[2][i], arrs[3][i]) for i in range(n)]


def wait_probe(problem: Problem, limit_cycles: int, stream=None) -> int:
    """Status of a bounded device wait on a barrier nothing completes (NQS_ERR_TIMEOUT when the
    timeout path works)."""
    return lib().nqs_wait_probe(problem.handle, int(limit_cycles), _stream(stream))


def set_scratch_limit(problem: Problem, nbytes: int):
    _check(lib().nqs_set_scratch_limit(problem.handle, int(nbytes)), "nqs_set_scratch_limit")


def pool_usage(problem: Problem):
    """(bytes in use, bytes reserved) of the problem's scratch pool."""
    u, r = C.c_int64(0), C.c_int64(0)
    _check(lib().nqs_pool_usage(problem.handle, C.byref(u), C.byref(r)), "nqs_pool_usage")
    return u.value, r.value


def profile_enable(on: bool = True):
    lib().nqs_profile_enable(1 if on else 0)


def profile_reset():
    lib().nqs_profile_reset()


def profile_read() -> dict:
    """{kernel family: (total ms, launches)} for the instrumented launches since the reset."""
    out = {}
    for name in PROFILED:
        ms = C.c_double(0)
        n = C.c_int64(0)
        _check(lib().nqs_profile_read(name.encode(), C.byref(ms), C.byref(n)), "nqs_profile_read")
        out[name] = (ms.value, n.value)
    return out


def launch_count() -> int:
    return lib().nqs_launch_count()


class EnergyFunction(torch.autograd.Function):
    """E_S as a differentiable function of the six trainable parameter tensors; the backward
    returns the gradient computed by the hand-written adjoint in nqs_energy_grad."""

    @staticmethod
    def forward(ctx, problem, net, csr, dets, *params):
        out, grad, _ = energy_grad(problem, net, csr, dets, with_grad=True)
        ctx.net = net
        ctx.save_for_backward(grad)
        return out[0].clone()

    @staticmethod
    def backward(ctx, gE):
        (grad,) = ctx.saved_tensors
        parts = ctx.net.split(grad)
        grads = [(g * gE).to(p.dtype) for g, p in zip(parts, ctx.net.params[:6])]
        return (None, None, None, None, *grads)


def energy(problem: Problem, net: Net, csr: CSR, dets: torch.Tensor) -> torch.Tensor:
    """Differentiable E_S (autograd through the adjoint kernel)."""
    return EnergyFunction.apply(problem, net, csr, dets, *net.params[:6])
