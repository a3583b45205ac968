"""Thin ctypes binding of ``libbpjd.so`` (include/bpjd.h): argument marshalling only.

Every numerical step runs inside the CUDA library.  Host arrays are NumPy
arrays; device arrays are ``torch`` CUDA tensors (PyTorch is used only for
device memory and streams).  If the library has not been built the import of
this module raises: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbpjd.so")

# ---- status codes and options (mirrors include/bpjd.h) ----------------------
OK = 0
ERR_BAD_ARG = -1
ERR_CSR_INVALID = -2
ERR_MAP_INVALID = -3
ERR_K_TOO_LARGE = -4
ERR_GAP = -5
ERR_LOCAL_INDEFINITE = -6
ERR_BREAKDOWN = -7
ERR_NOCONV = -8
ERR_OOM = -9
ERR_CUDA = -10
ERR_UNSUPPORTED = -11
ERR_TOO_LARGE = -12
ERR_TIMEOUT = -13

FP64, MIXED, MIXED_LOCAL = 0, 1, 2
ADMIT_SMALLEST, ADMIT_FIFO = 0, 1
W_2K, W_3K = 0, 1
STOP_RESIDUAL, STOP_DLAMBDA = 0, 1

EXPORTED = [
    "bpjd_default_opts", "bpjd_status_string", "bpjd_setup", "bpjd_solve", "bpjd_free", "bpjd_dims",
    "bpjd_spmm", "bpjd_apply_preconditioner", "bpjd_history", "bpjd_device_bytes",
    "bpjd_problem_create", "bpjd_problem_free", "bpjd_profile", "bpjd_profile_read",
    "bpjd_layout", "bpjd_block_gram", "bpjd_block_gram_noalloc",
    "bpjd_server_default_opts", "bpjd_server_create", "bpjd_server_submit", "bpjd_server_poll",
    "bpjd_server_free", "bpjd_set_wait_limit",
]
PENDING = 1
PROF_NAMES = ["local", "coarse", "prolong", "spmm", "inner", "combine", "rr", "resid"]


class Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class Partition(C.Structure):
    _fields_ = [("n_sub", C.c_int32), ("sub_ptr", C.c_void_p), ("sub_dofs", C.c_void_p),
                ("sub_color", C.c_void_p), ("n_colors", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("k", C.c_int32), ("precision", C.c_int32), ("subspace", C.c_int32), ("stop_rule", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int32), ("drop_tol", C.c_double), ("H", C.c_double),
                ("delta", C.c_double), ("inputs_on_device", C.c_int32), ("stream", C.c_void_p),
                ("local_scratch_bytes", C.c_size_t), ("local_refactor_tol", C.c_double),
                ("host_loop", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("max_rel_resid", C.c_double),
                ("sum_abs_dlambda", C.c_double), ("t_setup_s", C.c_double), ("t_solve_s", C.c_double),
                ("status", C.c_int32)]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("workers", C.c_int32), ("precision", C.c_int32),
                ("subspace", C.c_int32), ("stop_rule", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("admission", C.c_int32), ("starvation_s", C.c_double), ("host_loop", C.c_int32),
                ("batch_local", C.c_int32), ("batch_wait_us", C.c_int32)]


class MeshS(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32 * 3), ("length", C.c_double * 3), ("nsub", C.c_int32 * 3),
                ("delta", C.c_int32), ("tau", C.c_int32), ("kappa", C.c_void_p), ("partition", C.c_int32)]


class ProblemS(C.Structure):
    _fields_ = [("K", Csr), ("M", Csr), ("P", Csr), ("P0", Csr), ("part", Partition)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2203_06327_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    lib.bpjd_default_opts.argtypes = [C.POINTER(Opts)]
    lib.bpjd_status_string.restype = C.c_char_p
    lib.bpjd_status_string.argtypes = [C.c_int]
    lib.bpjd_setup.argtypes = [C.POINTER(Csr), C.POINTER(Csr), C.POINTER(Csr), C.POINTER(Csr),
                               C.POINTER(Partition), C.POINTER(Opts), C.POINTER(C.c_void_p)]
    lib.bpjd_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(Stats)]
    lib.bpjd_free.argtypes = [C.c_void_p]
    lib.bpjd_free.restype = None
    lib.bpjd_dims.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.bpjd_spmm.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    lib.bpjd_apply_preconditioner.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.bpjd_history.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    lib.bpjd_device_bytes.argtypes = [C.c_void_p]
    lib.bpjd_device_bytes.restype = C.c_size_t
    lib.bpjd_problem_create.argtypes = [C.POINTER(MeshS), C.POINTER(C.POINTER(ProblemS))]
    lib.bpjd_problem_free.argtypes = [C.POINTER(ProblemS)]
    lib.bpjd_problem_free.restype = None
    lib.bpjd_layout.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.bpjd_block_gram.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]
    lib.bpjd_server_default_opts.argtypes = [C.POINTER(ServerOpts)]
    lib.bpjd_server_default_opts.restype = None
    lib.bpjd_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]
    lib.bpjd_server_submit.argtypes = [C.c_void_p, C.POINTER(Csr), C.POINTER(Csr), C.POINTER(Csr), C.POINTER(Csr),
                                       C.POINTER(Partition), C.c_int32, C.POINTER(C.c_uint64)]
    lib.bpjd_server_poll.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(Stats),
                                     C.c_void_p]
    lib.bpjd_server_free.argtypes = [C.c_void_p]
    lib.bpjd_server_free.restype = None
    lib.bpjd_server_batch_stats.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.bpjd_set_wait_limit.argtypes = [C.c_void_p, C.c_int32]
    lib.bpjd_profile.argtypes = [C.c_void_p, C.c_int32]
    lib.bpjd_profile_read.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return lib


lib = _load()


class BpjdError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {lib.bpjd_status_string(code).decode()} ({code})")


def _check(code: int, where: str):
    if code != OK:
        raise BpjdError(code, where)


# ---- arrays -----------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data


def _to_device(a, device):
    import torch
    if _is_torch(a):
        return a.to(device).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a)).to(device).contiguous()


@dataclass
class CsrArrays:
    """0-based CSR with int64 row pointers, int32 columns, float64 values (NumPy or torch CUDA)."""
    n_rows: int
    n_cols: int
    row_ptr: object
    col_idx: object
    val: object

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def c(self) -> Csr:
        return Csr(self.n_rows, self.n_cols, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(self.val))

    @staticmethod
    def from_scipy(A) -> "CsrArrays":
        A = A.tocsr()
        A.sort_indices()
        return CsrArrays(A.shape[0], A.shape[1], np.ascontiguousarray(A.indptr, np.int64),
                         np.ascontiguousarray(A.indices, np.int32), np.ascontiguousarray(A.data, np.float64))

    def to(self, device) -> "CsrArrays":
        f = lambda a: _to_device(a, device)
        return CsrArrays(self.n_rows, self.n_cols, f(self.row_ptr), f(self.col_idx), f(self.val))


@dataclass
class PartitionArrays:
    sub_ptr: object      # int64 [n_sub + 1]
    sub_dofs: object     # int32
    sub_color: object    # int32 [n_sub] or None
    n_colors: int = 0

    @property
    def n_sub(self) -> int:
        return int(self.sub_ptr.shape[0]) - 1

    def c(self) -> Partition:
        return Partition(self.n_sub, _ptr(self.sub_ptr), _ptr(self.sub_dofs), _ptr(self.sub_color), self.n_colors)

    def to(self, device) -> "PartitionArrays":
        f = lambda a: None if a is None else _to_device(a, device)
        return PartitionArrays(f(self.sub_ptr), f(self.sub_dofs), f(self.sub_color), self.n_colors)


# ---- problem generation -----------------------------------------------------
_KINDS = {"p1_2d": 0, "p1_3d": 1, "q1_3d": 2, "morley_2d": 3, "bfs_2d": 4, "p1_lshape": 5, "q1_lshape": 6}


@dataclass
class Problem:
    """Host arrays of an assembled model problem (copied out of the library)."""
    K: CsrArrays
    M: CsrArrays
    P: CsrArrays
    P0: CsrArrays
    part: PartitionArrays
    tau: int


def _copy_csr(c: Csr) -> CsrArrays:
    n1 = c.n_rows + 1
    rp = np.ctypeslib.as_array(C.cast(c.row_ptr, C.POINTER(C.c_int64)), shape=(n1,)).copy()
    nnz = int(c.nnz)
    ci = np.ctypeslib.as_array(C.cast(c.col_idx, C.POINTER(C.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
    v = np.ctypeslib.as_array(C.cast(c.val, C.POINTER(C.c_double)), shape=(max(nnz, 1),))[:nnz].copy()
    return CsrArrays(c.n_rows, c.n_cols, rp, ci, v)


_PARTITIONS = {"boxes": 0, "triangles": 1}


def problem_create(kind: str, n, length, nsub, delta: int, tau: int = 0, kappa: Optional[np.ndarray] = None,
                   partition: str = "boxes") -> Problem:
    m = MeshS()
    m.kind = _KINDS[kind]
    for d in range(3):
        m.n[d] = int(n[d]) if d < len(n) else 1
        m.length[d] = float(length[d]) if d < len(length) else 1.0
        m.nsub[d] = int(nsub[d]) if d < len(nsub) else 1
    m.delta = int(delta)
    m.tau = int(tau)
    m.partition = _PARTITIONS[partition]
    kap = None
    if kappa is not None:
        kap = np.ascontiguousarray(kappa, dtype=np.float64)
        m.kappa = kap.ctypes.data
    out = C.POINTER(ProblemS)()
    _check(lib.bpjd_problem_create(C.byref(m), C.byref(out)), "bpjd_problem_create")
    try:
        p = out.contents
        part = p.part
        ns = part.n_sub
        sp = np.ctypeslib.as_array(C.cast(part.sub_ptr, C.POINTER(C.c_int64)), shape=(ns + 1,)).copy()
        sd = np.ctypeslib.as_array(C.cast(part.sub_dofs, C.POINTER(C.c_int32)), shape=(int(sp[-1]),)).copy()
        sc = np.ctypeslib.as_array(C.cast(part.sub_color, C.POINTER(C.c_int32)), shape=(ns,)).copy()
        res = Problem(_copy_csr(p.K), _copy_csr(p.M), _copy_csr(p.P), _copy_csr(p.P0),
                      PartitionArrays(sp, sd, sc, part.n_colors), int(tau))
    finally:
        lib.bpjd_problem_free(out)
    return res


def problem_from_spec(spec) -> Problem:
    """Builds the library's own problem arrays for a ``workloads.ProblemSpec``."""
    return problem_create(spec.kind, spec.n, spec.length, spec.nsub, spec.delta, spec.tau, spec.kappa,
                          getattr(spec, "partition", "boxes"))


# ---- solver -------------------------------------------------------------------
class Solver:
    """Owns a bpjd_handle.  Inputs may be host (NumPy) or device (torch CUDA) arrays."""

    def __init__(self, K: CsrArrays, M: CsrArrays, P: CsrArrays, P0: Optional[CsrArrays], part: PartitionArrays,
                 k: int, precision: int = FP64, subspace: int = W_2K, stop_rule: int = STOP_RESIDUAL,
                 tol: float = 1e-8, max_iter: int = 500, drop_tol: float = 1e-10, stream=None,
                 local_scratch_bytes: int = 0, local_refactor_tol: float = 0.0, host_loop: bool = False):
        o = Opts()
        lib.bpjd_default_opts(C.byref(o))
        o.k, o.precision, o.subspace, o.stop_rule = k, precision, subspace, stop_rule
        o.local_scratch_bytes = int(local_scratch_bytes)
        o.local_refactor_tol = float(local_refactor_tol)
        o.host_loop = 1 if host_loop else 0
        o.tol, o.max_iter, o.drop_tol = tol, max_iter, drop_tol
        o.inputs_on_device = 1 if _is_torch(K.val) and K.val.is_cuda else 0
        o.stream = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        self.k = k
        self.max_iter = max_iter
        self._stream = stream
        h = C.c_void_p()
        a, m, p = K.c(), M.c(), P.c()
        p0 = P0.c() if P0 is not None else None
        pt = part.c()
        rc = lib.bpjd_setup(C.byref(a), C.byref(m), C.byref(p), C.byref(p0) if p0 is not None else None,
                            C.byref(pt), C.byref(o), C.byref(h))
        _check(rc, "bpjd_setup")
        self._h = h
        n, nh, kk = C.c_int32(), C.c_int32(), C.c_int32()
        lib.bpjd_dims(h, C.byref(n), C.byref(nh), C.byref(kk))
        self.n, self.n_coarse = n.value, nh.value

    @classmethod
    def from_problem(cls, pb: Problem, k: int, device=None, **kw) -> "Solver":
        if device is not None:
            return cls(pb.K.to(device), pb.M.to(device), pb.P.to(device),
                       pb.P0.to(device) if pb.tau > 0 else None, pb.part.to(device), k, **kw)
        return cls(pb.K, pb.M, pb.P, pb.P0 if pb.tau > 0 else None, pb.part, k, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib.bpjd_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, eigvecs: str = "host", out=None, raise_on_noconv: bool = True):
        """Returns (eigenvalues, eigenvectors or None, stats dict).  eigvecs: "host" | "device" | None;
        out: the n x k float64 array (host) or CUDA tensor (device) that receives them."""
        lam = np.empty(self.k, dtype=np.float64)
        X = None
        on_dev = 0
        if eigvecs == "host":
            X = out if out is not None else np.empty((self.n, self.k), dtype=np.float64)
        elif eigvecs == "device":
            import torch
            X = out if out is not None else torch.empty((self.n, self.k), dtype=torch.float64, device="cuda")
            on_dev = 1
        st = Stats()
        rc = lib.bpjd_solve(self._h, lam.ctypes.data, _ptr(X), on_dev, C.byref(st))
        if rc != OK and not (rc == ERR_NOCONV and not raise_on_noconv):
            raise BpjdError(rc, "bpjd_solve")
        stats = {f: getattr(st, f) for f, _ in Stats._fields_}
        return lam, X, stats

    def spmm(self, X, YA, YM):
        _check(lib.bpjd_spmm(self._h, _ptr(X), _ptr(YA), _ptr(YM), int(X.shape[1])), "bpjd_spmm")

    def apply_preconditioner(self, rho, lam, Z):
        _check(lib.bpjd_apply_preconditioner(self._h, _ptr(rho), _ptr(lam), _ptr(Z)), "bpjd_apply_preconditioner")

    def block_gram(self, U, V, out, symmetric: bool = False):
        """out = [U_0..]^T [V_0..] (double-word arithmetic); U, V lists of n x k CUDA tensors."""
        pu = (C.c_void_p * len(U))(*[_ptr(u) for u in U])
        pv = (C.c_void_p * len(V))(*[_ptr(v) for v in V])
        _check(lib.bpjd_block_gram(self._h, len(U), pu, len(V), pv, 1 if symmetric else 0, _ptr(out)),
               "bpjd_block_gram")

    def history(self) -> np.ndarray:
        buf = np.empty((self.max_iter + 1, self.k), dtype=np.float64)
        rows = lib.bpjd_history(self._h, buf.ctypes.data, buf.shape[0])
        if rows < 0:
            raise BpjdError(rows, "bpjd_history")
        return buf[:rows].copy()

    def set_wait_limit(self, attempts: int):
        """Attempts of every bounded device-side wait before a kernel gives up (TIMEOUT)."""
        _check(lib.bpjd_set_wait_limit(self._h, int(attempts)), "bpjd_set_wait_limit")

    def profile(self, enable: bool = True):
        _check(lib.bpjd_profile(self._h, 1 if enable else 0), "bpjd_profile")

    def profile_read(self):
        """{class: (ms, launches)} and the total kernel-launch count since profile()."""
        ms = np.zeros(len(PROF_NAMES))
        cnt = np.zeros(len(PROF_NAMES), dtype=np.int64)
        tot = C.c_int64()
        _check(lib.bpjd_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data, C.byref(tot)), "bpjd_profile_read")
        return {n: (float(ms[i]), int(cnt[i])) for i, n in enumerate(PROF_NAMES)}, int(tot.value)

    def layout(self) -> dict:
        Bw, sn, ns, nz = C.c_int32(), C.c_int64(), C.c_int32(), C.c_int64()
        _check(lib.bpjd_layout(self._h, C.byref(Bw), C.byref(sn), C.byref(ns), C.byref(nz)), "bpjd_layout")
        return {"band_window": Bw.value, "sum_local": sn.value, "n_sub": ns.value, "nnz": nz.value}

    def device_bytes(self) -> int:
        return int(lib.bpjd_device_bytes(self._h))


# ---- serving --------------------------------------------------------------------
class Server:
    """Many independent eigenproblems on one GPU (bpjd_server_*): requests are queued,
    admitted under a device-memory budget (smallest estimated work first with aging, or
    first-in first-out) and solved by worker threads with one CUDA stream each; with
    batch_local the local solves of the requests in flight share grouped launches."""

    def __init__(self, workers: int = 8, hbm_budget_bytes: int = 0, precision: int = MIXED,
                 subspace: int = W_3K, stop_rule: int = STOP_RESIDUAL, tol: float = 1e-8, max_iter: int = 500,
                 admission: int = 0, starvation_s: float = 1.0, host_loop: bool = True,
                 batch_local: bool = True, batch_wait_us: int = 100):
        o = ServerOpts()
        lib.bpjd_server_default_opts(C.byref(o))
        o.workers, o.hbm_budget_bytes = int(workers), int(hbm_budget_bytes)
        o.precision, o.subspace, o.stop_rule = precision, subspace, stop_rule
        o.tol, o.max_iter = float(tol), int(max_iter)
        o.admission, o.starvation_s = int(admission), float(starvation_s)
        o.host_loop = 1 if host_loop else 0
        o.batch_local = 1 if batch_local else 0
        o.batch_wait_us = int(batch_wait_us)
        h = C.c_void_p()
        _check(lib.bpjd_server_create(C.byref(o), C.byref(h)), "bpjd_server_create")
        self._h = h
        self._meta = {}

    def submit(self, pb: "Problem", k: int) -> int:
        """Queues one problem (host arrays; copied before returning) and returns its ticket."""
        K, M, P = pb.K.c(), pb.M.c(), pb.P.c()
        P0 = pb.P0.c() if pb.tau > 0 else None
        part = pb.part.c()
        t = C.c_uint64()
        _check(lib.bpjd_server_submit(self._h, C.byref(K), C.byref(M), C.byref(P),
                                      C.byref(P0) if P0 is not None else None, C.byref(part), int(k),
                                      C.byref(t)), "bpjd_server_submit")
        self._meta[t.value] = (pb.K.n_rows, int(k))
        return t.value

    def poll(self, ticket: int, wait: bool = True):
        """None while pending (wait=False); else (status, eigenvalues, eigenvectors,
        stats dict, (queued s, service s, latency s))."""
        n, k = self._meta[ticket]
        lam = np.empty(k, dtype=np.float64)
        X = np.empty((n, k), dtype=np.float64)
        st = Stats()
        times = np.empty(3, dtype=np.float64)
        rc = lib.bpjd_server_poll(self._h, C.c_uint64(ticket), 1 if wait else 0, lam.ctypes.data, X.ctypes.data,
                                  C.byref(st), times.ctypes.data)
        if rc == PENDING:
            return None
        del self._meta[ticket]
        stats = {f: getattr(st, f) for f, _ in Stats._fields_}
        return rc, lam, X, stats, tuple(float(x) for x in times)

    def batch_stats(self):
        """(shared launch groups so far, preconditioner applications they carried)."""
        a, b = C.c_int64(), C.c_int64()
        _check(lib.bpjd_server_batch_stats(self._h, C.byref(a), C.byref(b)), "bpjd_server_batch_stats")
        return a.value, b.value

    def close(self):
        if self._h:
            lib.bpjd_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
