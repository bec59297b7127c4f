"""Python binding of the pipelined-PCG CUDA library (include/ppcg.h).

Argument marshalling only: every step of a solve runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the compiled
library (libppcg.so, built for sm_103a by ``build.py``) is missing or cannot be loaded,
every entry point raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "Opts", "Info", "Solver", "batch_solve", "Server", "status_name",
    "OK", "PENDING", "ERR_ARG", "ERR_NOT_SPD", "ERR_BREAKDOWN", "ERR_NOT_CONVERGED",
    "ERR_NONFINITE", "ERR_OOM", "ERR_CUDA", "ERR_TIMEOUT", "ERR_BUSY", "ERR_UNKNOWN_TICKET",
    "FP64", "FP32_IR", "FP32_RU", "NORM_REL_R", "NORM_PAPER_U_ABS", "PATH_AUTO", "PATH_GRID", "PATH_CLUSTER", "PATH_ONCHIP",
    "FMT_AUTO", "FMT_CSR", "FMT_SELL", "FMT_BOX", "VARIANT_ALG2", "VARIANT_JACOBI_SCALED", "EXPORTED_SYMBOLS",
]

OK, PENDING, ERR_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NOT_CONVERGED = 0, 1, -1, -2, -3, -4
ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_UNKNOWN_TICKET = -5, -6, -7, -8, -9, -10
FP64, FP32_IR, FP32_RU = 0, 1, 2
FMT_AUTO, FMT_CSR, FMT_SELL, FMT_BOX = 0, 1, 2, 3
NORM_REL_R, NORM_PAPER_U_ABS = 0, 1
PATH_AUTO, PATH_GRID, PATH_CLUSTER, PATH_ONCHIP = 0, 1, 2, 3
VARIANT_ALG2, VARIANT_JACOBI_SCALED = 0, 1
COLS_SELL, COLS_DICT, COLS_PATTERN, COLS_MATRIX_FREE = 0, 1, 2, 3

_NAMES = {OK: "OK", PENDING: "PENDING", ERR_ARG: "ERR_ARG", ERR_NOT_SPD: "ERR_NOT_SPD",
          ERR_BREAKDOWN: "ERR_BREAKDOWN", ERR_NOT_CONVERGED: "ERR_NOT_CONVERGED",
          ERR_NONFINITE: "ERR_NONFINITE", ERR_OOM: "ERR_OOM", ERR_CUDA: "ERR_CUDA",
          ERR_TIMEOUT: "ERR_TIMEOUT", ERR_BUSY: "ERR_BUSY", ERR_UNKNOWN_TICKET: "ERR_UNKNOWN_TICKET"}

# Every symbol include/ppcg.h declares.
EXPORTED_SYMBOLS = (
    "ppcg_opts_default", "ppcg_create", "ppcg_solve", "ppcg_last_info", "ppcg_batch_solve", "ppcg_destroy",
    "ppcg_server_create", "ppcg_submit", "ppcg_poll", "ppcg_server_stats", "ppcg_server_destroy",
    "ppcg_last_error", "ppcg_selftest_barrier_timeout", "ppcg_solve_noalloc", "ppcg_plan_info",
)


def status_name(s):
    return _NAMES.get(int(s), str(s))


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("format", ctypes.c_int32), ("norm", ctypes.c_int32),
                ("path", ctypes.c_int32), ("sigma", ctypes.c_int32), ("rr_period", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("inner_maxit", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("spin_limit_ns", ctypes.c_int64),
                ("cluster_max_rows", ctypes.c_int32), ("epoch_iters", ctypes.c_int32),
                ("max_restarts", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("gap_theta", ctypes.c_double), ("gap_fall", ctypes.c_int32),
                ("cluster_ctas", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("columns", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("pattern_k", ctypes.c_int32), ("dict_size", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("slots", ctypes.c_int64), ("padding", ctypes.c_double), ("convert_seconds", ctypes.c_double),
                ("create_seconds", ctypes.c_double), ("bytes_per_iter", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("rr_count", ctypes.c_int32), ("rel_res_recursive", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("seconds", ctypes.c_double),
                ("bytes_per_iter", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("fp64_fallback", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def __repr__(self):
        return f"Info({status_name(self.status)}, " + ", ".join(
            f"{k}={getattr(self, k)}" for k, _ in self._fields_[1:]) + ")"


_lib = None
P = ctypes.c_void_p


def lib(build_if_missing=True):
    """Load libppcg.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"pipelined-PCG CUDA library not found at {_build.LIB}; run build.py")
    L = ctypes.CDLL(_build.LIB)
    L.ppcg_opts_default.argtypes = [ctypes.POINTER(Opts)]
    L.ppcg_opts_default.restype = None
    L.ppcg_create.argtypes = [ctypes.POINTER(P), ctypes.c_int64, ctypes.c_int64, P, P, P,
                              ctypes.POINTER(Opts), P]
    L.ppcg_create.restype = ctypes.c_int
    L.ppcg_solve.argtypes = [P, P, P, P, ctypes.c_double, ctypes.c_int32, P, ctypes.POINTER(Info)]
    L.ppcg_solve.restype = ctypes.c_int
    L.ppcg_last_info.argtypes = [P, ctypes.POINTER(Info)]
    L.ppcg_last_info.restype = ctypes.c_int
    L.ppcg_batch_solve.argtypes = [ctypes.c_int32, P, P, P, P, P, P, P, P]
    L.ppcg_batch_solve.restype = ctypes.c_int
    L.ppcg_destroy.argtypes = [P]
    L.ppcg_destroy.restype = None
    L.ppcg_last_error.argtypes = []
    L.ppcg_last_error.restype = ctypes.c_char_p
    L.ppcg_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_size_t, ctypes.POINTER(Opts)]
    L.ppcg_server_create.restype = ctypes.c_int
    L.ppcg_submit.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, ctypes.c_double,
                              ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
    L.ppcg_submit.restype = ctypes.c_int
    L.ppcg_poll.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(Info)]
    L.ppcg_poll.restype = ctypes.c_int
    L.ppcg_server_stats.argtypes = [P] + [ctypes.POINTER(ctypes.c_int64)] * 4
    L.ppcg_server_stats.restype = ctypes.c_int
    L.ppcg_server_destroy.argtypes = [P]
    L.ppcg_server_destroy.restype = None
    L.ppcg_selftest_barrier_timeout.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_int32)]
    L.ppcg_selftest_barrier_timeout.restype = ctypes.c_int
    L.ppcg_solve_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P, ctypes.c_double,
                                     ctypes.c_int32, P, ctypes.POINTER(Info)]
    L.ppcg_solve_noalloc.restype = ctypes.c_int
    L.ppcg_plan_info.argtypes = [P, ctypes.POINTER(Plan)]
    L.ppcg_plan_info.restype = ctypes.c_int
    _lib = L
    return L


def last_error():
    return lib().ppcg_last_error().decode(errors="replace")


class PPCGError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {status_name(status)} ({last_error()})")
        self.status = status


def default_opts(**kw):
    o = Opts()
    lib().ppcg_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a):
    """Raw pointer of a torch tensor (host or device) or a numpy array (host)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


class Solver:
    """One SPD matrix on the GPU (ppcg_create) and its solves (ppcg_solve).

    row_ptr (int64), col (int32), val (float64): numpy arrays or torch tensors, host or
    device; copied at creation."""

    def __init__(self, n, row_ptr, col, val, opts=None, stream=None, **kw):
        import torch  # noqa: F401  (CUDA context through torch)
        self._keep = (row_ptr, col, val)
        self.n = int(n)
        self.nnz = int(len(col))
        o = opts if opts is not None else default_opts(**kw)
        h = P()
        st = lib().ppcg_create(ctypes.byref(h), self.n, self.nnz, _ptr(row_ptr), _ptr(col), _ptr(val),
                               ctypes.byref(o), _stream_ptr(stream))
        if st != OK:
            raise PPCGError(st, "ppcg_create")
        self.handle = h
        self.opts = o
        self._keep = None

    @classmethod
    def from_csr(cls, a, **kw):
        return cls(a.n, np.ascontiguousarray(a.row_ptr, dtype=np.int64),
                   np.ascontiguousarray(a.col, dtype=np.int32),
                   np.ascontiguousarray(a.val, dtype=np.float64), **kw)

    def solve(self, b, x0=None, x=None, tol=1e-8, maxit=10000, stream=None, sync=True, host_fn_info=None):
        """Enqueue a solve.  b/x0/x: torch tensors (device or host) or numpy arrays.
        Returns (x, info); info is valid once the stream is synchronised (sync=True does it).
        host_fn_info (default: not sync) passes info to ppcg_solve, which fills it from a
        host function on the stream; otherwise info is NULL there, and with sync=True the
        record is read after the synchronisation (ppcg_last_info), with sync=False info is
        None and last_info() reads it after the caller's synchronisation."""
        import torch
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device if hasattr(b, "device") else "cuda")
        if host_fn_info is None:
            host_fn_info = not sync
        info = Info() if host_fn_info else None
        s = _stream_ptr(stream)
        st = lib().ppcg_solve(self.handle, _ptr(b), _ptr(x0), _ptr(x), float(tol), int(maxit), s,
                              ctypes.byref(info) if host_fn_info else None)
        if st != OK:
            raise PPCGError(st, "ppcg_solve")
        if sync:
            torch.cuda.synchronize()
            if not host_fn_info:
                info = self.last_info()
        self._last_info = info
        return x, info

    def plan(self):
        """ppcg_plan_info: the plan ppcg_create chose (path, column mode, sigma, padding,
        conversion and create times)."""
        p = Plan()
        st = lib().ppcg_plan_info(self.handle, ctypes.byref(p))
        if st != OK:
            raise PPCGError(st, "ppcg_plan_info")
        return p

    def last_info(self):
        """ppcg_last_info: the record of this handle's latest solve (after a stream sync)."""
        info = Info()
        st = lib().ppcg_last_info(self.handle, ctypes.byref(info))
        if st != OK:
            raise PPCGError(st, "ppcg_last_info")
        return info

    def close(self):
        if getattr(self, "handle", None):
            lib().ppcg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(solvers, bs, xs, x0s=None, tol=1e-8, maxit=10000, stream=None, sync=True):
    """ppcg_batch_solve over Solver objects with device tensors.  Returns the Info list."""
    import torch
    m = len(solvers)
    H = (P * m)(*[s.handle for s in solvers])
    B = (P * m)(*[_ptr(b) for b in bs])
    X = (P * m)(*[_ptr(x) for x in xs])
    X0 = (P * m)(*[_ptr(x) for x in x0s]) if x0s is not None else None
    tols = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)))
    its = np.ascontiguousarray(np.broadcast_to(np.asarray(maxit, dtype=np.int32), (m,)))
    infos = (Info * m)()
    st = lib().ppcg_batch_solve(m, ctypes.cast(H, P), ctypes.cast(B, P),
                                ctypes.cast(X0, P) if X0 is not None else None, ctypes.cast(X, P),
                                tols.ctypes.data, its.ctypes.data, _stream_ptr(stream),
                                ctypes.cast(infos, P))
    if st != OK:
        raise PPCGError(st, "ppcg_batch_solve")
    if sync:
        torch.cuda.synchronize()
    return list(infos)


class Server:
    """Continuous-batching server (ppcg_server_*)."""

    def __init__(self, hbm_budget=0, opts=None, **kw):
        import torch  # noqa: F401
        o = opts if opts is not None else default_opts(**kw)
        h = P()
        st = lib().ppcg_server_create(ctypes.byref(h), int(hbm_budget), ctypes.byref(o))
        if st != OK:
            raise PPCGError(st, "ppcg_server_create")
        self.handle = h

    def submit(self, a, b, x0=None, tol=1e-8, maxit=10000):
        rp = np.ascontiguousarray(a.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(a.col, dtype=np.int32)
        v = np.ascontiguousarray(a.val, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        t = ctypes.c_uint64()
        st = lib().ppcg_submit(self.handle, a.n, len(ci), rp.ctypes.data, ci.ctypes.data, v.ctypes.data,
                               b.ctypes.data, None if x0 is None else x0.ctypes.data, float(tol),
                               int(maxit), ctypes.byref(t))
        if st != OK:
            raise PPCGError(st, "ppcg_submit")
        return t.value

    def poll(self, ticket, n):
        """Returns (status, x or None, Info)."""
        x = np.empty(n)
        info = Info()
        st = lib().ppcg_poll(self.handle, ticket, x.ctypes.data, ctypes.byref(info))
        if st == PENDING:
            return st, None, None
        return st, x, info

    def stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        st = lib().ppcg_server_stats(self.handle, *[ctypes.byref(t) for t in v])
        if st != OK:
            raise PPCGError(st, "ppcg_server_stats")
        return dict(zip(("completed", "running", "queued", "hbm_in_use"), [t.value for t in v]))

    def close(self):
        if getattr(self, "handle", None):
            lib().ppcg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def barrier_timeout_selftest(grid=64, drop_rank=3, limit_ns=50_000_000):
    """Runs the grid barrier with one CTA that never arrives; returns (status, n_timed_out)."""
    out = ctypes.c_int32()
    st = lib().ppcg_selftest_barrier_timeout(grid, drop_rank, limit_ns, ctypes.byref(out))
    return st, out.value
