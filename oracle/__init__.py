"""Oracle for pipelined PCG -- test infrastructure only.

A ctypes wrapper over ``ppcg_oracle.c``: a plain sequential FP64 C restatement of
Algorithm 1 (PCG) and Algorithm 2 (pipelined PCG) of Tiwari & Vadhiyar (arXiv 2105.06176,
Sec. III) with the Jacobi preconditioner of Sec. V-A.  Only ``tests/``, the smoke check
and the CPU-baseline leg of the benchmark use it; the CUDA library never does.

Parity pins (all in ``tests/test_oracle_pins.py``): exact termination against dense
solves on spectra with k distinct eigenvalues, closed-form Poisson eigenpairs, Ritz values
of the Lanczos matrix built from (alpha, beta), the Algorithm 2 invariants checked with an
independent library SpMV, A-orthogonality of search directions, agreement with
Algorithm 1, and rounding-sensitivity calibration between two summation orders.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppcg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

OK, ERR_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_NONFINITE = 0, -1, -2, -3, -4, -5
NORM_REL_R, NORM_PAPER_U_ABS = 0, 1
STATE_NAMES = ("x", "r", "u", "w", "p", "q", "s", "z", "m", "n")


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("rr_count", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("bnorm", ctypes.c_double), ("res_recursive", ctypes.c_double),
                ("res_true", ctypes.c_double), ("gamma", ctypes.c_double),
                ("delta", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def build(force=False, openmp=False):
    """Compile the oracle with gcc (no FMA contraction, no fast-math).  openmp: the same
    source with -fopenmp (row loops over all host cores, bitwise-identical results), used
    only to time the oracle on every core."""
    out = _LIB_OMP if openmp else _LIB
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]
                          + (["-fopenmp"] if openmp else [])
                          + ["-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)
    return out


_libs = {}


def lib(openmp=False):
    if openmp not in _libs:
        _lib = ctypes.CDLL(build(openmp=openmp))
        P = ctypes.c_void_p
        _lib.oracle_threads.argtypes = []
        _lib.oracle_threads.restype = ctypes.c_int
        _lib.oracle_spmv.argtypes = [ctypes.c_int64, P, P, P, P, P]
        _lib.oracle_spmv.restype = None
        _lib.oracle_pipecg.argtypes = [ctypes.c_int64, P, P, P, P, P, P, ctypes.c_double,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                       P, P, P, P, ctypes.POINTER(Result)]
        _lib.oracle_pipecg.restype = ctypes.c_int
        _lib.oracle_pcg.argtypes = [ctypes.c_int64, P, P, P, P, P, P, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    P, P, P, P, ctypes.POINTER(Result)]
        _lib.oracle_pcg.restype = ctypes.c_int
        _libs[openmp] = _lib
    return _libs[openmp]


def threads(openmp=False):
    """Host threads the oracle's row loops use (1 for the plain build)."""
    return lib(openmp).oracle_threads()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr_args(a):
    rp = np.ascontiguousarray(a.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(a.col, dtype=np.int32)
    v = np.ascontiguousarray(a.val, dtype=np.float64)
    return rp, ci, v


def spmv(a, x, openmp=False):
    """y = A x (CSR order; rows over all host cores with openmp)."""
    rp, ci, v = _csr_args(a)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(a.n)
    lib(openmp).oracle_spmv(a.n, _ptr(rp), _ptr(ci), _ptr(v), _ptr(x), _ptr(y))
    return y


GAP_THETA, GAP_FALL = 1e-6, 100.0


def pipecg(a, b, x0=None, tol=1e-8, maxit=10000, norm=NORM_REL_R, rr_period=0, max_restarts=8,
           jacobi_elim=False, sum_mode=0, gap_theta=GAP_THETA, gap_fall=GAP_FALL, history=False,
           state=False, openmp=False):
    """Algorithm 2 (with restart on breakdown, up to max_restarts times).  jacobi_elim: the
    variant with q = M^-1 s and u = M^-1 r in place of their recurrences.  gap_theta > 0:
    measured-gap residual replacement (each time gamma has fallen by gap_fall since the
    residuals were last measured or replaced, replace them if ||(b - A x) - r|| exceeds
    gap_theta ||r||); 0 turns it off.  openmp: the OpenMP build of the same source
    (bitwise-identical results).
    Returns dict(x, result, [alpha, beta, res], [state])."""
    rp, ci, v = _csr_args(a)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    x = np.empty(a.n)
    ah = np.full(maxit, np.nan) if history else None
    bh = np.full(maxit, np.nan) if history else None
    rh = np.full(maxit + 1, np.nan) if history else None
    st = np.empty(10 * a.n) if state else None
    res = Result()
    lib(openmp).oracle_pipecg(a.n, _ptr(rp), _ptr(ci), _ptr(v), _ptr(b), _ptr(x0), _ptr(x), tol,
                        maxit, norm, rr_period, max_restarts, int(bool(jacobi_elim)), sum_mode,
                        float(gap_theta), float(gap_fall), _ptr(ah),
                        _ptr(bh), _ptr(rh),
                        _ptr(st), ctypes.byref(res))
    out = {"x": x, "result": res.as_dict()}
    if history:
        k = res.iters
        out.update(alpha=ah[:k], beta=bh[:k], res=rh[:k + 1])
    if state:
        out["state"] = {nm: st[i * a.n:(i + 1) * a.n] for i, nm in enumerate(STATE_NAMES)}
    return out


def pcg(a, b, x0=None, tol=1e-8, maxit=10000, norm=NORM_REL_R, sum_mode=0, history=False,
        state=False, openmp=False):
    """Algorithm 1.  Returns dict(x, result, [alpha, beta, res], [state: x r u p])."""
    rp, ci, v = _csr_args(a)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    x = np.empty(a.n)
    ah = np.full(maxit, np.nan) if history else None
    bh = np.full(maxit, np.nan) if history else None
    rh = np.full(maxit + 1, np.nan) if history else None
    st = np.empty(4 * a.n) if state else None
    res = Result()
    lib(openmp).oracle_pcg(a.n, _ptr(rp), _ptr(ci), _ptr(v), _ptr(b), _ptr(x0), _ptr(x), tol, maxit,
                     norm, sum_mode, _ptr(ah), _ptr(bh), _ptr(rh), _ptr(st), ctypes.byref(res))
    out = {"x": x, "result": res.as_dict()}
    if history:
        k = res.iters
        out.update(alpha=ah[:k], beta=bh[:k], res=rh[:k + 1])
    if state:
        out["state"] = {nm: st[i * a.n:(i + 1) * a.n] for i, nm in enumerate(("x", "r", "u", "p"))}
    return out
