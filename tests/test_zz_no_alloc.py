"""The allocation-free entry point, ppcg_solve_noalloc, called through the C ABI.

It exists for callers that may not allocate device memory while solving (framework-owned
memory pools, real-time loops where cudaMalloc/cudaFree would stall the device, plug-ins
that forbid allocation after start-up); it keeps its working vectors in a static device
array of the library.  This file checks, on two calls in a row, that its result agrees
with the regular entry point (ppcg_create + ppcg_solve) within the tolerance the parity
tests use, that the second call is not disturbed by what the first left in the shared
scratch, and that sizes over its limit are refused.  It is named so that pytest collects it
last, and it passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def pp():
    import paper_2105_06176_b300 as m
    return m


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def noalloc(a, b, tol, maxit, x0=None):
    m = pp()
    rp = dev(a.row_ptr.astype(np.int64), torch.int64)
    ci = dev(a.col.astype(np.int32), torch.int32)
    va = dev(a.val)
    bd = dev(b)
    x = torch.empty(a.n, dtype=torch.float64, device="cuda")
    info = m.Info()
    stream = torch.cuda.current_stream().cuda_stream
    st = m.lib().ppcg_solve_noalloc(a.n, a.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), bd.data_ptr(),
                                    None if x0 is None else x0.data_ptr(), x.data_ptr(), tol, maxit, stream,
                                    ctypes.byref(info))
    assert st == m.OK, m.last_error()
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


def regular(a, b, tol, maxit):
    m = pp()
    s = m.Solver.from_csr(a)
    x, info = s.solve(dev(b), tol=tol, maxit=maxit)
    out = x.cpu().numpy(), info
    s.close()
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [("poisson2d_64", 30), ("varcoeff2d_150", 25), ("varcoeff3d_31", 20)]


def system(name):
    if name == "poisson2d_64":
        a = synth.poisson2d(64)
        return a, a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    if name == "varcoeff2d_150":
        a = synth.varcoeff2d(150, seed=4)
        return a, synth.rhs_uniform(a.n, 4)
    a = synth.varcoeff3d(31, seed=1)
    return a, synth.rhs_uniform(a.n, 1)


@pytest.mark.parametrize("name,k", CASES)
def test_two_calls_match_regular_entry_point(name, k):
    m = pp()
    a, b = system(name)
    ref_k, _ = regular(a, b, 0.0, k)
    ref_full, ref_info = regular(a, b, 1e-8, 20000)
    for call in range(2):                       # two calls in a row share the scratch
        xk, ik = noalloc(a, b, 0.0, k)
        assert ik.status == m.ERR_NOT_CONVERGED and ik.iters == k
        assert rel(xk, ref_k) <= 1e-10, (call, rel(xk, ref_k))
        xf, inf = noalloc(a, b, 1e-8, 20000)
        assert inf.status == m.OK
        assert abs(inf.iters - ref_info.iters) <= 2
        assert inf.rel_res_true <= 1e-8
        t = np.linalg.norm(b - a.to_scipy() @ xf) / np.linalg.norm(b)
        assert t <= 1e-8
        assert rel(xf, ref_full) <= 1e-6


def test_small_then_large_call_and_limits():
    """A larger system right after a smaller one (stale scratch beyond the small n is never
    read), then the size limit."""
    m = pp()
    a1, b1 = system("poisson2d_64")
    a2, b2 = system("varcoeff2d_150")
    noalloc(a1, b1, 1e-8, 20000)
    x2, i2 = noalloc(a2, b2, 1e-8, 20000)
    r2, ri2 = regular(a2, b2, 1e-8, 20000)
    assert i2.status == m.OK and abs(i2.iters - ri2.iters) <= 2 and rel(x2, r2) <= 1e-6
    big = synth.poisson2d(257)                   # 66,049 rows > 65,536
    st = m.lib().ppcg_solve_noalloc(big.n, big.nnz, None, None, None, None, None, None, 1e-8, 10, None, None)
    assert st == m.ERR_ARG
    assert "exceeds" in m.last_error()
