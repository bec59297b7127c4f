"""The allocation-free entry point, ppcg_solve_noalloc, called through the C ABI.

It exists for callers that may not allocate device memory while solving (framework-owned
memory pools, real-time loops where cudaMalloc/cudaFree would stall the device, plug-ins
that forbid allocation after start-up); it keeps its working vectors in a static device
array of the library.  This file checks, on two calls in a row, that its result agrees
with the regular entry point (ppcg_create + ppcg_solve) and with the oracle within the
tolerance the parity tests use, that the second call is not disturbed by what the first
left in the shared scratch, that a warmed call changes no device memory (and succeeds while
every library device allocation is made to fail), the edge cases (x0 aliasing x, b = 0, a
zero diagonal entry, a malformed matrix, info = NULL), and that sizes over its limit are
refused.  It is named so that pytest collects it last, and it passes both alone and after
the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


class DevCSR:
    """The caller's device copy of a CSR matrix (the entry point reads it in place)."""

    def __init__(self, a, col=None, nnz=None):
        self.n = a.n
        self.nnz = a.nnz if nnz is None else nnz
        self.rp = dev(a.row_ptr.astype(np.int64), torch.int64)
        self.ci = dev((a.col if col is None else col).astype(np.int32), torch.int32)
        self.va = dev(a.val)


def call(csr, bd, x, tol, maxit, x0=None, with_info=True):
    """One ppcg_solve_noalloc call on device buffers; returns (status, info or None)."""
    m = pp()
    info = m.Info() if with_info else None
    stream = torch.cuda.current_stream().cuda_stream
    st = m.lib().ppcg_solve_noalloc(csr.n, csr.nnz, csr.rp.data_ptr(), csr.ci.data_ptr(), csr.va.data_ptr(),
                                    bd.data_ptr(), None if x0 is None else x0.data_ptr(), x.data_ptr(), tol,
                                    maxit, stream, ctypes.byref(info) if with_info else None)
    return st, info


def noalloc(a, b, tol, maxit, x0=None):
    m = pp()
    csr = DevCSR(a)
    bd = dev(b)
    x = torch.empty(a.n, dtype=torch.float64, device="cuda")
    st, info = call(csr, bd, x, tol, maxit, x0)
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


def rel_inf(a, b):
    """Element-wise companion of rel(): max |a - b| / max |b|."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


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
    ora_k = oracle.pipecg(a, b, tol=0.0, maxit=k)["x"]
    ref_full, ref_info = regular(a, b, 1e-8, 20000)
    for rep in range(2):                        # two calls in a row share the scratch
        xk, ik = noalloc(a, b, 0.0, k)
        assert ik.status == m.ERR_NOT_CONVERGED and ik.iters == k
        assert rel(xk, ref_k) <= 1e-10, (rep, rel(xk, ref_k))
        assert rel(xk, ora_k) <= 1e-10 and rel_inf(xk, ora_k) <= 1e-10, (rep, rel(xk, ora_k), rel_inf(xk, ora_k))
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


def test_warmed_call_allocates_nothing(monkeypatch):
    """After the set-up call (n = 0) and one warm-up solve (the driver may size per-launch
    resources on a kernel's first launch), two solves leave the device's free memory
    unchanged, and they succeed while the library's own device allocator is made to fail."""
    m = pp()
    a, b = system("varcoeff3d_31")
    csr = DevCSR(a)
    bd = dev(b)
    x = torch.empty(a.n, dtype=torch.float64, device="cuda")
    assert m.lib().ppcg_solve_noalloc(0, 0, None, None, None, None, None, None, 1e-8, 10, None, None) == m.OK
    assert call(csr, bd, x, 1e-8, 20000)[0] == m.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("PPCG_FAIL_DEVICE_ALLOC", "1")
    infos = []
    for _ in range(2):
        st, info = call(csr, bd, x, 1e-8, 20000)
        assert st == m.OK, m.last_error()
        infos.append(info)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    monkeypatch.delenv("PPCG_FAIL_DEVICE_ALLOC")
    assert free1 == free0, (free0, free1)
    assert all(i.status == m.OK and i.rel_res_true <= 1e-8 for i in infos)
    assert infos[0].iters == infos[1].iters


def test_x0_aliasing_x_and_info_null():
    """A non-zero initial guess in the output buffer itself matches ppcg_solve from the same
    guess; a call with info = NULL computes the same x."""
    m = pp()
    a, b = system("varcoeff2d_150")
    k = 25
    x0 = synth.rhs_uniform(a.n, 77)
    s = m.Solver.from_csr(a)
    ref, _ = s.solve(dev(b), dev(x0), tol=0.0, maxit=k)
    ref = ref.cpu().numpy()
    s.close()
    ora = oracle.pipecg(a, b, x0=x0, tol=0.0, maxit=k)["x"]
    csr = DevCSR(a)
    bd = dev(b)
    x = dev(x0)
    st, info = call(csr, bd, x, 0.0, k, x0=x)
    assert st == m.OK and info.status == m.ERR_NOT_CONVERGED and info.iters == k
    got = x.cpu().numpy()
    assert rel(got, ref) <= 1e-10 and rel(got, ora) <= 1e-10 and rel_inf(got, ora) <= 1e-10
    y = dev(x0)
    st, none = call(csr, bd, y, 0.0, k, x0=y, with_info=False)
    assert st == m.OK and none is None
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(y.cpu().numpy(), got)


def test_zero_rhs_and_bad_matrices():
    """b = 0: x = 0 after 0 iterations, OK.  A zero diagonal entry: NOT_SPD.  A column just
    past n, or row pointers that disagree with nnz: the solve ends with ERR_ARG (the matrix
    is checked on the device before any gather), and a good call afterwards is unaffected."""
    m = pp()
    a, b = system("poisson2d_64")
    csr = DevCSR(a)
    x = torch.full((a.n,), 7.0, dtype=torch.float64, device="cuda")
    st, info = call(csr, dev(np.zeros(a.n)), x, 1e-8, 100)
    assert st == m.OK and info.status == m.OK and info.iters == 0
    assert not torch.any(x != 0).item()

    val = a.val.copy()
    diag = np.flatnonzero(a.col == np.repeat(np.arange(a.n), np.diff(a.row_ptr)))
    val[diag[100]] = 0.0
    bad_diag = synth.CSR(a.n, a.row_ptr, a.col, val)
    st, info = call(DevCSR(bad_diag), dev(b), x, 1e-8, 100)
    assert st == m.OK and info.status == m.ERR_NOT_SPD

    col = a.col.copy()
    col[5] = a.n                                  # one past the last column
    st, info = call(DevCSR(a, col=col), dev(b), x, 1e-8, 100)
    assert st == m.OK and info.status == m.ERR_ARG and info.iters == 0
    st, info = call(DevCSR(a, nnz=a.nnz - 1), dev(b), x, 1e-8, 100)   # row_ptr[n] != nnz
    assert st == m.OK and info.status == m.ERR_ARG

    xg, ig = noalloc(a, b, 1e-8, 20000)
    assert ig.status == m.OK and np.linalg.norm(b - a.to_scipy() @ xg) / np.linalg.norm(b) <= 1e-8
