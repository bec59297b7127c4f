"""GPU parity: the CUDA path (through the C ABI) against the oracle on the same seeded inputs.

Bars (FP64): x after a fixed number of iterations k within 1e-10 relative of the oracle's
x_k, at k where two summation orders of the oracle itself agree to 1e-12
(test_oracle_pins.test_summation_order_sensitivity); full solves reach a true relative
residual <= tol with the oracle's iteration count +-2.
"""
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
    import paper_2105_06176_b300 as pp
    pp.lib()


def pp():
    import paper_2105_06176_b300 as m
    return m


def rel(a, b):
    """Relative difference of a from b: the larger of the norm-wise ||a - b||_2 / ||b||_2 and
    the element-wise ||a - b||_inf / ||b||_inf, so that one wrong entry cannot hide in the
    norm of a long vector."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = a - b
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), np.max(np.abs(d)) / np.max(np.abs(b))))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu(a, b, x0=None, tol=1e-8, maxit=10000, **opts):
    s = pp().Solver.from_csr(a, **opts)
    x, info = s.solve(dev(b), None if x0 is None else dev(x0), tol=tol, maxit=maxit)
    out = x.cpu().numpy(), info
    s.close()
    return out


def problem(name):
    if name == "poisson2d_64":
        a = synth.poisson2d(64)
        return a, a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    if name == "varcoeff3d_31":         # 29,791 rows: 931 chunks, ragged last chunk
        a = synth.varcoeff3d(31, seed=1)
        return a, synth.rhs_uniform(a.n, 1)
    if name == "varcoeff2d_150":
        a = synth.varcoeff2d(150, seed=4)
        return a, synth.rhs_uniform(a.n, 4)
    if name == "rgg_20k":               # irregular row lengths (sorted SELL windows: see below)
        a = synth.rgg_laplacian(20000, (3 * 14.0 / (4 * np.pi * 20000)) ** (1 / 3), 1e-3, 5)
        return a, synth.rhs_uniform(a.n, 5)
    if name == "box125_12":             # Table II structure: 124 off-diagonals per interior row
        a = synth.box125(12)
        return a, synth.rhs_uniform(a.n, 6)
    raise KeyError(name)


PATHS = [dict(path=1), dict(path=2)]      # GRID, CLUSTER


@pytest.mark.parametrize("name,k", [("poisson2d_64", 50), ("varcoeff3d_31", 20), ("varcoeff2d_150", 30),
                                    ("rgg_20k", 20), ("box125_12", 15)])
@pytest.mark.parametrize("opts", PATHS, ids=["grid", "cluster"])
def test_fixed_k_parity(name, k, opts):
    a, b = problem(name)
    ref = oracle.pipecg(a, b, tol=0.0, maxit=k)
    x, info = gpu(a, b, tol=0.0, maxit=k, **opts)
    assert info.status == pp().ERR_NOT_CONVERGED and info.iters == k
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("sigma", [64, 256, 2048])
@pytest.mark.parametrize("opts", PATHS, ids=["grid", "cluster"])
def test_sorted_sell_parity(sigma, opts):
    """Rows sorted by length inside sigma-row windows: the solver runs on the permuted
    system and maps b, x0 and x through the permutation."""
    a, b = problem("rgg_20k")
    ref = oracle.pipecg(a, b, tol=0.0, maxit=20)
    x, info = gpu(a, b, tol=0.0, maxit=20, sigma=sigma, **opts)
    assert info.iters == 20 and rel(x, ref["x"]) <= 1e-10
    full = oracle.pipecg(a, b, tol=1e-8, maxit=5000)["result"]["iters"]
    x, info = gpu(a, b, tol=1e-8, maxit=5000, sigma=sigma, **opts)
    assert info.status == pp().OK and abs(info.iters - full) <= 2
    assert np.linalg.norm(b - a.to_scipy() @ x) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["poisson2d_64", "varcoeff3d_31", "rgg_20k", "box125_12"])
@pytest.mark.parametrize("opts", PATHS, ids=["grid", "cluster"])
def test_full_solve_parity(name, opts):
    a, b = problem(name)
    ref = oracle.pipecg(a, b, tol=1e-8, maxit=20000)
    x, info = gpu(a, b, tol=1e-8, maxit=20000, **opts)
    assert info.status == pp().OK
    assert abs(info.iters - ref["result"]["iters"]) <= 2
    assert info.rel_res_true <= 1e-8
    t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert t <= 1e-8
    assert info.rel_res_true == pytest.approx(t, rel=1e-6, abs=1e-14)
    assert rel(x, ref["x"]) <= 1e-6


def test_nonzero_x0_and_aliasing():
    a, b = problem("varcoeff2d_150")
    x0 = synth.xtrue_uniform(a.n, 9)
    ref = oracle.pipecg(a, b, x0=x0, tol=0.0, maxit=25)
    s = pp().Solver.from_csr(a)
    xd = dev(x0)
    x, info = s.solve(dev(b), xd, xd, tol=0.0, maxit=25)    # x aliases x0
    assert rel(xd.cpu().numpy(), ref["x"]) <= 1e-10


def test_host_pointers_match_device():
    a, b = problem("poisson2d_64")
    s = pp().Solver.from_csr(a)
    xh = np.empty(a.n)
    _, ih = s.solve(np.ascontiguousarray(b), None, xh, tol=1e-8)
    xd, idv = s.solve(dev(b), tol=1e-8)
    assert ih.status == idv.status == pp().OK and ih.iters == idv.iters
    assert np.array_equal(xh, xd.cpu().numpy())


def test_paper_norm_mode():
    """Sec. VI protocol: absolute tol 1e-5 on sqrt((u,u)), exact solution 1/sqrt(N)."""
    a = synth.varcoeff2d(64, seed=3)
    b = a.to_scipy() @ np.full(a.n, 1.0 / np.sqrt(a.n))
    ref = oracle.pipecg(a, b, tol=1e-5, maxit=10000, norm=oracle.NORM_PAPER_U_ABS)
    for path in (1, 2):
        x, info = gpu(a, b, tol=1e-5, maxit=10000, norm=pp().NORM_PAPER_U_ABS, path=path)
        assert info.status == pp().OK
        assert abs(info.iters - ref["result"]["iters"]) <= 2
        assert info.rel_res_recursive <= 1e-5


@pytest.mark.parametrize("period", [10, 37])
def test_residual_replacement_parity(period):
    a, b = problem("poisson2d_64")
    ref = oracle.pipecg(a, b, tol=0.0, maxit=60, rr_period=period)
    x, info = gpu(a, b, tol=0.0, maxit=60, rr_period=period, path=1)
    assert info.rr_count == ref["result"]["rr_count"]
    assert rel(x, ref["x"]) <= 1e-10


def test_edge_cases():
    m = pp()
    a = synth.poisson2d(16)
    b = synth.rhs_uniform(a.n, 2)
    # b = 0 -> x = 0, 0 iterations, OK
    s = m.Solver.from_csr(a)
    x, info = s.solve(dev(np.zeros(a.n)), dev(np.ones(a.n)))
    assert info.status == m.OK and info.iters == 0 and not x.cpu().numpy().any()
    # exact initial guess -> 0 iterations
    xs = np.linalg.solve(a.dense(), b)
    x, info = s.solve(dev(b), dev(xs), tol=1e-8)
    assert info.status == m.OK and info.iters == 0
    # maxit = 0 -> NOT_CONVERGED, x = x0
    x, info = s.solve(dev(b), None, tol=1e-8, maxit=0)
    assert info.status == m.ERR_NOT_CONVERGED and info.iters == 0 and not x.cpu().numpy().any()
    # NaN in b -> NONFINITE
    bn = b.copy()
    bn[3] = np.nan
    x, info = s.solve(dev(bn), tol=1e-8)
    assert info.status == m.ERR_NONFINITE
    # n = 1
    one = synth.CSR(1, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([4.0]))
    x, info = gpu(one, np.array([2.0]))
    assert info.status == m.OK and x[0] == pytest.approx(0.5)


def test_create_rejects_bad_matrices():
    m = pp()
    bad_diag = synth.CSR(2, np.array([0, 2, 3], dtype=np.int64), np.array([0, 1, 0], dtype=np.int32),
                         np.array([2.0, -1.0, -1.0]))
    with pytest.raises(m.PPCGError) as e:
        m.Solver.from_csr(bad_diag)
    assert e.value.status == m.ERR_NOT_SPD
    bad_col = synth.CSR(2, np.array([0, 2, 4], dtype=np.int64), np.array([0, 5, 0, 1], dtype=np.int32),
                        np.array([2.0, -1.0, -1.0, 2.0]))
    with pytest.raises(m.PPCGError) as e:
        m.Solver.from_csr(bad_col)
    assert e.value.status == m.ERR_ARG


def test_indefinite_breakdown():
    m = pp()
    mat = np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    import scipy.sparse as sp
    c = sp.csr_matrix(mat)
    a = synth.CSR(3, c.indptr.astype(np.int64), c.indices.astype(np.int32), c.data)
    for path in (1, 2):
        x, info = gpu(a, np.array([1.0, -1.0, 1.0]), path=path)
        assert info.status == m.ERR_BREAKDOWN


def test_barrier_timeout_is_reported_not_hung():
    """Failure detection: one CTA of the grid barrier never arrives; the others give up after
    50 ms and report a timeout (no hang, no fault, context still usable)."""
    m = pp()
    st, n = m.barrier_timeout_selftest(grid=32, drop_rank=5, limit_ns=50_000_000)
    assert st == m.OK
    assert n >= 1
    a, b = problem("poisson2d_64")
    x, info = gpu(a, b)             # the context still works
    assert info.status == m.OK


def test_breakdown_system_parity():
    """The 2-D log-normal system on which Alg. 2 broke down near 1e-8.  With the
    measured-gap residual replacement (the default, in the library and the oracle alike) it
    no longer breaks down, even with restarts off: every path converges with an iteration
    count inside the oracle's envelope (its sequential- and pairwise-sum counts, widened by
    2), which is also Alg. 1's count.  With the trigger off the old behaviour remains: the
    alpha denominator turns non-positive near the attainable accuracy, at an iteration that
    rounding decides (the bar: within 1% of the oracle's), and after restarts the solve
    still reaches the true residual -- a count after a restart is rounding-decided, so there
    only the outcome is compared."""
    m = pp()
    spec = [s for s in synth.batch_mix(128, 11) if s[0] == "varcoeff2d" and s[1] == 267][0]
    a, b = synth.build_spec(spec)
    seq = oracle.pipecg(a, b, tol=1e-8, maxit=20000)["result"]["iters"]
    pair = oracle.pipecg(a, b, tol=1e-8, maxit=20000, sum_mode=1)["result"]["iters"]
    classic = oracle.pcg(a, b, tol=1e-8, maxit=20000)["result"]["iters"]
    ref0 = oracle.pipecg(a, b, tol=1e-8, maxit=20000, max_restarts=0, gap_theta=0.0)
    for path in (1, 2):
        for restarts in (8, 0):
            x, info = gpu(a, b, tol=1e-8, maxit=20000, path=path, max_restarts=restarts)
            assert info.status == m.OK, (path, restarts, info)
            assert min(seq, pair) - 2 <= info.iters <= max(seq, pair) + 2, (path, info.iters, seq, pair)
            assert abs(info.iters - classic) <= 4
            assert np.linalg.norm(b - a.to_scipy() @ x) <= 1e-8 * np.linalg.norm(b)
        x0, info0 = gpu(a, b, tol=1e-8, maxit=20000, path=path, max_restarts=0, gap_theta=-1.0)
        assert info0.status == m.ERR_BREAKDOWN
        assert abs(info0.iters - ref0["result"]["iters"]) <= max(2, 0.01 * ref0["result"]["iters"])
        x, info = gpu(a, b, tol=1e-8, maxit=20000, path=path, gap_theta=-1.0)
        assert info.status == m.OK and info.rr_count >= 1
        assert np.linalg.norm(b - a.to_scipy() @ x) <= 1e-8 * np.linalg.norm(b)


# ------------------------------------------------------- on-chip path (one cluster's DSMEM) --

ONCHIP = dict(path=3)


def onchip_problem(name):
    if name == "poisson2d_64":
        return problem("poisson2d_64")
    if name == "varcoeff3d_20":          # 8,000 rows: 250 chunks over 8 CTAs (ragged split)
        a = synth.varcoeff3d(20, seed=7)
        return a, synth.rhs_uniform(a.n, 7)
    if name == "rgg_5000":               # irregular rows
        a = synth.rgg_laplacian(5000, (3 * 14.0 / (4 * np.pi * 5000)) ** (1 / 3), 1e-3, 8)
        return a, synth.rhs_uniform(a.n, 8)
    if name == "box125_9":               # 124 off-diagonals: long rows (8-slot batches)
        a = synth.box125(9)
        return a, synth.rhs_uniform(a.n, 9)
    if name == "poisson2d_7":            # 49 rows: one ragged chunk, seven idle CTAs
        a = synth.poisson2d(7)
        return a, a.to_scipy() @ synth.xtrue_uniform(a.n, 3)
    raise KeyError(name)


@pytest.mark.parametrize("name,k", [("poisson2d_64", 50), ("varcoeff3d_20", 20), ("rgg_5000", 20),
                                    ("box125_9", 10), ("poisson2d_7", 8)])
def test_onchip_fixed_k_parity(name, k):
    a, b = onchip_problem(name)
    ref = oracle.pipecg(a, b, tol=0.0, maxit=k)
    x, info = gpu(a, b, tol=0.0, maxit=k, **ONCHIP)
    assert info.status == pp().ERR_NOT_CONVERGED and info.iters == k
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("name", ["poisson2d_64", "varcoeff3d_20", "rgg_5000", "box125_9", "poisson2d_7"])
def test_onchip_full_solve_parity(name):
    a, b = onchip_problem(name)
    ref = oracle.pipecg(a, b, tol=1e-8, maxit=10000)
    x, info = gpu(a, b, tol=1e-8, maxit=10000, **ONCHIP)
    assert info.status == pp().OK
    assert abs(info.iters - ref["result"]["iters"]) <= 2
    t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert t <= 1e-8 and abs(info.rel_res_true - t) <= 1e-6 * t + 1e-15


def test_onchip_modes_and_plan():
    m = pp()
    a, b = onchip_problem("poisson2d_64")
    # AUTO takes the on-chip path when the system fits; the result equals the explicit one
    xa, ia = gpu(a, b, tol=1e-8)
    xo, io = gpu(a, b, tol=1e-8, **ONCHIP)
    assert ia.iters == io.iters and np.array_equal(xa, xo)
    # residual replacement, paper norm, x0 aliasing x, budgets through resumable launches
    ref = oracle.pipecg(a, b, tol=0.0, maxit=60, rr_period=10)
    x, info = gpu(a, b, tol=0.0, maxit=60, rr_period=10, **ONCHIP)
    assert info.rr_count == ref["result"]["rr_count"] and rel(x, ref["x"]) <= 1e-10
    bp = a.to_scipy() @ np.full(a.n, 1.0 / np.sqrt(a.n))
    refp = oracle.pipecg(a, bp, tol=1e-5, maxit=10000, norm=oracle.NORM_PAPER_U_ABS)
    x, info = gpu(a, bp, tol=1e-5, maxit=10000, norm=m.NORM_PAPER_U_ABS, **ONCHIP)
    assert info.status == m.OK and abs(info.iters - refp["result"]["iters"]) <= 2
    x0 = synth.xtrue_uniform(a.n, 5)
    refx = oracle.pipecg(a, b, x0=x0, tol=0.0, maxit=25)
    s = m.Solver.from_csr(a, **ONCHIP)
    xd = dev(x0)
    s.solve(dev(b), xd, xd, tol=0.0, maxit=25)
    assert rel(xd.cpu().numpy(), refx["x"]) <= 1e-10
    # indefinite: breakdown reported
    import scipy.sparse as sp
    c = sp.csr_matrix(np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]]))
    ind = synth.CSR(3, c.indptr.astype(np.int64), c.indices.astype(np.int32), c.data)
    _, info = gpu(ind, np.array([1.0, -1.0, 1.0]), **ONCHIP)
    assert info.status == m.ERR_BREAKDOWN
    # refused: FP32 modes, the scaled variant, systems that do not fit
    for kw in (dict(precision=m.FP32_RU), dict(variant=1)):
        with pytest.raises(m.PPCGError) as e:
            m.Solver.from_csr(a, **ONCHIP, **kw)
        assert e.value.status == m.ERR_ARG
    big = synth.varcoeff3d(40, seed=1)
    with pytest.raises(m.PPCGError) as e:
        m.Solver.from_csr(big, **ONCHIP)
    assert e.value.status == m.ERR_ARG


def test_onchip_in_batch_bitwise_equals_solo():
    m = pp()
    systems = [onchip_problem(nm) for nm in ("poisson2d_64", "varcoeff3d_20", "rgg_5000", "poisson2d_7")]
    systems.append(problem("varcoeff3d_31"))                     # a cluster-path member
    solvers = [m.Solver.from_csr(a) for a, _ in systems]
    bs = [dev(b) for _, b in systems]
    solo = [s.solve(b, tol=1e-8, maxit=10000) for s, b in zip(solvers, bs)]
    solo = [(x.cpu().numpy(), i.iters) for x, i in solo]
    xs = [torch.empty_like(b) for b in bs]
    infos = m.batch_solve(solvers, bs, xs, tol=1e-8, maxit=10000)
    for (x0, it0), xb, inf in zip(solo, xs, infos):
        assert inf.status == m.OK and inf.iters == it0
        assert np.array_equal(xb.cpu().numpy(), x0)


# ------------------------------------------- matrix-free box stencil (Table II family, f3) --

BOX = dict(format=3, path=1)


def box_problem(name):
    if name == "box125_24":              # R = 2, 13,824 rows: 432 chunks, grid rows of 24
        a = synth.box125(24)
        return a, synth.rhs_uniform(a.n, 11)
    if name == "box27_33":               # R = 1, 35,937 rows, a ragged last chunk
        a = synth.box_stencil(33, 1, 26.5, -1.0)
        return a, synth.rhs_uniform(a.n, 12)
    if name == "box343_12":              # R = 3
        a = synth.box_stencil(12, 3, 400.0, -1.0)
        return a, synth.rhs_uniform(a.n, 13)
    raise KeyError(name)


@pytest.mark.parametrize("name,k", [("box125_24", 12), ("box27_33", 25), ("box343_12", 8)])
def test_box_fixed_k_parity(name, k):
    a, b = box_problem(name)
    ref = oracle.pipecg(a, b, tol=0.0, maxit=k)
    x, info = gpu(a, b, tol=0.0, maxit=k, **BOX)
    assert info.bytes_per_iter == pytest.approx(21 * 8 * a.n)      # the matrix-free plan
    assert info.iters == k and rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("shape", [1, 2])
def test_box_launch_shapes(shape, monkeypatch):
    """The other launch shapes of the box kernel (256 and 1024 threads per CTA; the tuning
    knob indexes the box plan's own kernels) meet the same fixed-k bar."""
    monkeypatch.setenv("PPCG_GRID_SHAPE", str(shape))
    a, b = box_problem("box125_24")
    ref = oracle.pipecg(a, b, tol=0.0, maxit=12)
    x, info = gpu(a, b, tol=0.0, maxit=12, **BOX)
    assert info.status == pp().ERR_NOT_CONVERGED
    assert info.iters == 12 and rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("name", ["box125_24", "box27_33", "box343_12"])
def test_box_full_solve_parity(name):
    a, b = box_problem(name)
    ref = oracle.pipecg(a, b, tol=1e-8, maxit=5000)
    x, info = gpu(a, b, tol=1e-8, maxit=5000, **BOX)
    assert info.status == pp().OK and abs(info.iters - ref["result"]["iters"]) <= 2
    t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert t <= 1e-8 and abs(t - info.rel_res_true) <= 1e-6 * t


def test_box_modes_detection_and_rejects():
    m = pp()
    a, b = box_problem("box125_24")
    # AUTO detects the stencil on the grid path and gives the same iterates as FMT_BOX
    xa, ia = gpu(a, b, tol=1e-8, maxit=5000, path=1)
    xb, ib = gpu(a, b, tol=1e-8, maxit=5000, **BOX)
    assert ia.iters == ib.iters and np.array_equal(xa, xb)
    # FMT_SELL keeps the matrix: different plan, same answer within the parity bars
    xs, is_ = gpu(a, b, tol=1e-8, maxit=5000, format=2, path=1)
    assert abs(is_.iters - ib.iters) <= 2
    # residual replacement, paper norm, nonzero x0
    ref = oracle.pipecg(a, b, tol=0.0, maxit=30, rr_period=7)
    x, info = gpu(a, b, tol=0.0, maxit=30, rr_period=7, **BOX)
    assert info.rr_count == ref["result"]["rr_count"] and rel(x, ref["x"]) <= 1e-10
    bp = a.to_scipy() @ np.full(a.n, 1.0 / np.sqrt(a.n))
    refp = oracle.pipecg(a, bp, tol=1e-5, maxit=10000, norm=oracle.NORM_PAPER_U_ABS)
    x, info = gpu(a, bp, tol=1e-5, maxit=10000, norm=m.NORM_PAPER_U_ABS, **BOX)
    assert info.status == m.OK and abs(info.iters - refp["result"]["iters"]) <= 2
    x0 = synth.xtrue_uniform(a.n, 3)
    refx = oracle.pipecg(a, b, x0=x0, tol=0.0, maxit=10)
    x, info = gpu(a, b, x0=x0, tol=0.0, maxit=10, **BOX)
    assert rel(x, refx["x"]) <= 1e-10
    # not a constant box stencil, or not FP64 Alg. 2, or not the grid path: refused
    v = synth.varcoeff3d(24, seed=2)
    for mat, kw in ((v, dict(path=1)), (a, dict(path=1, precision=m.FP32_RU)), (a, dict(path=1, variant=1)),
                    (a, dict(path=2))):
        with pytest.raises(m.PPCGError) as e:
            m.Solver.from_csr(mat, format=3, **kw)
        assert e.value.status == m.ERR_ARG
    # a perturbed value breaks the detection: AUTO keeps the SELL matrix
    bad = synth.CSR(a.n, a.row_ptr.copy(), a.col.copy(), a.val.copy())
    bad.val[len(bad.val) // 2] *= 1.0 + 1e-15
    _, info = gpu(bad, b, tol=1e-8, maxit=1, path=1)
    assert info.bytes_per_iter != pytest.approx(21 * 8 * a.n)


# ----------------------------------------------------- Jacobi-scaled variant (next row f1) --

SCALED = dict(variant=1)


@pytest.mark.parametrize("name,k", [("poisson2d_64", 50), ("varcoeff3d_31", 20), ("rgg_20k", 20)])
@pytest.mark.parametrize("path", [1, 2], ids=["grid", "cluster"])
def test_scaled_variant_fixed_k_parity(name, k, path):
    """The Jacobi-scaled variant against the oracle's Jacobi-elimination mode (its own
    definition) and against Alg. 2 itself, both to 1e-10 at the calibrated k."""
    a, b = problem(name)
    x, info = gpu(a, b, tol=0.0, maxit=k, path=path, **SCALED)
    assert info.iters == k
    assert rel(x, oracle.pipecg(a, b, tol=0.0, maxit=k, jacobi_elim=True)["x"]) <= 1e-10
    assert rel(x, oracle.pipecg(a, b, tol=0.0, maxit=k)["x"]) <= 1e-10


@pytest.mark.parametrize("name", ["poisson2d_64", "varcoeff3d_31", "rgg_20k"])
def test_scaled_variant_full_solve(name):
    a, b = problem(name)
    ref = oracle.pipecg(a, b, tol=1e-8, maxit=20000, jacobi_elim=True)
    for path in (1, 2):
        x, info = gpu(a, b, tol=1e-8, maxit=20000, path=path, **SCALED)
        assert info.status == pp().OK
        assert abs(info.iters - ref["result"]["iters"]) <= 2
        t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
        assert t <= 1e-8 and info.rel_res_true == pytest.approx(t, rel=1e-6, abs=1e-14)


def test_scaled_variant_modes():
    """Non-zero x0, periodic residual replacement and the paper's norm in the variant."""
    a, b = problem("varcoeff2d_150")
    x0 = synth.xtrue_uniform(a.n, 9)
    ref = oracle.pipecg(a, b, x0=x0, tol=0.0, maxit=40, rr_period=15, jacobi_elim=True)
    x, info = gpu(a, b, x0=x0, tol=0.0, maxit=40, rr_period=15, path=1, **SCALED)
    assert info.rr_count == ref["result"]["rr_count"]
    assert rel(x, ref["x"]) <= 1e-10
    a2 = synth.varcoeff2d(64, seed=3)
    b2 = a2.to_scipy() @ np.full(a2.n, 1.0 / np.sqrt(a2.n))
    r2 = oracle.pipecg(a2, b2, tol=1e-5, maxit=10000, norm=oracle.NORM_PAPER_U_ABS, jacobi_elim=True)
    x2, i2 = gpu(a2, b2, tol=1e-5, maxit=10000, norm=pp().NORM_PAPER_U_ABS, **SCALED)
    assert i2.status == pp().OK and abs(i2.iters - r2["result"]["iters"]) <= 2
    with pytest.raises(pp().PPCGError):
        pp().Solver.from_csr(a, precision=pp().FP32_IR, **SCALED)


# ------------------------------------------------------- every grid-path kernel shape --

# PPCG_GRID_SHAPE picks the launch shape of a SELL plan's grid kernel (threads per CTA,
# register budget, bulk-copy staging of the vector tiles for shapes 6-8); every shape must
# meet the bars of every form.
@pytest.mark.parametrize("shape", range(9))
def test_fp64_launch_shapes(shape, monkeypatch):
    monkeypatch.setenv("PPCG_GRID_SHAPE", str(shape))
    a, b = problem("varcoeff3d_31")
    ref = oracle.pipecg(a, b, tol=0.0, maxit=20)
    x, info = gpu(a, b, tol=0.0, maxit=20, path=1)
    assert info.status == pp().ERR_NOT_CONVERGED and info.iters == 20
    assert rel(x, ref["x"]) <= 1e-10


@pytest.mark.parametrize("shape", [0, 1, 6])
def test_scaled_launch_shapes(shape, monkeypatch):
    monkeypatch.setenv("PPCG_GRID_SHAPE", str(shape))
    a, b = problem("varcoeff3d_31")
    x, info = gpu(a, b, tol=0.0, maxit=20, path=1, variant=1)
    assert info.iters == 20
    assert rel(x, oracle.pipecg(a, b, tol=0.0, maxit=20, jacobi_elim=True)["x"]) <= 1e-10


@pytest.mark.parametrize("shape", [0, 1, 6])
@pytest.mark.parametrize("precision", [1, 2], ids=["fp32_ir", "fp32_ru"])
def test_mixed_launch_shapes(shape, precision, monkeypatch):
    monkeypatch.setenv("PPCG_GRID_SHAPE", str(shape))
    a, b = problem("varcoeff3d_31")
    x, info = gpu(a, b, tol=1e-8, maxit=20000, path=1, precision=precision)
    assert info.status == pp().OK
    t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert t <= 1e-8
    x64 = oracle.pipecg(a, b, tol=1e-10, maxit=20000)["x"]
    assert rel(x, x64) <= 1e-4


def test_column_modes_give_bitwise_the_same_iterates(monkeypatch):
    """A stencil's columns formed from its offset pattern (the default where every row draws
    its off-diagonals, in ascending order, from at most 16 offsets), read as one-byte indices
    into its distinct col - row offsets (PPCG_COL_PAT=0, the default where a matrix has at most
    255 of them) and read as plain 4-byte columns (PPCG_COL_DICT=0) give bitwise the same
    iterates: the pattern's extra slots hold zeros, which add nothing, and the nonzero terms
    of each row are summed in the same order.  Covers FP64 Alg. 2, FP32_RU, FP32_IR and the
    Jacobi-scaled variant on the grid path, a pattern matrix on the cluster path (whose
    kernel reads the pattern's stored columns), full solves, and the plan each mode reports."""
    m = pp()
    cases = [("varcoeff3d_31", dict(path=1, precision=0), m.COLS_PATTERN),
             ("varcoeff2d_150", dict(path=1, precision=0), m.COLS_PATTERN),
             ("varcoeff3d_31", dict(path=1, precision=2), m.COLS_PATTERN),
             ("varcoeff3d_31", dict(path=1, precision=1), m.COLS_PATTERN),
             ("varcoeff3d_31", dict(path=1, variant=1), m.COLS_PATTERN),
             ("varcoeff2d_150", dict(path=2, precision=0), m.COLS_SELL),
             ("box125_12", dict(path=1, precision=0), m.COLS_DICT)]
    for name, kw, want in cases:
        a, b = problem(name)
        res = {}
        for mode, env in (("default", {}), ("dict", {"PPCG_COL_PAT": "0"}), ("col4", {"PPCG_COL_DICT": "0"})):
            for k in ("PPCG_COL_PAT", "PPCG_COL_DICT"):
                monkeypatch.delenv(k, raising=False)
            for k, v in env.items():
                monkeypatch.setenv(k, v)
            s = m.Solver.from_csr(a, format=2, **kw)
            plan = s.plan()
            xk, ik = s.solve(dev(b), tol=0.0, maxit=25)
            xf, inf = s.solve(dev(b), tol=1e-8, maxit=20000)
            res[mode] = (plan, xk.cpu().numpy(), ik, xf.cpu().numpy(), inf)
            s.close()
        for k in ("PPCG_COL_PAT", "PPCG_COL_DICT"):
            monkeypatch.delenv(k, raising=False)
        p0 = res["default"][0]
        assert p0.columns == want, (name, kw, p0.columns)
        assert res["col4"][0].columns == m.COLS_SELL and res["col4"][0].pattern_k == 0
        if want == m.COLS_PATTERN:
            assert p0.pattern_k in (4, 6) and res["dict"][0].pattern_k == 0
        assert p0.convert_seconds > 0 and p0.create_seconds >= p0.convert_seconds
        for mode in ("dict", "col4"):
            assert res[mode][2].iters == res["default"][2].iters == 25
            assert np.array_equal(res[mode][1], res["default"][1]), (name, kw, mode)
            assert res[mode][4].iters == res["default"][4].iters and res[mode][4].status == m.OK
            assert np.array_equal(res[mode][3], res["default"][3]), (name, kw, mode)
