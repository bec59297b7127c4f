"""GPU tests of the three forms beside the plain FP64 solve: FP32 + FP64 iterative
refinement, the batched persistent launch, and the continuous-batching server.

Bars: FP32+IR reaches a true (FP64) relative residual <= 1e-8 and states its error against
the FP64 oracle; batched and served results are bitwise identical to solo ppcg_solve on the
same handle settings (each system's partition over CTAs and reduction order depend only on
the handle), and also meet the oracle bars of the plain solve.
"""
import time

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    """Relative difference of a from b: the larger of the norm-wise ||a - b||_2 / ||b||_2 and
    the element-wise ||a - b||_inf / ||b||_inf, so that one wrong entry cannot hide in the
    norm of a long vector."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = a - b
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), np.max(np.abs(d)) / np.max(np.abs(b))))


def rgg(npts, seed):
    return synth.rgg_laplacian(npts, (3 * 14.0 / (4 * np.pi * npts)) ** (1 / 3), 1e-3, seed)


# ------------------------------------------------------------------ FP32 + refinement ---

@pytest.mark.parametrize("name", ["varcoeff3d_40", "rgg_30k", "poisson2d_64"])
@pytest.mark.parametrize("path", [1, 2], ids=["grid", "cluster"])
def test_fp32_ir_reaches_fp64_accuracy(name, path):
    m = pp()
    if name == "varcoeff3d_40":
        a = synth.varcoeff3d(40, seed=2); b = synth.rhs_uniform(a.n, 2)
    elif name == "rgg_30k":
        a = rgg(30000, 3); b = synth.rhs_uniform(a.n, 3)
    else:
        a = synth.poisson2d(64); b = a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    ref = oracle.pipecg(a, b, tol=1e-10, maxit=50000)
    s = m.Solver.from_csr(a, precision=m.FP32_IR, path=path)
    x, info = s.solve(dev(b), tol=1e-8, maxit=50000)
    x = x.cpu().numpy()
    assert info.status == m.OK, info
    t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert t <= 1e-8 and info.rel_res_true <= 1e-8
    assert info.outer_iters >= 2 and info.fp64_fallback == 0
    err = rel(x, ref["x"])
    # x error is bounded by cond(A) times the residual gap; both solves sit at <= 1e-8
    assert err <= 1e-4, err


def test_fp32_ir_falls_back_to_fp64_when_refinement_stalls():
    """A 2-D log-normal system with kappa near 1/eps32 (1164^2 rows): FP32 inner solves cannot
    reduce the FP64 residual, so the refinement step is undone and the solve finishes with
    the FP64 iteration -- to the same true residual as the plain FP64 solve."""
    m = pp()
    a = synth.varcoeff2d(1164, 77)
    b = dev(synth.rhs_uniform(a.n, 78))
    s = m.Solver.from_csr(a, precision=m.FP32_IR)
    x, info = s.solve(b, tol=1e-8, maxit=200000)
    assert info.status == m.OK, info
    assert info.fp64_fallback == 1
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - a.to_scipy() @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(bn)


# ------------------------------------------------- FP32 with FP64 reliable updates ----

@pytest.mark.parametrize("name", ["varcoeff3d_40", "rgg_30k", "poisson2d_64"])
@pytest.mark.parametrize("path", [1, 2], ids=["grid", "cluster"])
def test_fp32_ru_reaches_fp64_accuracy(name, path):
    """One FP32 Krylov sequence with FP64 reliable updates: true residual <= 1e-8, and (the
    point of keeping the search direction across updates) about the FP64 iteration count."""
    m = pp()
    if name == "varcoeff3d_40":
        a = synth.varcoeff3d(40, seed=2); b = synth.rhs_uniform(a.n, 2)
    elif name == "rgg_30k":
        a = rgg(30000, 3); b = synth.rhs_uniform(a.n, 3)
    else:
        a = synth.poisson2d(64); b = a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    ref = oracle.pipecg(a, b, tol=1e-10, maxit=50000)
    it64 = oracle.pipecg(a, b, tol=1e-8, maxit=50000)["result"]["iters"]
    s = m.Solver.from_csr(a, precision=m.FP32_RU, path=path)
    x, info = s.solve(dev(b), tol=1e-8, maxit=50000)
    x = x.cpu().numpy()
    assert info.status == m.OK, info
    t = np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b)
    assert t <= 1e-8 and info.rel_res_true <= 1e-8
    # rel_res_true is the FP64 residual of the returned x, computed on the device
    assert abs(t - info.rel_res_true) <= 1e-3 * t + 1e-15
    assert info.fp64_fallback == 0 and info.outer_iters >= 2
    assert info.iters <= 1.6 * it64 + 10, (info.iters, it64)
    assert rel(x, ref["x"]) <= 1e-4


def test_fp32_ru_hard_system_finishes_in_fp64_accuracy():
    """kappa near 1/eps32 (2-D log-normal, 1164^2 rows): whether the reliable updates keep the
    FP32 sequence going or the solve falls back to the FP64 iteration, the returned x meets
    the FP64 residual bar."""
    m = pp()
    a = synth.varcoeff2d(1164, 77)
    b = dev(synth.rhs_uniform(a.n, 78))
    s = m.Solver.from_csr(a, precision=m.FP32_RU)
    x, info = s.solve(b, tol=1e-8, maxit=200000)
    assert info.status == m.OK, info
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - a.to_scipy() @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(bn)


def test_fp32_ru_falls_back_when_fp32_cannot_progress():
    """A 1-D Laplacian chain of 8,000 rows (kappa ~ 2.6e7 > 1/eps32): FP32 corrections carry no
    correct digits, so the recursion claims progress that the FP64 residual of the reliable
    updates does not show; after three such updates the solve switches to the FP64 iteration
    and still meets the FP64 residual bar."""
    m = pp()
    import scipy.sparse as sp
    n = 8000
    c = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    a = synth.CSR(n, c.indptr.astype(np.int64), c.indices.astype(np.int32), c.data.astype(np.float64))
    b = synth.rhs_uniform(n, 21)
    s = m.Solver.from_csr(a, precision=m.FP32_RU, path=m.PATH_GRID)
    x, info = s.solve(dev(b), tol=1e-8, maxit=200000)
    assert info.status == m.OK, info
    assert info.fp64_fallback == 1
    assert np.linalg.norm(b - a.to_scipy() @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)


def test_fp32_ru_edge_cases():
    m = pp()
    a = synth.poisson2d(40)
    s = m.Solver.from_csr(a, precision=m.FP32_RU)
    x, info = s.solve(torch.zeros(a.n, dtype=torch.float64, device="cuda"), tol=1e-8, maxit=100)
    assert info.status == m.OK and info.iters == 0 and not x.abs().max().item()
    xt = synth.xtrue_uniform(a.n, 4)
    b = a.to_scipy() @ xt
    x, info = s.solve(dev(b), x0=dev(xt), tol=1e-8, maxit=100)     # exact initial guess
    assert info.status == m.OK and info.iters == 0
    assert np.array_equal(x.cpu().numpy(), xt)
    x, info = s.solve(dev(b), tol=1e-8, maxit=5)                     # maxit: x still written
    assert info.status == m.ERR_NOT_CONVERGED and info.iters == 5
    t = np.linalg.norm(b - a.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
    assert abs(t - info.rel_res_true) <= 1e-6 * t
    with pytest.raises(m.PPCGError):
        m.Solver.from_csr(a, precision=m.FP32_RU, norm=m.NORM_PAPER_U_ABS)


# ------------------------------------------------------------------ batched ------------

def _batch_systems():
    specs = synth.batch_mix(10, 7, lo=1e3, hi=3e4)
    return [synth.build_spec(s) for s in specs]


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp32_ir", "fp32_ru"])
def test_batch_bitwise_equals_solo(precision):
    m = pp()
    systems = _batch_systems()
    solvers, bs = [], []
    for k, (a, b) in enumerate(systems):
        path = m.PATH_GRID if k == 3 else m.PATH_CLUSTER     # one whole-GPU system in the mix
        solvers.append(m.Solver.from_csr(a, precision=precision, path=path))
        bs.append(dev(b))
    solo = []
    for s, b in zip(solvers, bs):
        x, info = s.solve(b, tol=1e-8, maxit=20000)
        solo.append((x.cpu().numpy(), info.iters, info.status))
    xs = [torch.empty_like(b) for b in bs]
    infos = m.batch_solve(solvers, bs, xs, tol=1e-8, maxit=20000)
    for k, ((a, b), (xs0, it0, st0), xb, inf) in enumerate(zip(systems, solo, xs, infos)):
        assert inf.status == st0 == m.OK, (k, inf)
        assert inf.iters == it0, k
        assert np.array_equal(xb.cpu().numpy(), xs0), k
        t = np.linalg.norm(b - a.to_scipy() @ xs0) / np.linalg.norm(b)
        assert t <= 1e-8
    if precision == 0:
        for (a, b), (_, it0, _) in zip(systems[:4], solo[:4]):
            assert abs(it0 - oracle.pipecg(a, b, tol=1e-8, maxit=20000)["result"]["iters"]) <= 2


def test_batch_dynamic_schedule_bitwise_equals_solo():
    """More than two systems per cluster: the clusters take systems from a shared counter, in
    an order that depends on timing; every result is still bitwise the solo result."""
    m = pp()
    specs = synth.batch_mix(400, 23, lo=1e3, hi=6e3)
    systems = [synth.build_spec(sp) for sp in specs]
    solvers = [m.Solver.from_csr(a, path=m.PATH_CLUSTER) for a, _ in systems]
    bs = [dev(b) for _, b in systems]
    xs = [torch.empty_like(b) for b in bs]
    infos = m.batch_solve(solvers, bs, xs, tol=1e-8, maxit=20000)
    for k in range(0, len(systems), 37):
        x0, i0 = solvers[k].solve(bs[k], tol=1e-8, maxit=20000)
        assert infos[k].status == i0.status == m.OK and infos[k].iters == i0.iters
        assert np.array_equal(xs[k].cpu().numpy(), x0.cpu().numpy())
    assert all(i.status == m.OK for i in infos)


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "fp32_ru"])
def test_batch_mixed_cluster_sizes_bitwise_equal_solo(precision):
    """Handles whose plans have different cluster sizes (2, 4, 8, 16 and the create-time
    tuner) in one batch: one launch per size on its own stream; every result is bitwise the
    solo result on the same handle, and the fixed-k iterate matches the oracle."""
    m = pp()
    specs = synth.batch_mix(24, 31, lo=1e3, hi=4e4)
    systems = [synth.build_spec(sp) for sp in specs]
    sizes = [(0, 2, 4, 8, 16)[k % 5] for k in range(len(systems))]
    solvers = [m.Solver.from_csr(a, precision=precision, path=m.PATH_CLUSTER, cluster_ctas=c)
               for (a, _), c in zip(systems, sizes)]
    for s, c in zip(solvers, sizes):
        assert s.plan().ctas in ((2, 4, 8) if c == 0 else (c,))
    bs = [dev(b) for _, b in systems]
    xs = [torch.empty_like(b) for b in bs]
    infos = m.batch_solve(solvers, bs, xs, tol=1e-8, maxit=20000)
    for k, (s, b) in enumerate(zip(solvers, bs)):
        x0, i0 = s.solve(b, tol=1e-8, maxit=20000)
        assert infos[k].status == i0.status == m.OK and infos[k].iters == i0.iters, k
        assert np.array_equal(xs[k].cpu().numpy(), x0.cpu().numpy()), k
    if precision == 0:
        xk = [torch.empty_like(b) for b in bs]
        m.batch_solve(solvers[:6], bs[:6], xk[:6], tol=0.0, maxit=25)
        for (a, b), x in zip(systems[:6], xk[:6]):
            assert rel(x.cpu().numpy(), oracle.pipecg(a, b, tol=0.0, maxit=25)["x"]) <= 1e-10
    with pytest.raises(m.PPCGError):
        m.Solver.from_csr(systems[0][0], path=m.PATH_CLUSTER, cluster_ctas=3)


def test_cluster_size_tuner_picks_small_clusters_for_small_systems():
    """The create-time tuner (cluster_ctas = 0) times 2, 4 and 8 CTAs per system: a
    1,000-row system, bound by its per-iteration barrier and reduction, gets 2; the choice
    is cached, so a second handle of the same family and size is not timed again."""
    m = pp()
    a, _ = synth.build_spec(("varcoeff2d", 32, 5, 6))
    s1 = m.Solver.from_csr(a, path=m.PATH_CLUSTER, cluster_ctas=0)
    s2 = m.Solver.from_csr(a, path=m.PATH_CLUSTER, cluster_ctas=0)
    assert s1.plan().ctas == 2 and s2.plan().ctas == 2
    assert s2.plan().create_seconds <= s1.plan().create_seconds + 0.05
    s1.close()
    s2.close()


def test_batch_fixed_k_parity():
    m = pp()
    systems = _batch_systems()[:6]
    solvers = [m.Solver.from_csr(a, path=m.PATH_CLUSTER) for a, _ in systems]
    bs = [dev(b) for _, b in systems]
    xs = [torch.empty_like(b) for b in bs]
    infos = m.batch_solve(solvers, bs, xs, tol=0.0, maxit=30)
    for (a, b), x, inf in zip(systems, xs, infos):
        assert inf.iters == 30
        assert rel(x.cpu().numpy(), oracle.pipecg(a, b, tol=0.0, maxit=30)["x"]) <= 1e-10


# ------------------------------------------------------------------ server -------------

def _wait(srv, tickets, n_of, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t in out:
                continue
            st, x, info = srv.poll(t, n_of[t])
            if st != pp().PENDING:
                out[t] = (st, x, info)
        time.sleep(0.002)
    assert len(out) == len(tickets), "server did not finish in time"
    return out


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp32_ir", "fp32_ru"])
def test_server_results_same_alone_and_in_mix(precision):
    m = pp()
    systems = _batch_systems()[:6] + [(rgg(40000, 9), synth.rhs_uniform(40000, 9))]
    # alone: one request at a time
    alone = []
    srv = m.Server(precision=precision, epoch_iters=64)
    for a, b in systems:
        t = srv.submit(a, b, tol=1e-8, maxit=20000)
        res = _wait(srv, [t], {t: a.n})[t]
        alone.append(res)
    srv.close()
    # mix: staggered arrivals while earlier requests are resident
    srv = m.Server(precision=precision, epoch_iters=64)
    tickets, n_of = [], {}
    for k, (a, b) in enumerate(systems):
        t = srv.submit(a, b, tol=1e-8, maxit=20000)
        tickets.append(t)
        n_of[t] = a.n
        if k % 2 == 1:
            time.sleep(0.01)
    mix = _wait(srv, tickets, n_of)
    srv.close()
    for (a, b), (st0, x0, i0), t in zip(systems, alone, tickets):
        st1, x1, i1 = mix[t]
        assert st0 == st1 == m.OK, (i0, i1)
        assert i0.iters == i1.iters
        assert np.array_equal(x0, x1)
        r = np.linalg.norm(b - a.to_scipy() @ x1) / np.linalg.norm(b)
        assert r <= 1e-8
    # and the served result equals a solo ppcg_solve with the same settings (the server's
    # plan: the cluster path up to 131,072 rows)
    a, b = systems[0]
    s = m.Solver.from_csr(a, precision=precision, path=m.PATH_CLUSTER)
    xs, info = s.solve(dev(b), tol=1e-8, maxit=20000)
    assert np.array_equal(xs.cpu().numpy(), alone[0][1])


def test_server_large_and_small_requests_admitted_side_by_side():
    """A whole-GPU-path request (216,000 rows, above the cluster path's 131,072) submitted
    together with small ones: the two admission threads take them side by side; every result
    is OK and bitwise the same as the same request served alone, and the HBM accounting
    returns to zero."""
    m = pp()
    big = synth.varcoeff3d(60, seed=12)
    systems = [(big, synth.rhs_uniform(big.n, 12))] + _batch_systems()[:5]
    alone = []
    srv = m.Server(precision=m.FP32_RU, epoch_iters=64)
    for a, b in systems:
        t = srv.submit(a, b, tol=1e-8, maxit=20000)
        alone.append(_wait(srv, [t], {t: a.n})[t])
    srv.close()
    srv = m.Server(precision=m.FP32_RU, epoch_iters=64)
    tickets = [srv.submit(a, b, tol=1e-8, maxit=20000) for a, b in systems]
    mix = _wait(srv, tickets, {t: a.n for t, (a, _) in zip(tickets, systems)})
    assert srv.stats()["hbm_in_use"] == 0 and srv.stats()["completed"] == len(systems)
    srv.close()
    for (a, b), (st0, x0, i0), t in zip(systems, alone, tickets):
        st1, x1, i1 = mix[t]
        assert st0 == st1 == m.OK, (a.n, i0, i1)
        assert i0.iters == i1.iters and np.array_equal(x0, x1), a.n
        assert np.linalg.norm(b - a.to_scipy() @ x1) / np.linalg.norm(b) <= 1e-8


def test_server_keeps_arrival_order_under_memory_pressure():
    """Admission by class: a small request A (long-running) is resident; a large request B
    (above the cluster path's 131,072 rows) does not fit beside A in the budget, a small one
    C would.  B arrived first, so C is not admitted while B waits for memory: as long as A
    runs, one request runs and the other two stay queued.  Then B and C are served."""
    m = pp()

    def footprint(a):      # the library's FP64 admission estimate (ppcg_create's layout)
        slots = 1.05 * a.nnz + 32.0 * (a.n / 32.0 + 1.0)
        return int(slots * 13 + a.n * 48 + a.n * 80) + (1 << 20)
    A, B, C = synth.poisson2d(150), synth.varcoeff3d(52, seed=3), synth.poisson2d(30)
    assert A.n <= 131072 < B.n and C.n <= 131072
    budget = footprint(B) + (2 << 20)
    assert footprint(A) + footprint(B) > budget and footprint(A) + footprint(C) <= budget
    srv = m.Server(hbm_budget=budget, precision=m.FP64, epoch_iters=64)
    ta = srv.submit(A, synth.rhs_uniform(A.n, 1), tol=0.0, maxit=20000)
    tb = srv.submit(B, synth.rhs_uniform(B.n, 2), tol=1e-8, maxit=20000)
    tc = srv.submit(C, synth.rhs_uniform(C.n, 3), tol=1e-8, maxit=20000)
    samples = 0
    t0 = time.time()
    while time.time() - t0 < 120.0:
        st = srv.stats()
        a_st, _, _ = srv.poll(ta, A.n)
        if a_st != m.PENDING:
            break
        # A still runs, so it ran when stats() was taken: B cannot fit, and C may not pass it
        assert st["running"] <= 1, st
        samples += 1
        time.sleep(0.001)
    assert samples > 0
    res = _wait(srv, [tb, tc], {tb: B.n, tc: C.n})
    assert res[tb][0] == m.OK and res[tc][0] == m.OK
    assert srv.stats()["hbm_in_use"] == 0
    srv.close()


def test_injected_allocation_failures_are_reported_and_recovered(monkeypatch):
    """Host-side fault injection (no GPU fault): every device allocation of ppcg_create is
    made to fail in turn; each attempt returns PPCG_ERR_OOM without crashing or leaking into
    later calls, and a clean create + solve afterwards meets the parity bar.  The server
    reports an injected failure as that request's status and serves the next request."""
    m = pp()
    a = synth.varcoeff3d(30, seed=4)
    b = synth.rhs_uniform(a.n, 4)
    failures = 0
    for k in range(1, 40):
        monkeypatch.setenv("PPCG_FAIL_DEVICE_ALLOC", str(k))
        try:
            s = m.Solver.from_csr(a, precision=m.FP32_RU, path=m.PATH_GRID)
        except m.PPCGError as e:
            assert e.status == m.ERR_OOM, str(e)
            failures += 1
            continue
        s.close()
        break
    assert failures >= 5                      # create makes several device allocations
    monkeypatch.delenv("PPCG_FAIL_DEVICE_ALLOC")
    ref = oracle.pipecg(a, b, tol=1e-8, maxit=5000)
    x, info = m.Solver.from_csr(a, path=m.PATH_GRID).solve(dev(b), tol=1e-8, maxit=5000)
    assert info.status == m.OK and abs(info.iters - ref["result"]["iters"]) <= 2
    # server: the admitter's allocation fails for one request only
    srv = m.Server(epoch_iters=64)
    monkeypatch.setenv("PPCG_FAIL_DEVICE_ALLOC", "1")
    t_bad = srv.submit(a, b, tol=1e-8, maxit=5000)
    res = _wait(srv, [t_bad], {t_bad: a.n})
    monkeypatch.delenv("PPCG_FAIL_DEVICE_ALLOC")
    assert res[t_bad][0] == m.ERR_OOM
    t_ok = srv.submit(a, b, tol=1e-8, maxit=5000)
    res = _wait(srv, [t_ok], {t_ok: a.n})
    assert res[t_ok][0] == m.OK
    assert srv.stats()["hbm_in_use"] == 0
    srv.close()


def test_server_admission_by_budget_and_errors():
    m = pp()
    systems = _batch_systems()[:5]

    def footprint(a):      # the library's FP64 admission estimate
        slots = 1.05 * a.nnz + 32.0 * (a.n / 32.0 + 1.0)
        return int(slots * 12 + a.n * 48 + a.n * 80) + (1 << 20)
    # a budget that admits about one request at a time
    srv = m.Server(hbm_budget=int(1.3 * max(footprint(a) for a, _ in systems)), epoch_iters=32)
    tickets, n_of = [], {}
    for a, b in systems:
        t = srv.submit(a, b, tol=1e-8, maxit=20000)
        tickets.append(t)
        n_of[t] = a.n
    st = srv.stats()
    assert st["queued"] + st["running"] + st["completed"] == len(systems)
    res = _wait(srv, tickets, n_of)
    assert all(v[0] == m.OK for v in res.values())
    assert srv.stats()["completed"] == len(systems) and srv.stats()["hbm_in_use"] == 0
    # unknown ticket, too-large request
    st, _, _ = srv.poll(987654321, 1)
    assert st == m.ERR_UNKNOWN_TICKET
    huge = synth.poisson2d(400)
    with pytest.raises(m.PPCGError) as e:
        srv.submit(huge, np.ones(huge.n))
    assert e.value.status == m.ERR_OOM
    srv.close()


def test_last_info_matches_host_function_info():
    """ppcg_last_info after a synchronised solve with info == NULL gives the record that
    ppcg_solve's host function writes into a non-NULL info; before any solve it is refused."""
    m = pp()
    a = synth.varcoeff3d(24, seed=4)
    b = dev(synth.rhs_uniform(a.n, 4))
    for path in (m.PATH_ONCHIP, m.PATH_CLUSTER, m.PATH_GRID):
        s = m.Solver.from_csr(a, path=path)
        with pytest.raises(m.PPCGError):
            s.last_info()
        x1, i1 = s.solve(b, tol=1e-8, maxit=5000, sync=False)        # host-function info
        torch.cuda.synchronize()
        x2, i2 = s.solve(b, tol=1e-8, maxit=5000, sync=True)         # info read after the sync
        assert i2.status == i1.status == m.OK
        for f in ("iters", "outer_iters", "rr_count", "rel_res_recursive", "rel_res_true", "bnorm",
                  "bytes_per_iter", "fp64_fallback"):
            assert getattr(i1, f) == getattr(i2, f), f
        assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
        x3, i3 = s.solve(b, tol=0.0, maxit=7, sync=False, host_fn_info=False)
        assert i3 is None
        torch.cuda.synchronize()
        i4 = s.last_info()
        assert i4.status == m.ERR_NOT_CONVERGED and i4.iters == 7
        s.close()
