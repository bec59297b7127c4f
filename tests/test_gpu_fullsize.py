"""Parity at the benchmark's full sizes, in the plans the benchmark times.

The oracle (Alg. 2 of arXiv 2105.06176, Sec. III, plain FP64 C) cannot run these systems to
convergence inside a test, so each one is checked in two ways:
  * x after a fixed k iterations against the oracle run live for k iterations (its OpenMP
    build: the plain build's iterates bit for bit, in a fraction of the time), k the
    calibrated one stored with the golden values;
  * the full solve against the oracle's iteration counts and true residuals stored in
    ``golden/fullsize_oracle.json`` (written by ``golden/make_fullsize_oracle.py``, which
    calls only ``oracle/`` and ``synth/``), with the residual of the returned x recomputed
    here by scipy in FP64.
The workloads: the 256^3 log-normal diffusion system of the main benchmark line (grid path,
default launch shape), the 4M-point random geometric graph (FP64, FP32_RU, FP32_IR), and
the 1024-system ragged batch (one batched launch of cluster-path handles).  GPU only.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_oracle.json")) as _f:
    GOLD = json.load(_f)


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


def true_rel_res(a, b, x):
    return float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b))


def in_envelope(iters, seq, pairwise):
    """The count the oracle fixes: its sequential-sum count and its pairwise-sum count bound
    how far rounding order alone moves it; the GPU's count must lie in that range widened
    by 2 iterations."""
    return min(seq, pairwise) - 2 <= iters <= max(seq, pairwise) + 2


# --------------------------------------------------------- 3-D diffusion, 256^3 (main line) --

@pytest.fixture(scope="module")
def vc256():
    g = GOLD["varcoeff3d_256"]
    a = synth.varcoeff3d(g["grid"], g["matrix_seed"])
    return a, synth.rhs_uniform(a.n, g["rhs_seed"])


def test_varcoeff256_fixed_k_parity(vc256):
    a, b = vc256
    m = pp()
    # at the calibrated k, x_k does not depend on the dot products' summation order beyond
    # 1e-12, so the 1e-10 bar tests the kernel, not rounding order
    g = GOLD["varcoeff3d_256"]
    k = g["fixed_k"]
    assert g["fixed_k_rel_diff_seq_vs_pairwise"] <= 1e-12
    s = m.Solver.from_csr(a)                 # the benchmark's plan: grid path, SELL-C-sigma
    x, info = s.solve(dev(b), tol=0.0, maxit=k)
    s.close()
    assert info.status == m.ERR_NOT_CONVERGED and info.iters == k
    ref = oracle.pipecg(a, b, tol=0.0, maxit=k, openmp=True)["x"]
    assert rel(x.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("precision", [0, 2, 1], ids=["fp64", "fp32_ru", "fp32_ir"])
def test_varcoeff256_full_solve(vc256, precision):
    a, b = vc256
    m = pp()
    g = GOLD["varcoeff3d_256"]
    assert g["status"] == oracle.OK and g["rel_res_true"] <= 1e-8
    s = m.Solver.from_csr(a, precision=precision)
    x, info = s.solve(dev(b), tol=1e-8, maxit=20000)
    s.close()
    x = x.cpu().numpy()
    assert info.status == m.OK, info
    t = true_rel_res(a, b, x)
    assert t <= 1e-8 and abs(t - info.rel_res_true) <= 1e-3 * t
    if precision == 0:
        assert in_envelope(info.iters, g["iters"], g["iters_pairwise"]), (info.iters, g["iters"], g["iters_pairwise"])


# ------------------------------------------------------------- RGG Laplacian, 4M points --

@pytest.fixture(scope="module")
def rgg4m():
    g = GOLD["rgg_4M"]
    npts = g["points"]
    a = synth.rgg_laplacian(npts, (3 * g["degree"] / (4 * np.pi * npts)) ** (1 / 3), g["shift"], g["matrix_seed"])
    return a, synth.rhs_uniform(a.n, g["rhs_seed"])


def test_rgg4m_fixed_k_parity(rgg4m):
    a, b = rgg4m
    m = pp()
    g = GOLD["rgg_4M"]
    k = g["fixed_k"]
    assert g["fixed_k_rel_diff_seq_vs_pairwise"] <= 1e-12
    s = m.Solver.from_csr(a)
    x, info = s.solve(dev(b), tol=0.0, maxit=k)
    s.close()
    assert info.iters == k
    ref = oracle.pipecg(a, b, tol=0.0, maxit=k, openmp=True)["x"]
    assert rel(x.cpu().numpy(), ref) <= 1e-10


def test_rgg4m_full_solves(rgg4m):
    """FP64 to 1e-8 and 1e-10 within +-2 iterations of the oracle; the FP32 forms to 1e-8
    with their error against the FP64 1e-10 solution stated as a bound."""
    a, b = rgg4m
    m = pp()
    g = GOLD["rgg_4M"]
    bd = dev(b)
    sols = {}
    for tol, key in ((1e-8, "1e-08"), (1e-10, "1e-10")):
        assert g[f"status_{key}"] == oracle.OK
        s = m.Solver.from_csr(a)
        x, info = s.solve(bd, tol=tol, maxit=20000)
        s.close()
        x = x.cpu().numpy()
        assert info.status == m.OK, info
        assert in_envelope(info.iters, g[f"iters_{key}"], g[f"iters_pairwise_{key}"]), \
            (tol, info.iters, g[f"iters_{key}"], g[f"iters_pairwise_{key}"])
        assert true_rel_res(a, b, x) <= tol
        sols[key] = x
    for precision in (m.FP32_RU, m.FP32_IR):
        s = m.Solver.from_csr(a, precision=precision)
        x, info = s.solve(bd, tol=1e-8, maxit=20000)
        s.close()
        x = x.cpu().numpy()
        assert info.status == m.OK, info
        assert true_rel_res(a, b, x) <= 1e-8
        # kappa <= (2 * max degree + shift) / shift < 1e5 for this graph, so two solutions
        # with residuals 1e-8 and 1e-10 differ by < 1e-3 relative (measured: ~1e-7)
        assert rel(x, sols["1e-10"]) <= 1e-3


# --------------------------------------------------------------- 1024-system ragged batch --

def test_batch1024_against_oracle_and_solo():
    """The benchmark's batch (1024 systems, 39.1M rows) in one batched launch: every system
    OK with its residual at the bar and its iteration count inside the oracle's envelope
    (its sequential- and pairwise-sum counts, widened by 2), and a sample of the systems
    bitwise equal to their solo solves.  The measured-gap residual replacement, on in the
    library and the oracle alike, is what makes a 2-iteration envelope hold: without it,
    122 of these 2-D log-normal systems replaced their residuals only after the recursive
    one had passed the stopping test, the iteration then drifted into a breakdown, and the
    restart that followed cost a rounding-dependent 0-30% more iterations."""
    m = pp()
    gold = GOLD["batch_1024"]
    specs = synth.batch_mix(gold["count"], gold["seed"])
    systems = [synth.build_spec(sp) for sp in specs]
    solvers = [m.Solver.from_csr(a, path=m.PATH_CLUSTER) for a, _ in systems]
    bs = [dev(b) for _, b in systems]
    xs = [torch.empty_like(b) for b in bs]
    infos = m.batch_solve(solvers, bs, xs, tol=1e-8, maxit=20000)
    off = []
    for k, ((a, b), inf, ref) in enumerate(zip(systems, infos, gold["systems"])):
        assert a.n == ref["n"] and ref["status"] == oracle.OK
        assert inf.status == m.OK, (k, inf)
        assert inf.rel_res_true <= 1e-8, (k, inf.rel_res_true)
        if not in_envelope(inf.iters, ref["iters"], ref["iters_pairwise"]):
            off.append((k, a.n, inf.iters, ref["iters"], ref["iters_pairwise"], inf.rr_count, ref["rr_count"]))
    assert not off, off[:10]
    for k in range(0, len(systems), 61):
        a, b = systems[k]
        x = xs[k].cpu().numpy()
        assert true_rel_res(a, b, x) <= 1e-8, k
        x0, i0 = solvers[k].solve(bs[k], tol=1e-8, maxit=20000)
        assert i0.iters == infos[k].iters and np.array_equal(x0.cpu().numpy(), x), k
    for s in solvers:
        s.close()
