#!/usr/bin/env python3
"""Benchmark: pipelined PCG (Alg. 2, Jacobi) on one B300 per rank.

One step = one full solve of the 3-D 7-point variable-coefficient diffusion system on a
256^3 grid (N = 16,777,216, nnz = 117,047,296; face coefficients exp(N(0,1)); b ~ U[-1,1];
x0 = 0; relative tolerance 1e-8; FP64) through the C ABI: setup, every iteration and the
final true residual, all inside the library's persistent kernel.

Printed (rank 0, one JSON line): iterations/s over all ranks (value), end-to-end
iterations/s through host buffers (e2e), the roofline of the solve kernel against the
measured HBM copy bandwidth (with the DRAM traffic of the committed ncu capture), SM clocks
sampled during the timed region, the FP32 forms (reliable updates; inner solves in FP64
refinement) and the Jacobi-scaled variant against FP64 in time to 1e-8 on the same system,
the 64^2 solve latency, the 1024-system batch (FP64 and FP32_RU against sequential FP64), a
serving slice over 1e3-4e6 rows at two offered rates, the create (conversion) time, and the
CPU oracle (single-thread and OpenMP builds) timed on a bounded sample.

Multi-GPU: replicas only.  Each rank solves its own copy; value = all ranks' iterations /
the slowest rank's time ("scaling": "weak").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --mode batch|serve|rgg|paper|box125|latency   (one workload's figures)
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pipelined-PCG iter/s, % HBM peak; mixed vs FP64 at 1e-8; p50/p99 solve latency"
UNIT = "iter/s"
GRID_N = 256
SEED = 1
TOL = 1e-8
MAXIT = 20000
SERVE_MAXIT = 200000       # served requests include 2-D stencils of up to 4e6 rows (kappa ~1e7)
def workload(g, n, nnz):
    return (f"3D 7-point variable-coefficient diffusion {g}^3 (N={n:,}, nnz={nnz:,}), "
            "log-normal(0,1) face coefficients, Jacobi, b~U[-1,1], x0=0, rel tol 1e-8, FP64 pipelined PCG")


def b_alg(n, nnz, v):
    """Algorithmic bytes of one iteration: SELL values + int32 columns, row pointers, and
    17 vector streams (w gather once; invd z q s p x r u read; z q s p x r u w written)."""
    return (v + 4) * nnz + 4 * (n + 1) + 17 * v * n


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for ln in f:
                    parts = [t.strip() for t in ln.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = sorted(sm)[len(sm) // 4:] if len(sm) >= 4 else sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": reasons, "samples": len(rows)}


def profiled_traffic(bytes_iter, iters_per_launch):
    """DRAM bytes per launch from the committed ncu capture of the solve kernel on this
    workload (the capture's bytes per iteration times this launch's iterations); None once
    the kernel source has changed since the capture, or for another grid size (the L2 serves
    a roughly fixed amount per pass, so traffic does not scale with the algorithmic bytes)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_grid_traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, "paper_2105_06176_b300", "csrc", "solver.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None, "no capture"
    if rec.get("kernel_source_sha256") != sha:
        return None, "kernel changed since the last capture"
    if rec.get("b_alg_per_iter") != bytes_iter:
        return None, "captured on another grid size"
    return rec["dram_bytes_per_launch"] / rec["iterations"] * iters_per_launch, \
        f"ncu capture: {rec['workload']}"


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(dist, device, times, counts):
    """Whole-job figures of a multi-rank run: the maximum over ranks of each time and the sum
    over ranks of each count (every rank calls it with lists of the same length)."""
    import torch
    t = torch.tensor(times, dtype=torch.float64, device=device)
    c = torch.tensor(counts, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def cpu_oracle_rate(a, b, k_lo=2, k_hi=8):
    """Oracle (plain single-thread C, FP64) iterations/s on the same system: the time of
    k_hi - k_lo iterations, from two runs that share setup and final-residual costs.  The
    same source built with OpenMP (row loops on every host core, dot products sequential,
    bitwise-identical iterates) is timed the same way and reported beside it."""
    import oracle

    def rate(openmp):
        oracle.lib(openmp)
        t0 = time.perf_counter()
        oracle.pipecg(a, b, tol=0.0, maxit=k_lo, openmp=openmp)
        t1 = time.perf_counter()
        oracle.pipecg(a, b, tol=0.0, maxit=k_hi, openmp=openmp)
        t2 = time.perf_counter()
        return 1.0 / (max((t2 - t1) - (t1 - t0), 1e-9) / (k_hi - k_lo)), t2 - t0

    v1, s1 = rate(False)
    vo, so = rate(True)
    return {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k_hi - k_lo} iterations of the 256^3 system (difference of {k_hi}- and {k_lo}-iteration "
                      f"runs), single-thread plain C, {os.cpu_count()} host cores present",
            "seconds": s1,
            "openmp": {"value": vo, "unit": UNIT, "cores": oracle.threads(openmp=True), "kind": "oracle",
                       "sample": "the same iterations, the same source built with -fopenmp (row loops "
                                 "threaded, dot products sequential)", "seconds": so}}


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_latency_2d(pp, torch):
    """64x64 2-D Poisson (N = 4,096), b = A x_true: solve latency and time per iteration
    on the default path (on chip: the system in one cluster's shared memory), the cluster
    path with vectors in global memory, and the whole-GPU path.  Latency = CUDA events
    around ppcg_solve with the result record read after the synchronisation
    (ppcg_last_info); the same with the info-filling host function on the stream is
    reported beside it."""
    a = synth.poisson2d(64)
    b = torch.from_numpy(a.to_scipy() @ synth.xtrue_uniform(a.n, 1)).cuda()
    out = {"workload": "2D 5-point Poisson 64x64, FP64, rel tol 1e-8"}
    for name, path in (("onchip", pp.PATH_ONCHIP), ("cluster", pp.PATH_CLUSTER), ("grid", pp.PATH_GRID)):
        s = pp.Solver.from_csr(a, path=path)
        x = torch.empty_like(b)
        for _ in range(3):
            s.solve(b, None, x, tol=TOL, maxit=MAXIT)
        ts, th = [], []
        for _ in range(20):
            # info read after the synchronisation (ppcg_last_info): no host function on the stream
            e0, e1 = _events()
            e0.record()
            s.solve(b, None, x, tol=TOL, maxit=MAXIT, sync=False, host_fn_info=False)
            e1.record()
            torch.cuda.synchronize()
            info = s.last_info()
            ts.append(e0.elapsed_time(e1) * 1e3)
            # info filled by the host function ppcg_solve enqueues
            e0, e1 = _events()
            e0.record()
            _, info_h = s.solve(b, None, x, tol=TOL, maxit=MAXIT, sync=False)
            e1.record()
            torch.cuda.synchronize()
            th.append(e0.elapsed_time(e1) * 1e3)
        assert info.iters == info_h.iters and info.status == info_h.status == pp.OK
        out[name] = {"solve_us_p50": float(np.median(ts)), "iters": info.iters,
                     "us_per_iter": float(np.median(ts)) / max(info.iters, 1),
                     "rel_res_true": info.rel_res_true,
                     "solve_us_p50_info_by_host_fn": float(np.median(th))}
        s.close()
    return out


def measure_batch(pp, torch, count, seed=11, precisions=(0,)):
    """Ragged batch (sizes log-uniform 1e3-2e5, half 2-D / half 3-D log-normal stencils), to
    rel 1e-8: one ppcg_batch_solve of CLUSTER-path handles per precision, against `count`
    sequential ppcg_solve calls of default-plan FP64 handles (the plain solver)."""
    specs = synth.batch_mix(count, seed)
    systems = [synth.build_spec(sp) for sp in specs]
    rows = sum(a.n for a, _ in systems)
    bs = [torch.from_numpy(b).cuda() for _, b in systems]
    xs = [torch.empty_like(b) for b in bs]
    seq = [pp.Solver.from_csr(a) for a, _ in systems]
    # warm-up (first launches of each kernel shape)
    seq[0].solve(bs[0], None, xs[0], tol=TOL, maxit=MAXIT)
    e0, e1 = _events()
    e0.record()
    infos_seq = [s.solve(b, None, x, tol=TOL, maxit=MAXIT, sync=False)[1] for s, b, x in zip(seq, bs, xs)]
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) * 1e-3
    seq_ok = all(i.status == pp.OK for i in infos_seq)
    for s in seq:
        s.close()
    out = {"systems": count, "rows": rows, "sequential_fp64_s": t_seq, "sequential_all_ok": seq_ok}
    for precision in precisions:
        name = ("fp64", "fp32_ir", "fp32_ru")[precision]
        bat = [pp.Solver.from_csr(a, precision=precision, path=pp.PATH_CLUSTER) for a, _ in systems]
        pp.batch_solve(bat[:2], bs[:2], xs[:2], tol=TOL, maxit=MAXIT)
        e0, e1 = _events()
        e0.record()
        infos = pp.batch_solve(bat, bs, xs, tol=TOL, maxit=MAXIT, sync=False)
        e1.record()
        torch.cuda.synchronize()
        t_bat = e0.elapsed_time(e1) * 1e-3
        bad = [{"n": a.n, "status": pp.status_name(j.status), "iters": j.iters}
               for (a, _), j in zip(systems, infos) if j.status != pp.OK][:8]
        out[name] = {"batched_s": t_bat, "speedup_vs_sequential_fp64": t_seq / t_bat,
                     "all_ok": not bad, "not_ok": bad, "iters_total": sum(i.iters for i in infos),
                     "row_iters_per_s": sum(i.iters * a.n for i, (a, _) in zip(infos, systems)) / t_bat}
        for s in bat:
            s.close()
    return out


def measure_tuned_batch(pp, torch, count=1024, lo=1e3, hi=3e3, seed=23):
    """1024 small ragged systems (1e3-3e3 rows, half 2-D / half 3-D log-normal stencils), to
    rel 1e-8, in one batched launch of CLUSTER-path handles: the default plan (8 CTAs per
    system) against the create-time tuned plan (cluster_ctas = 0), FP64 and FP32_RU."""
    specs = synth.batch_mix(count, seed, lo=lo, hi=hi)
    systems = [synth.build_spec(sp) for sp in specs]
    bs = [torch.from_numpy(b).cuda() for _, b in systems]
    xs = [torch.empty_like(b) for b in bs]
    out = {"systems": count, "size_range": [lo, hi]}
    for precision, pname in ((pp.FP64, "fp64"), (pp.FP32_RU, "fp32_ru")):
        rec = {}
        for label, cc in (("fixed_8", 8), ("tuned", 0)):
            hs = [pp.Solver.from_csr(a, precision=precision, path=pp.PATH_CLUSTER, cluster_ctas=cc)
                  for a, _ in systems]
            pp.batch_solve(hs[:2], bs[:2], xs[:2], tol=TOL, maxit=MAXIT)
            ts = []
            for _ in range(2):
                e0, e1 = _events()
                e0.record()
                infos = pp.batch_solve(hs, bs, xs, tol=TOL, maxit=MAXIT, sync=False)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
            sizes = {}
            for h in hs:
                c = h.plan().ctas
                sizes[str(c)] = sizes.get(str(c), 0) + 1
            rec[label] = {"s": min(ts), "ctas_per_system": sizes, "all_ok": all(i.status == pp.OK for i in infos)}
            for h in hs:
                h.close()
        rec["tuned_speedup"] = rec["fixed_8"]["s"] / rec["tuned"]["s"]
        out[pname] = rec
    return out


def _serving_pool(seed, count, hi, buckets=24):
    """Request stream: sizes log-uniform [1e3, hi] over {2-D, 3-D var-coeff, RGG}.  Sizes are
    snapped to `buckets` log-spaced values so each (family, size) matrix is built once;
    every request gets its own right-hand side."""
    specs = synth.serving_mix(count, seed, hi=hi)
    grid = np.exp(np.linspace(np.log(1e3), np.log(hi), buckets))
    built = {}
    reqs = []
    for k, (fam, size, _, _) in enumerate(specs):
        rows = size * size if fam == "varcoeff2d" else size ** 3 if fam == "varcoeff3d" else size
        rb = grid[np.argmin(np.abs(np.log(grid) - np.log(rows)))]
        if fam == "varcoeff2d":
            size = max(2, int(round(np.sqrt(rb))))
        elif fam == "varcoeff3d":
            size = max(2, int(round(np.cbrt(rb))))
        else:
            size = int(round(rb))
        key = (fam, size)
        if key not in built:
            built[key] = synth.build_spec((fam, size, 7919 * len(built) + seed, 0))[0]
        a = built[key]
        reqs.append((a, synth.rhs_uniform(a.n, 100000 + k)))
    return reqs


def run_server(pp, reqs, arrivals, precision=2, epoch_iters=128):
    """Submit reqs at the given arrival offsets (s); poll until all finish.  Returns
    (latencies, wall seconds, statuses)."""
    srv = pp.Server(precision=precision, epoch_iters=epoch_iters)
    t0 = time.perf_counter()
    pending = {}
    lat = [None] * len(reqs)
    status = [None] * len(reqs)
    infos = [None] * len(reqs)
    k = 0
    while k < len(reqs) or pending:
        now = time.perf_counter() - t0
        while k < len(reqs) and arrivals[k] <= now:
            a, b = reqs[k]
            pending[srv.submit(a, b, tol=TOL, maxit=SERVE_MAXIT)] = (k, a.n, t0 + arrivals[k])
            k += 1
        for t in list(pending):
            st, _, info = srv.poll(t, pending[t][1])
            if st != pp.PENDING:
                i, _, ta = pending.pop(t)
                lat[i] = time.perf_counter() - ta
                status[i] = st
                infos[i] = info
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    srv.close()
    run_server.last_infos = infos
    return lat, wall, status


def measure_serving(pp, nreq=160, hi=2e5, seed=5, rate_factors=(0.5,), buckets=24):
    """Continuous batching: saturation throughput (all requests at t = 0), then Poisson
    arrivals at rate_factor x saturation; p50/p99 latency = poll-visible completion - arrival."""
    reqs = _serving_pool(seed, nreq, hi, buckets)
    run_server(pp, reqs[:8], [0.0] * 8)                       # warm-up
    lat, wall, st = run_server(pp, reqs, [0.0] * len(reqs))
    sat = len(reqs) / wall
    # the plain FP64 solver on the same stream, one request after another: create from the
    # host CSR, solve, read x back (what the server does per request, without overlap)
    t0 = time.perf_counter()
    seq_ok = True
    for a, b in reqs:
        s = pp.Solver.from_csr(a)
        x, info = s.solve(b, tol=TOL, maxit=SERVE_MAXIT)
        seq_ok &= info.status == pp.OK
        s.close()
    seq = len(reqs) / (time.perf_counter() - t0)
    print(json.dumps({"progress": {"saturation_solves_per_s": sat, "sequential_fp64_solves_per_s": seq}}),
          file=sys.stderr, flush=True)
    out = {"requests": nreq, "size_range": [1e3, hi], "size_buckets_per_family": buckets,
           "largest_rows": max(a.n for a, _ in reqs), "precision": "fp32_ru", "saturation_solves_per_s": sat,
           "sequential_fp64_solves_per_s": seq, "speedup_vs_sequential_fp64": sat / seq,
           "all_ok": all(s == pp.OK for s in st) and seq_ok, "rates": []}
    rng = np.random.default_rng(seed)
    for f in rate_factors:
        rate = f * sat
        arr = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
        arr -= arr[0]
        lat, wall, st = run_server(pp, reqs, arr)
        entry = {"rate_factor": f, "offered_per_s": rate, "solves_per_s": len(reqs) / wall,
                 "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                 "all_ok": all(s == pp.OK for s in st)}
        # the same split by the path the server gives a request: up to 131,072 rows on
        # thread-block clusters (all advance in every epoch), larger ones on the whole GPU
        lat_a, rows = np.asarray(lat), np.array([a.n for a, _ in reqs])
        for key, sel in (("cluster_path_requests", rows <= 131072), ("grid_path_requests", rows > 131072)):
            if sel.any():
                entry[key] = {"count": int(sel.sum()), "p50_s": float(np.percentile(lat_a[sel], 50)),
                              "p99_s": float(np.percentile(lat_a[sel], 99))}
        out["rates"].append(entry)
        print(json.dumps({"progress": out["rates"][-1]}), file=sys.stderr, flush=True)
    return out


def measure_rgg(pp, torch, npts=4_000_000, seed=3, profile_iters=0):
    """Random geometric graph Laplacian (expected degree 14) + 1e-3 I: FP32_RU and FP32_IR to
    1e-8 and FP64 to 1e-8 and 1e-10, time to solution and each result's error against the
    FP64 1e-10 solution.  profile_iters > 0: a single FP64 solve stopped after that many
    iterations instead (one short launch of the solve kernel for a profiler)."""
    radius = (3 * 14.0 / (4 * np.pi * npts)) ** (1 / 3)
    a = synth.rgg_laplacian(npts, radius, 1e-3, seed)
    b = torch.from_numpy(synth.rhs_uniform(a.n, seed)).cuda()
    out = {"workload": f"RGG Laplacian {npts} points, radius {radius:.6f}, shift 1e-3", "N": a.n, "nnz": a.nnz}
    if profile_iters > 0:
        s = pp.Solver.from_csr(a)
        _, info = s.solve(b, None, None, tol=1e-8, maxit=profile_iters)
        s.close()
        out["profile_solve"] = {"iters": info.iters, "status": pp.status_name(info.status),
                                "kernel_s": info.seconds}
        return out
    runs = {}
    for name, prec, tol in (("fp64_1e-10", pp.FP64, 1e-10), ("fp64_1e-8", pp.FP64, 1e-8),
                            ("fp32_ru_1e-8", pp.FP32_RU, 1e-8), ("fp32_ir_1e-8", pp.FP32_IR, 1e-8)):
        s = pp.Solver.from_csr(a, precision=prec)
        x = torch.empty_like(b)
        s.solve(b, None, x, tol=tol, maxit=MAXIT)
        e0, e1 = _events()
        e0.record()
        _, info = s.solve(b, None, x, tol=tol, maxit=MAXIT, sync=False)
        e1.record()
        torch.cuda.synchronize()
        runs[name] = (x.clone(), info, e0.elapsed_time(e1) * 1e-3)
        s.close()
    ref = runs["fp64_1e-10"][0]
    peaks, _ = measured_peaks()
    for name, (x, info, t) in runs.items():
        # algorithmic bytes (B_alg of the iteration's precision, SELL padding not counted)
        gbs = info.bytes_per_iter * info.iters / t / 1e9
        out[name] = {"s": t, "iters": info.iters, "outer": info.outer_iters, "status": pp.status_name(info.status),
                     "rel_res_true": info.rel_res_true, "iters_per_s": info.iters / t,
                     "bytes_per_iter": info.bytes_per_iter, "achieved_gbs": gbs,
                     "frac_of_measured_hbm": gbs / peaks["hbm_gbs"],
                     "err_vs_fp64_1e-10": (torch.linalg.norm(x - ref) / torch.linalg.norm(ref)).item()}
    out["fp32_ru_speedup_vs_fp64_1e-8"] = runs["fp64_1e-8"][2] / runs["fp32_ru_1e-8"][2]
    out["fp32_ir_speedup_vs_fp64_1e-8"] = runs["fp64_1e-8"][2] / runs["fp32_ir_1e-8"][2]
    return out


def measure_paper(pp, torch, batch_count=1024):
    """The paper's own experimental setting (Sec. VI): stop when sqrt((u, u)) <= 1e-5
    (absolute, preconditioned), maxit 10000, exact solution x = 1/sqrt(N) (b = A x), x0 = 0,
    FP64 -- on the 2-D 64^2 Poisson system, the 256^3 diffusion system, the 4M-point RGG
    Laplacian and the ragged batch."""
    def one(a, label):
        xe = np.full(a.n, 1.0 / np.sqrt(a.n))
        b = torch.from_numpy(a.to_scipy() @ xe).cuda()
        s = pp.Solver.from_csr(a, norm=pp.NORM_PAPER_U_ABS)
        x = torch.empty_like(b)
        s.solve(b, None, x, tol=1e-5, maxit=10000)
        e0, e1 = _events()
        e0.record()
        _, info = s.solve(b, None, x, tol=1e-5, maxit=10000, sync=False)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        err = float(np.linalg.norm(x.cpu().numpy() - xe) / np.linalg.norm(xe))
        s.close()
        return {"workload": label, "N": a.n, "nnz": a.nnz, "iters": info.iters, "s": t,
                "iters_per_s": info.iters / t, "status": pp.status_name(info.status),
                "u_norm_at_exit": info.rel_res_recursive, "rel_res_true": info.rel_res_true,
                "err_vs_exact": err}
    out = {"setting": "sqrt((u,u)) <= 1e-5 absolute, maxit 10000, x_exact = 1/sqrt(N), x0 = 0, FP64"}
    out["poisson2d_64"] = one(synth.poisson2d(64), "2D 5-point Poisson 64x64")
    out["varcoeff3d_256"] = one(synth.varcoeff3d(GRID_N, SEED), "3D 7-point log-normal diffusion 256^3")
    npts = 4_000_000
    out["rgg_4M"] = one(synth.rgg_laplacian(npts, (3 * 14.0 / (4 * np.pi * npts)) ** (1 / 3), 1e-3, 3),
                        "RGG Laplacian 4M points + 1e-3 I")
    systems = [synth.build_spec(sp)[0] for sp in synth.batch_mix(batch_count, 11)]
    hs = [pp.Solver.from_csr(a, norm=pp.NORM_PAPER_U_ABS, path=pp.PATH_CLUSTER) for a in systems]
    xes = [np.full(a.n, 1.0 / np.sqrt(a.n)) for a in systems]
    bs = [torch.from_numpy(a.to_scipy() @ xe).cuda() for a, xe in zip(systems, xes)]
    xs = [torch.empty_like(b) for b in bs]
    pp.batch_solve(hs[:2], bs[:2], xs[:2], tol=1e-5, maxit=10000)
    e0, e1 = _events()
    e0.record()
    infos = pp.batch_solve(hs, bs, xs, tol=1e-5, maxit=10000, sync=False)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    errs = [float(np.linalg.norm(x.cpu().numpy() - xe) / np.linalg.norm(xe)) for x, xe in zip(xs, xes)]
    out["batch"] = {"systems": batch_count, "rows": sum(a.n for a in systems), "s": t,
                    "iters_total": sum(i.iters for i in infos), "all_ok": all(i.status == pp.OK for i in infos),
                    "err_vs_exact_max": max(errs), "err_vs_exact_median": float(np.median(errs))}
    for h in hs:
        h.close()
    return out


def measure_box125(pp, torch, sizes=(165, 170, 181, 185), seed=9):
    """Table II's 125-point box-stencil Poisson family (diag 124, off -1; N = n^3, nnz =
    (5n - 6)^3, 549M-776M nonzeros): the SpMV-dominated regime.  FP64 with the SELL matrix,
    FP64 matrix-free (axis-wise box sums, no matrix stream) and FP32_RU with the SELL matrix,
    to rel 1e-8 from b ~ U[-1, 1]; iterations/s and GB/s against the measured HBM peak."""
    peaks, _ = measured_peaks()
    out = {"workload": "125-point box stencil n^3 (Table II sizes), diag 124, off -1, b~U[-1,1], x0=0, rel tol 1e-8",
           "runs": []}
    for n in sizes:
        t0 = time.perf_counter()
        a = synth.box125(n)
        t_gen = time.perf_counter() - t0
        b = torch.from_numpy(synth.rhs_uniform(a.n, seed)).cuda()
        rec = {"n": n, "N": a.n, "nnz": a.nnz, "gen_s": t_gen}
        x64 = None
        for name, prec, fmt in (("fp64", pp.FP64, pp.FMT_SELL), ("fp64_matrix_free", pp.FP64, pp.FMT_BOX),
                                ("fp32_ru", pp.FP32_RU, pp.FMT_SELL)):
            t0 = time.perf_counter()
            s = pp.Solver.from_csr(a, precision=prec, format=fmt, path=pp.PATH_GRID)
            torch.cuda.synchronize()
            t_create = time.perf_counter() - t0
            x = torch.empty_like(b)
            s.solve(b, None, x, tol=TOL, maxit=3)                  # first launch
            e0, e1 = _events()
            e0.record()
            _, info = s.solve(b, None, x, tol=TOL, maxit=MAXIT, sync=False)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            # bytes per iteration: B_alg for the SELL plans; 21 v N (17 vector streams and the
            # two stage arrays) for the matrix-free plan (info.bytes_per_iter is the library's)
            balg = info.bytes_per_iter
            r = {"s": t, "iters": info.iters, "iters_per_s": info.iters / t, "status": pp.status_name(info.status),
                 "rel_res_true": info.rel_res_true, "create_s": t_create, "bytes_per_iter": balg,
                 "achieved_gbs": balg * info.iters / t / 1e9}
            r["frac_of_measured_hbm"] = r["achieved_gbs"] / peaks["hbm_gbs"]
            if fmt == pp.FMT_BOX:
                # The matrix-free passes are bound by the FP64 pipe: per interior row and
                # iteration 2R adds for the x-sums, 2 + 2 for the marching y- and z-sums and
                # 13 for the update and the two dots (the optional norm dot not counted).
                # Peak: the nominal 1.25 TFLOP/s FP64 rate counts an FMA as two flops, so the
                # pipe retires 0.625 T FP64 operations per second (an add or a multiply
                # takes an FMA's slot).
                ops = (2 * 2 + 4 + 13) * a.n
                r["fp64_ops_per_iter"] = ops
                r["fp64_tops"] = ops * info.iters / t / 1e12
                r["frac_of_fp64_pipe_nominal"] = r["fp64_tops"] / 0.625
            if name == "fp64":
                x64 = x.clone()
            else:
                r["speedup_vs_fp64_sell"] = rec["fp64"]["s"] / t
                r["err_vs_fp64_solution"] = (torch.linalg.norm(x - x64) / torch.linalg.norm(x64)).item()
            rec[name] = r
            s.close()
            del x
        out["runs"].append(rec)
        del a, b, x64
    return out


def run_reference(args, ws, rank):
    """Reference arm: the oracle, as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    a = synth.varcoeff3d(args.grid, SEED)
    b = synth.rhs_uniform(a.n, SEED)
    oracle.lib()
    k = 3
    for _ in range(args.warmup):
        oracle.pipecg(a, b, tol=0.0, maxit=1)
    t0 = time.perf_counter()
    iters = 0
    for _ in range(args.steps):
        out = oracle.pipecg(a, b, tol=0.0, maxit=k)
        iters += out["result"]["iters"]
    dt = time.perf_counter() - t0
    val = iters / dt
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload(args.grid, a.n, a.nnz), "sample": f"{k} iterations per step incl. setup and final residual"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{k} iterations of the {args.grid}^3 system per step, including setup "
                                       f"(3 SpMV) and the final residual, single-thread plain C"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=GRID_N, help="grid side (256 = the benchmark workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the latency, batch and serving figures")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_ru", "fp32_ir"],
                    help="precision of the main line's timed solver (the headline is fp64; the "
                         "others exist to profile the FP32 kernels on the same workload)")
    ap.add_argument("--mode", default="main",
                    choices=["main", "batch", "serve", "rgg", "paper", "box125", "latency"],
                    help="batch: the 1024-system ragged batch; serve: the serving rate sweep; "
                         "rgg: FP32 forms vs FP64 on the 4M-point random geometric graph; "
                         "paper: the paper's stopping rule and exact solution on every config; "
                         "box125: Table II's 125-point family; latency: the 64^2 solve latency")
    ap.add_argument("--batch-count", type=int, default=1024)
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="rgg mode: one FP64 solve stopped after this many iterations (a short "
                         "kernel launch to capture with a profiler) instead of the figures")
    ap.add_argument("--box-sizes", type=int, nargs="+", default=[165, 170, 181, 185],
                    help="grid sides of the box125 mode (default: Table II's four)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.mode != "main":
        import torch
        import paper_2105_06176_b300 as pp
        torch.cuda.set_device(local)
        if args.mode == "rgg":
            res = {"mode": "rgg", "rgg": measure_rgg(pp, torch, profile_iters=args.profile_iters)}
        elif args.mode == "box125":
            res = {"mode": "box125", "box125": measure_box125(pp, torch, sizes=tuple(args.box_sizes))}
        elif args.mode == "paper":
            res = {"mode": "paper", "paper": measure_paper(pp, torch, args.batch_count)}
        elif args.mode == "latency":
            res = {"mode": "latency", "latency_2d64": measure_latency_2d(pp, torch)}
        elif args.mode == "batch":
            res = {"mode": "batch", "batch": measure_batch(pp, torch, args.batch_count,
                                                           precisions=(pp.FP64, pp.FP32_RU))}
        else:
            res = {"mode": "serve", "serving": measure_serving(pp, nreq=2000, hi=4e6,
                                                               rate_factors=(0.25, 0.5, 1.0, 2.0, 4.0))}
        if rank == 0:
            print(json.dumps(res), flush=True)
        return

    import torch
    import paper_2105_06176_b300 as pp
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    def barrier():
        if pg:
            pg.barrier()

    a = synth.varcoeff3d(args.grid, SEED)
    b = synth.rhs_uniform(a.n, SEED)
    n, nnz = a.n, a.nnz
    prec = {"fp64": pp.FP64, "fp32_ru": pp.FP32_RU, "fp32_ir": pp.FP32_IR}[args.precision]
    solver = pp.Solver.from_csr(a, precision=prec)
    plan = solver.plan()
    b_d = torch.from_numpy(b).cuda()
    x_d = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        _, info = solver.solve(b_d, None, x_d, tol=TOL, maxit=MAXIT)
    assert info.status == pp.OK, info
    iters_per_solve = info.iters

    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.steps):
            step_ev[k][0].record(stream)
            _, info = solver.solve(b_d, None, x_d, tol=TOL, maxit=MAXIT, sync=False)
            step_ev[k][1].record(stream)
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    clocks = clk.summary()
    dt = ev0.elapsed_time(ev1) * 1e-3
    iters = sum(i.iters for i in infos)
    assert all(i.status == pp.OK for i in infos), [i.status for i in infos]
    step_s = [s.elapsed_time(e) * 1e-3 for s, e in step_ev]
    if pg:
        (dt_max,), (iters_all,) = reduce_over_ranks(pg, "cuda", [dt], [float(iters)])
    else:
        dt_max, iters_all = dt, float(iters)
    value = iters_all / dt_max

    # end to end through the C ABI with pinned host buffers: H2D of b, D2H of x inside each step
    b_h = torch.from_numpy(b).pin_memory()
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    solver.solve(b_h, None, x_h, tol=TOL, maxit=MAXIT)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_iters = 0
    for _ in range(args.steps):
        _, info = solver.solve(b_h, None, x_h, tol=TOL, maxit=MAXIT, sync=True)
        e_iters += info.iters
    e_dt = time.perf_counter() - t0
    barrier()
    e2e = {"value": e_iters / e_dt, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}
    if pg:
        (e_dt_max,), (e_iters_all,) = reduce_over_ranks(pg, "cuda", [e_dt], [float(e_iters)])
        e2e["value"] = e_iters_all / e_dt_max

    # roofline of the solve kernel (one launch = one step)
    peaks, peak_kind = measured_peaks()
    # (FP32 modes: B_alg of an FP32 iteration; the FP64 reliable updates are not counted)
    bytes_iter = b_alg(n, nnz, 8 if prec == pp.FP64 else 4)
    per_launch_s = float(np.mean(step_s))
    achieved = bytes_iter * (iters / len(infos)) / per_launch_s / 1e9
    kernel_s = float(np.mean([i.seconds for i in infos]))
    if prec == pp.FP64:
        traffic, traffic_src = profiled_traffic(bytes_iter, iters / len(infos))
    else:
        traffic, traffic_src = None, "captured for the FP64 solve only"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": traffic_src,
                "peak_kind": peak_kind,
                "kernel": "k_grid (persistent solve: setup + iterations + final residual)",
                "bytes_per_iter": bytes_iter, "iters_per_launch": iters / len(infos),
                "launch_ms": 1e3 * per_launch_s, "device_timer_ms": 1e3 * kernel_s,
                "frac_of_8TBs_nominal": achieved / 8000.0}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == pp.FP64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload(args.grid, n, nnz), "grid": args.grid, "N": n, "nnz": nnz,
                       "precision": args.precision,
                       "iters_per_solve": iters_per_solve, "format": "SELL-C-sigma C=32",
                       "path": "grid (cooperative persistent kernel)",
                       "l2": f"inputs larger than L2 ({bytes_iter / 1e9:.2f} GB streamed per iteration vs 126 MB L2)",
                       "parallelism": f"replicas x{ws}"},
            "e2e": e2e, "roofline": roofline, "clocks": clocks,
            # ppcg_create of the timed handle (host CSR upload, validation, CSR -> device
            # layout conversion, detection, workspace): paid once per matrix
            "create_s": plan.create_seconds,
            "plan": {"columns": ("sell", "sell+dictionary", "offset pattern", "matrix-free")[plan.columns],
                     "pattern_k": plan.pattern_k, "sigma": plan.sigma, "ctas": plan.ctas,
                     "padding": plan.padding, "convert_s": plan.convert_seconds},
            "gpu_launches": 4 * args.steps}   # per solve: x0 fill, control init, k_grid, x copy-out

    if not args.no_mixed:
        # FP32 recurrences with FP64 reliable updates (the mixed-precision form), and FP32
        # inner solves inside FP64 iterative refinement, against the FP64 solve above
        line["mixed_vs_fp64"] = {"fp64_s": per_launch_s, "fp32_bytes_per_iter": b_alg(n, nnz, 4)}
        for name, prec in (("fp32_ru", pp.FP32_RU), ("fp32_ir", pp.FP32_IR)):
            sm = pp.Solver.from_csr(a, precision=prec)
            xm = torch.empty(n, dtype=torch.float64, device="cuda")
            sm.solve(b_d, None, xm, tol=TOL, maxit=MAXIT)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, im = sm.solve(b_d, None, xm, tol=TOL, maxit=MAXIT, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
            t_mixed = e0.elapsed_time(e1) * 1e-3
            err = (torch.linalg.norm(xm - x_d) / torch.linalg.norm(x_d)).item()
            line["mixed_vs_fp64"][name] = {"s": t_mixed, "speedup": per_launch_s / t_mixed, "iters": im.iters,
                                           "outer": im.outer_iters, "status": pp.status_name(im.status),
                                           "fp64_fallback": im.fp64_fallback, "rel_res_true": im.rel_res_true,
                                           "err_vs_fp64_solution": err}
            sm.close()

    if not args.no_mixed:
        # the Jacobi-scaled form of the same iteration (u = r, q = s; 13 streams per row)
        sv = pp.Solver.from_csr(a, variant=pp.VARIANT_JACOBI_SCALED)
        xv = torch.empty(n, dtype=torch.float64, device="cuda")
        sv.solve(b_d, None, xv, tol=TOL, maxit=MAXIT)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, iv = sv.solve(b_d, None, xv, tol=TOL, maxit=MAXIT, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t_var = e0.elapsed_time(e1) * 1e-3
        err = (torch.linalg.norm(xv - x_d) / torch.linalg.norm(x_d)).item()
        line["jacobi_scaled_vs_alg2"] = {"alg2_s": per_launch_s, "scaled_s": t_var,
                                         "speedup": per_launch_s / t_var, "iters": iv.iters,
                                         "alg2_iters": iters_per_solve,
                                         "status": pp.status_name(iv.status),
                                         "rel_res_true": iv.rel_res_true, "err_vs_alg2_solution": err,
                                         "scaled_bytes_per_iter": iv.bytes_per_iter}
        sv.close()

    if not args.no_extras:
        line["latency_2d64"] = measure_latency_2d(pp, torch)
        # the 1024-system ragged batch, FP64 and FP32 + reliable updates, against 1024
        # sequential FP64 solves
        line["batch"] = measure_batch(pp, torch, 1024, precisions=(pp.FP64, pp.FP32_RU))
        # the create-time cluster-size tuner on a batch of small systems (where it matters)
        line["batch_small_tuned"] = measure_tuned_batch(pp, torch)
        # a bounded slice of the serving stream: sizes 1e3-4e6 rows over the three families,
        # saturation and two offered rates
        line["serving"] = measure_serving(pp, nreq=96, hi=4e6, rate_factors=(0.5, 1.0), buckets=8)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(a, b)
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
