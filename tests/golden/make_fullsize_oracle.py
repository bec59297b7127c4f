"""Write ``fullsize_oracle.json``: what the oracle (Alg. 2 of arXiv 2105.06176, Sec. III, in
plain sequential FP64 C) gives on the benchmark workloads at their full sizes, for the GPU
parity tests that cannot run the oracle to convergence themselves.

Every value comes from ``oracle/`` alone; the inputs come from the seeded generators in
``synth/``.  The OpenMP build of the oracle is used for speed: it threads only row-independent
loops and keeps the dot products sequential, so its iterates are bitwise those of the plain
build (tested in ``tests/test_oracle_pins.py``).

Records (the oracle's defaults, measured-gap residual replacement included):
  * 3-D 7-point log-normal diffusion 256^3 (seed 1, b ~ U[-1, 1] seed 1), rel tol 1e-8:
    iterations, exit status and true relative residual; and the fixed k for the GPU's x_k
    comparison: the largest k of (20, 10, 5) at which the oracle's x_k with sequential and
    with pairwise dot products agree to 1e-12, so that the 1e-10 parity bar measures the
    kernel and not the rounding order.
  * RGG Laplacian, 4,000,000 points (seed 3, expected degree 14, shift 1e-3), b seed 3, rel
    tol 1e-8 and 1e-10: iterations; and the fixed k chosen the same way.
  * The 1024-system ragged batch (batch_mix(1024, 11)), rel tol 1e-8: iterations and
    residual replacements per system.
Every iteration count is stored twice: with the oracle's sequential dot products (the
definition) and with pairwise ones ("_pairwise").  The two bound how far rounding order alone
moves the count; the GPU tests hold the GPU's count within that envelope widened by 2.

Run from the repository root:  python tests/golden/make_fullsize_oracle.py   (about half
an hour on eight cores).
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_oracle.json")


def _batch_one(spec):
    a, b = synth.build_spec(tuple(spec))
    r = oracle.pipecg(a, b, tol=1e-8, maxit=20000)["result"]
    p = oracle.pipecg(a, b, tol=1e-8, maxit=20000, sum_mode=1)["result"]
    return {"n": a.n, "iters": r["iters"], "iters_pairwise": p["iters"], "status": r["status"],
            "rr_count": r["rr_count"], "rel_res_true": r["res_true"] / r["bnorm"]}


def calibrated_k(a, b):
    for k in (20, 10, 5):
        x0 = oracle.pipecg(a, b, tol=0.0, maxit=k, openmp=True)["x"]
        x1 = oracle.pipecg(a, b, tol=0.0, maxit=k, sum_mode=1, openmp=True)["x"]
        d = float(np.linalg.norm(x0 - x1) / np.linalg.norm(x0))
        if d <= 1e-12:
            return k, d
    raise RuntimeError("no fixed k with a 1e-12 rounding sensitivity")


def main():
    out = {"source": "oracle/ppcg_oracle.c (Alg. 2, plain FP64, sequential dot products), "
                     "inputs from synth/; written by tests/golden/make_fullsize_oracle.py"}
    t0 = time.time()
    a = synth.varcoeff3d(256, 1)
    b = synth.rhs_uniform(a.n, 1)
    r = oracle.pipecg(a, b, tol=1e-8, maxit=20000, openmp=True)["result"]
    rp = oracle.pipecg(a, b, tol=1e-8, maxit=20000, sum_mode=1, openmp=True)["result"]
    k, d = calibrated_k(a, b)
    out["varcoeff3d_256"] = {"grid": 256, "matrix_seed": 1, "rhs_seed": 1, "tol": 1e-8,
                             "iters": r["iters"], "iters_pairwise": rp["iters"], "status": r["status"],
                             "rel_res_true": r["res_true"] / r["bnorm"],
                             "fixed_k": k, "fixed_k_rel_diff_seq_vs_pairwise": d}
    print("varcoeff3d_256", out["varcoeff3d_256"], f"{time.time() - t0:.0f} s", flush=True)
    del a, b

    npts = 4_000_000
    a = synth.rgg_laplacian(npts, (3 * 14.0 / (4 * np.pi * npts)) ** (1 / 3), 1e-3, 3)
    b = synth.rhs_uniform(a.n, 3)
    rec = {"points": npts, "matrix_seed": 3, "rhs_seed": 3, "degree": 14.0, "shift": 1e-3}
    rec["fixed_k"], rec["fixed_k_rel_diff_seq_vs_pairwise"] = calibrated_k(a, b)
    for tol in (1e-8, 1e-10):
        r = oracle.pipecg(a, b, tol=tol, maxit=20000, openmp=True)["result"]
        rp = oracle.pipecg(a, b, tol=tol, maxit=20000, sum_mode=1, openmp=True)["result"]
        rec[f"iters_{tol:.0e}"] = r["iters"]
        rec[f"iters_pairwise_{tol:.0e}"] = rp["iters"]
        rec[f"status_{tol:.0e}"] = r["status"]
        rec[f"rel_res_true_{tol:.0e}"] = r["res_true"] / r["bnorm"]
    out["rgg_4M"] = rec
    print("rgg_4M", rec, f"{time.time() - t0:.0f} s", flush=True)
    del a, b

    specs = synth.batch_mix(1024, 11)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(_batch_one, [list(s) for s in specs], chunksize=4)
    out["batch_1024"] = {"count": 1024, "seed": 11, "tol": 1e-8, "systems": res}
    print("batch_1024", sum(r["iters"] for r in res), f"{time.time() - t0:.0f} s", flush=True)

    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
