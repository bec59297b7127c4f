"""Host-side logic of bench.py on the CPU: the roofline's DRAM traffic comes from the
committed ncu record only for the workload and kernel source it was captured on (after a
kernel change the bench reports none until the record is taken again)."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record():
    with open(os.path.join(ROOT, "profiles", "k_grid_traffic.json")) as f:
        return json.load(f)


def _current(rec):
    with open(os.path.join(ROOT, "paper_2105_06176_b300", "csrc", "solver.cu"), "rb") as f:
        return rec["kernel_source_sha256"] == hashlib.sha256(f.read()).hexdigest()


def test_traffic_record_is_of_the_bench_workload():
    rec = _record()
    n, nnz = 256 ** 3, 7 * 256 ** 3 - 6 * 256 ** 2
    assert rec["b_alg_per_iter"] == bench.b_alg(n, nnz, 8)
    # per iteration the kernel moves at most its algorithmic bytes (B_alg counts bytes the
    # offset-pattern kernel never reads) and at least the 17 vector streams it must write/read
    per_iter = rec["dram_bytes_per_launch"] / rec["iterations"]
    assert 17 * 8 * n * 0.9 < per_iter < rec["b_alg_per_iter"]
    assert abs(rec["dram_over_balg"] - per_iter / rec["b_alg_per_iter"]) < 1e-3


def test_profiled_traffic_scales_by_iterations_and_refuses_other_sizes():
    rec = _record()
    t, src = bench.profiled_traffic(rec["b_alg_per_iter"], rec["iterations"])
    if not _current(rec):      # kernel source changed since the capture: no traffic claimed
        assert t is None and "kernel changed" in src
        return
    assert t == rec["dram_bytes_per_launch"] and "ncu capture" in src
    t2, _ = bench.profiled_traffic(rec["b_alg_per_iter"], rec["iterations"] / 2)
    assert abs(t2 - t / 2) < 1.0
    t3, src3 = bench.profiled_traffic(rec["b_alg_per_iter"] // 8, rec["iterations"])
    assert t3 is None and "another grid size" in src3
