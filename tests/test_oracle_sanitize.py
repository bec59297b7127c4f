"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU only).

tests/oracle_sanitize_driver.c runs oracle/ppcg_oracle.c through every branch the other
tests use; this test builds it with -fsanitize=address,undefined, requires a clean run, and
checks that the instrumented build reports the same status, iteration count and
replacement count as the library the tests load."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_oracle_clean_under_asan_ubsan(tmp_path):
    exe = str(tmp_path / "oracle_asan")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-omit-frame-pointer",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-o", exe,
                           os.path.join(ROOT, "oracle", "ppcg_oracle.c"),
                           os.path.join(HERE, "oracle_sanitize_driver.c"), "-lm"])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    p = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert "runtime error" not in p.stderr and "ERROR: AddressSanitizer" not in p.stderr
    got = {ln.split()[0]: tuple(int(t) for t in ln.split()[1:]) for ln in p.stdout.strip().splitlines()}

    a = synth.poisson2d(24)
    i = np.arange(a.n)
    b = ((i * 7919) % 97) / 97.0 - 0.5
    x0 = 0.01 * (i % 13)

    def key(out):
        r = out["result"]
        return (r["status"], r["iters"], r["rr_count"])
    P = oracle.NORM_PAPER_U_ABS
    want = {
        "pipecg": key(oracle.pipecg(a, b, tol=1e-8, maxit=2000)),
        "pipecg_nogap": key(oracle.pipecg(a, b, tol=1e-8, maxit=2000, gap_theta=0.0)),
        "pipecg_gap_every": key(oracle.pipecg(a, b, tol=1e-8, maxit=2000, gap_theta=1e-300, gap_fall=1.0)),
        "pipecg_paper": key(oracle.pipecg(a, b, tol=1e-5, maxit=2000, norm=P)),
        "pipecg_rr": key(oracle.pipecg(a, b, x0=x0, tol=1e-8, maxit=2000, rr_period=7)),
        "pipecg_elim": key(oracle.pipecg(a, b, tol=1e-8, maxit=2000, jacobi_elim=True)),
        "pipecg_pairwise": key(oracle.pipecg(a, b, tol=1e-8, maxit=2000, sum_mode=1)),
        "pipecg_maxit": key(oracle.pipecg(a, b, tol=1e-8, maxit=5)),
        "pcg": key(oracle.pcg(a, b, tol=1e-8, maxit=2000)),
        "pcg_paper_x0": key(oracle.pcg(a, b, x0=x0, tol=1e-5, maxit=2000, norm=P, sum_mode=1)),
    }
    ind = synth.CSR(3, np.array([0, 2, 4, 5], dtype=np.int64), np.array([0, 1, 0, 1, 2], dtype=np.int32),
                    np.array([1.0, 2.0, 2.0, 1.0, 1.0]))
    b3 = np.array([1.0, -1.0, 1.0])
    want["indefinite"] = key(oracle.pipecg(ind, b3, tol=1e-8, maxit=100))
    want["indefinite_norestart"] = key(oracle.pipecg(ind, b3, tol=1e-8, maxit=100, max_restarts=0))
    assert got == want
    assert got["indefinite_norestart"][0] == oracle.ERR_BREAKDOWN
