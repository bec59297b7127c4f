"""Pins of the oracle (Algorithms 1 and 2 of arXiv 2105.06176, Sec. III) against facts the
mathematics fixes independently of the oracle's own code: dense library solves, exact
termination on spectra with k distinct eigenvalues, closed-form Poisson eigenpairs, Ritz
values of the Lanczos matrix built from (alpha, beta), the Algorithm 2 invariants checked
with scipy's SpMV, A-orthogonality, agreement with Algorithm 1, and rounding-sensitivity
calibration.  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def csr_from_dense(m):
    s = sp.csr_matrix(m)
    return synth.CSR(m.shape[0], s.indptr.astype(np.int64), s.indices.astype(np.int32),
                     s.data.astype(np.float64))


def poisson2d_mode(n, j, k):
    """Eigenvector sin(j pi (x+1)/(n+1)) sin(k pi (y+1)/(n+1)) of the 5-point Laplacian,
    row index y*n + x, with eigenvalue 4 - 2cos(j pi/(n+1)) - 2cos(k pi/(n+1))."""
    t = np.arange(1, n + 1) / (n + 1)
    v = np.outer(np.sin(k * np.pi * t), np.sin(j * np.pi * t)).ravel()
    lam = 4 - 2 * np.cos(j * np.pi / (n + 1)) - 2 * np.cos(k * np.pi / (n + 1))
    return v, lam


# ---------------------------------------------------------------- dense pins -------------

@pytest.mark.parametrize("solver", ["pipecg", "pcg"])
def test_exact_termination_k_distinct_eigenvalues(solver):
    """Jacobi-PCG on A = S B S (B = Q diag(eigs) Q^T, Hadamard Q) is CG on B/mean(eigs):
    with 6 distinct eigenvalues the Krylov space is exhausted after 6 steps, so x_6 is the
    exact solution (library dense solve) while x_5 is still far from it."""
    n = 64
    vals = np.array([1.0, 3.0, 7.0, 20.0, 50.0, 100.0])
    eigs = np.repeat(vals, [11, 11, 11, 11, 10, 10])
    a, dense = synth.hadamard_spd(n, eigs, seed=11)
    b = synth.rhs_uniform(n, 12)
    xs = np.linalg.solve(dense, b)
    f = getattr(oracle, solver)
    assert rel(f(a, b, tol=0.0, maxit=5)["x"], xs) > 1e-2
    assert rel(f(a, b, tol=0.0, maxit=6)["x"], xs) < 1e-11


@pytest.mark.parametrize("n,hi", [(16, 20.0), (32, 50.0)])
def test_n_steps_match_dense_solve(n, hi):
    """CG finishes in at most N steps in exact arithmetic (Sec. I); on well-conditioned
    dense SPD matrices FP64 reaches the library solution to 1e-10 after N steps."""
    a, dense = synth.hadamard_spd(n, np.linspace(1.0, hi, n), seed=3)
    b = synth.rhs_uniform(n, 4)
    out = oracle.pipecg(a, b, tol=0.0, maxit=n)
    assert out["result"]["iters"] == n
    assert rel(out["x"], np.linalg.solve(dense, b)) < 1e-10


def test_nonzero_x0_dense():
    a, dense = synth.hadamard_spd(32, np.linspace(1.0, 10.0, 32), seed=5)
    b = synth.rhs_uniform(32, 6)
    x0 = synth.xtrue_uniform(32, 7)
    out = oracle.pipecg(a, b, x0=x0, tol=1e-12, maxit=100)
    assert out["result"]["status"] == oracle.OK
    assert rel(out["x"], np.linalg.solve(dense, b)) < 1e-10


# ---------------------------------------------------------------- Poisson closed forms ----

def test_poisson_eigenvector_rhs_one_step():
    """b = eigenvector v of the 2-D 5-point Laplacian (diag 4): u0 = v/4, w0 = lam v/4, so
    alpha_0 = gamma_0/delta_0 = 4/lam and x_1 = v/lam exactly; the solve stops after one step."""
    n = 16
    a = synth.poisson2d(n)
    for j, k in [(1, 1), (3, 7), (16, 16), (5, 2)]:
        v, lam = poisson2d_mode(n, j, k)
        out = oracle.pipecg(a, v, tol=1e-10, maxit=50, history=True)
        assert out["result"]["iters"] == 1
        assert out["alpha"][0] == pytest.approx(4.0 / lam, rel=1e-13)
        assert rel(out["x"], v / lam) < 1e-13


def test_poisson_k_modes_exact_at_k():
    """b = sum of modes with 3 distinct eigenvalues -> exact solution at step 3."""
    n = 16
    a = synth.poisson2d(n)
    modes = [poisson2d_mode(n, 1, 2), poisson2d_mode(n, 4, 4), poisson2d_mode(n, 9, 13)]
    b = sum(v for v, _ in modes)
    xs = sum(v / lam for v, lam in modes)
    assert rel(oracle.pipecg(a, b, tol=0.0, maxit=2)["x"], xs) > 1e-3
    out = oracle.pipecg(a, b, tol=1e-10, maxit=50)
    assert out["result"]["iters"] == 3
    assert rel(out["x"], xs) < 1e-12


def lanczos_ritz(alpha, beta):
    """Eigenvalues of the Lanczos tridiagonal T built from CG coefficients (Saad, Iterative
    Methods for Sparse Linear Systems, 6.7.3): T_jj = 1/alpha_j + beta_j/alpha_{j-1},
    T_{j,j+1} = sqrt(beta_{j+1})/alpha_j, with beta_j = gamma_j/gamma_{j-1}."""
    k = len(alpha) - 1
    d = np.array([1.0 / alpha[j] + (beta[j] / alpha[j - 1] if j > 0 else 0.0) for j in range(k)])
    e = np.array([np.sqrt(beta[j + 1]) / alpha[j] for j in range(k - 1)])
    return np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_ritz_values_poisson(dim, n):
    """Extreme Ritz values from (alpha_j, beta_j) converge to the extreme eigenvalues of
    D^-1 A for the Poisson stencils: 1 -+ cos(pi/(n+1)) in 2-D, 1 -+ cos(pi/(n+1)) in 3-D
    as well (the constant diagonal 2*dim cancels the dim cosines)."""
    a = synth.poisson2d(n) if dim == 2 else synth.poisson3d(n)
    b = synth.rhs_uniform(a.n, 21)
    out = oracle.pipecg(a, b, tol=1e-13, maxit=40, history=True)
    ritz = lanczos_ritz(out["alpha"], out["beta"])
    c = np.cos(np.pi / (n + 1))
    assert ritz.min() == pytest.approx(1 - c, rel=1e-7)
    assert ritz.max() == pytest.approx(1 + c, rel=1e-9)
    assert ritz.min() > (1 - c) * (1 - 1e-9) and ritz.max() < (1 + c) * (1 + 1e-9)


def test_cg_iteration_bound_cfg_2d():
    """Iterations to 1e-8 on the 64x64 Poisson problem stay below the Chebyshev bound
    k <= sqrt(kappa)/2 * ln(2 sqrt(kappa)/tol) with kappa = (1+c)/(1-c), c = cos(pi/65)."""
    a = synth.poisson2d(64)
    b = a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    out = oracle.pipecg(a, b, tol=1e-8, maxit=10000)
    c = np.cos(np.pi / 65)
    kappa = (1 + c) / (1 - c)
    bound = np.sqrt(kappa) / 2 * np.log(2 * np.sqrt(kappa) / 1e-8)
    assert out["result"]["status"] == oracle.OK
    assert 0 < out["result"]["iters"] <= bound


# ---------------------------------------------------------------- Algorithm 2 invariants --

def test_pipecg_invariants():
    """By induction over the vector updates: s = A p, q = M^-1 s, z = A q, u = M^-1 r,
    w = A u, m = M^-1 w, n = A m, r = b - A x.  Checked with scipy's SpMV, after 15 steps."""
    a = synth.varcoeff3d(10, seed=5)
    A = a.to_scipy()
    dinv = 1.0 / A.diagonal()
    b = synth.rhs_uniform(a.n, 6)
    st = oracle.pipecg(a, b, tol=0.0, maxit=15, state=True)["state"]
    checks = {
        "s=Ap": (st["s"], A @ st["p"]),
        "q=M^-1 s": (st["q"], dinv * st["s"]),
        "z=Aq": (st["z"], A @ st["q"]),
        "u=M^-1 r": (st["u"], dinv * st["r"]),
        "w=Au": (st["w"], A @ st["u"]),
        "m=M^-1 w": (st["m"], dinv * st["w"]),
        "n=Am": (st["n"], A @ st["m"]),
        "r=b-Ax": (st["r"], b - A @ st["x"]),
    }
    for name, (lhs, rhs) in checks.items():
        assert rel(lhs, rhs) < 1e-11, name


def test_a_orthogonality_and_residual_orthogonality():
    """(p_i, A p_j) = 0 and (r_i, M^-1 r_j) = 0 for i != j (exact arithmetic); in FP64 the
    normalised values stay near rounding level over the first 10 steps."""
    a = synth.varcoeff2d(20, seed=9)
    A = a.to_scipy()
    b = synth.rhs_uniform(a.n, 10)
    P, R, U = [], [], []
    for k in range(1, 11):
        st = oracle.pipecg(a, b, tol=0.0, maxit=k, state=True)["state"]
        P.append(st["p"])
    for k in range(0, 10):
        st = oracle.pipecg(a, b, tol=0.0, maxit=k, state=True)["state"]
        R.append(st["r"])
        U.append(st["u"])
    P = np.array(P).T
    G = P.T @ (A @ P)
    dg = np.sqrt(np.diag(G))
    Gn = G / np.outer(dg, dg)
    assert np.abs(Gn - np.diag(np.diag(Gn))).max() < 1e-8
    R, U = np.array(R).T, np.array(U).T
    H = R.T @ U
    dh = np.sqrt(np.diag(H))
    Hn = H / np.outer(dh, dh)
    assert np.abs(Hn - np.diag(np.diag(Hn))).max() < 1e-8


# ---------------------------------------------------------------- Alg. 1 vs Alg. 2 -------

@pytest.mark.parametrize("k", [5, 20, 50])
def test_classic_and_pipelined_agree_early(k):
    a = synth.poisson2d(64)
    b = a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    x1 = oracle.pcg(a, b, tol=0.0, maxit=k)["x"]
    x2 = oracle.pipecg(a, b, tol=0.0, maxit=k)["x"]
    assert rel(x2, x1) < 1e-10


def test_classic_and_pipelined_same_iterations_varcoeff():
    a = synth.varcoeff3d(24, seed=2)
    b = synth.rhs_uniform(a.n, 3)
    r1 = oracle.pcg(a, b, tol=1e-8, maxit=5000)
    r2 = oracle.pipecg(a, b, tol=1e-8, maxit=5000)
    assert r1["result"]["status"] == r2["result"]["status"] == oracle.OK
    assert abs(r1["result"]["iters"] - r2["result"]["iters"]) <= 1
    assert r2["result"]["res_true"] <= 1e-8 * r2["result"]["bnorm"]
    assert rel(r2["x"], r1["x"]) < 1e-7


def test_config_2d_solution_error():
    """64x64 Poisson, b = A x_true: converged x is close to x_true (kappa ~ 1.7e3)."""
    a = synth.poisson2d(64)
    xt = synth.xtrue_uniform(a.n, 1)
    out = oracle.pipecg(a, a.to_scipy() @ xt, tol=1e-8, maxit=10000)
    assert out["result"]["status"] == oracle.OK
    assert out["result"]["res_true"] <= 1e-8 * out["result"]["bnorm"]
    assert rel(out["x"], xt) < 2e-5


# ---------------------------------------------------------------- rounding calibration ---

@pytest.mark.parametrize("family,k", [("poisson2d_64", 50), ("varcoeff3d_32", 20)])
def test_summation_order_sensitivity(family, k):
    """Two summation orders (sequential, pairwise) agree on x_k to 1e-12 at the k used by
    the GPU parity tests, so a 1e-10 GPU-vs-oracle bound at that k is meaningful."""
    if family == "poisson2d_64":
        a = synth.poisson2d(64)
        b = a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    else:
        a = synth.varcoeff3d(32, seed=1)
        b = synth.rhs_uniform(a.n, 1)
    x1 = oracle.pipecg(a, b, tol=0.0, maxit=k, sum_mode=0)["x"]
    x2 = oracle.pipecg(a, b, tol=0.0, maxit=k, sum_mode=1)["x"]
    assert rel(x1, x2) < 1e-12


# ---------------------------------------------------------------- modes and edge cases ---

def test_paper_norm_mode():
    """Sec. VI protocol: absolute tolerance on sqrt((u, u)), exact solution 1/sqrt(N)."""
    a = synth.varcoeff2d(32, seed=3)
    xs = np.full(a.n, 1.0 / np.sqrt(a.n))
    b = a.to_scipy() @ xs
    out = oracle.pipecg(a, b, tol=1e-5, maxit=10000, norm=oracle.NORM_PAPER_U_ABS, history=True)
    assert out["result"]["status"] == oracle.OK
    h = out["res"]
    assert h[-1] <= 1e-5 < h[-2]
    st = oracle.pipecg(a, b, tol=0.0, maxit=out["result"]["iters"], state=True)["state"]
    assert np.sqrt(st["u"] @ st["u"]) == pytest.approx(h[-1], rel=1e-12)


def test_zero_rhs():
    a = synth.poisson2d(8)
    out = oracle.pipecg(a, np.zeros(a.n), x0=np.ones(a.n), tol=1e-8, maxit=10)
    assert out["result"]["status"] == oracle.OK and out["result"]["iters"] == 0
    assert not out["x"].any()


def test_exact_initial_guess():
    a = synth.poisson2d(8)
    xs = synth.xtrue_uniform(a.n, 3)
    b = a.to_scipy() @ xs
    out = oracle.pipecg(a, b, x0=xs, tol=1e-8, maxit=10)
    assert out["result"]["status"] == oracle.OK and out["result"]["iters"] == 0
    assert np.array_equal(out["x"], xs)


def test_maxit_zero_and_not_converged():
    a = synth.poisson2d(16)
    b = synth.rhs_uniform(a.n, 4)
    out = oracle.pipecg(a, b, tol=1e-8, maxit=0)
    assert out["result"]["status"] == oracle.ERR_NOT_CONVERGED and out["result"]["iters"] == 0
    assert not out["x"].any()
    out = oracle.pipecg(a, b, tol=1e-8, maxit=3)
    assert out["result"]["status"] == oracle.ERR_NOT_CONVERGED and out["result"]["iters"] == 3


def test_not_spd_diagonal():
    m = np.array([[2.0, -1.0, 0.0], [-1.0, 0.0, -1.0], [0.0, -1.0, 2.0]])
    out = oracle.pipecg(csr_from_dense(m), np.ones(3), tol=1e-8, maxit=10)
    assert out["result"]["status"] == oracle.ERR_NOT_SPD
    m2 = np.array([[2.0, -1.0], [-1.0, 2.0]])
    a = csr_from_dense(m2)
    a = synth.CSR(2, np.array([0, 2, 3], dtype=np.int64), np.array([0, 1, 0], dtype=np.int32),
                  np.array([2.0, -1.0, -1.0]))      # row 1 has no diagonal entry
    assert oracle.pipecg(a, np.ones(2), tol=1e-8, maxit=10)["result"]["status"] == oracle.ERR_NOT_SPD


def test_indefinite_breakdown():
    m = np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    out = oracle.pipecg(csr_from_dense(m), np.array([1.0, -1.0, 1.0]), tol=1e-8, maxit=20)
    assert out["result"]["status"] == oracle.ERR_BREAKDOWN


def test_nonfinite_input():
    a = synth.poisson2d(8)
    b = synth.rhs_uniform(a.n, 2)
    b[5] = np.nan
    out = oracle.pipecg(a, b, tol=1e-8, maxit=10)
    assert out["result"]["status"] == oracle.ERR_NONFINITE


def test_residual_replacement():
    """Periodic replacement resets r, u, w, s, q, z to their true values; the solve still
    converges and, right after a replacement, r equals b - A x to rounding."""
    a = synth.poisson2d(64)
    b = a.to_scipy() @ synth.xtrue_uniform(a.n, 1)
    plain = oracle.pipecg(a, b, tol=1e-8, maxit=10000)
    rr = oracle.pipecg(a, b, tol=1e-8, maxit=10000, rr_period=25)
    assert rr["result"]["status"] == oracle.OK and rr["result"]["rr_count"] >= 5
    assert abs(rr["result"]["iters"] - plain["result"]["iters"]) <= 3
    st = oracle.pipecg(a, b, tol=0.0, maxit=25, rr_period=25, state=True)["state"]
    A = a.to_scipy()
    assert rel(st["r"], b - A @ st["x"]) < 1e-14
    assert rel(st["s"], A @ st["p"]) < 1e-14
    assert rel(st["z"], A @ st["q"]) < 1e-14


def _breakdown_system():
    """A 2-D log-normal variable-coefficient system (267^2 rows) on which plain pipelined
    PCG breaks down (alpha denominator <= 0) just before reaching 1e-8."""
    spec = [s for s in synth.batch_mix(128, 11) if s[0] == "varcoeff2d" and s[1] == 267][0]
    return synth.build_spec(spec)


def test_restart_on_breakdown():
    """With the measured-gap replacement off: Alg. 2 stops with a breakdown near its
    attainable accuracy while Alg. 1 converges; with restarts (true residuals, reset
    directions, beta = 0) the pipelined solve reaches the same true residual as Alg. 1."""
    a, b = _breakdown_system()
    plain = oracle.pipecg(a, b, tol=1e-8, maxit=20000, max_restarts=0, gap_theta=0.0)
    assert plain["result"]["status"] == oracle.ERR_BREAKDOWN
    classic = oracle.pcg(a, b, tol=1e-8, maxit=20000)
    assert classic["result"]["status"] == oracle.OK
    out = oracle.pipecg(a, b, tol=1e-8, maxit=20000, gap_theta=0.0)
    r = out["result"]
    assert r["status"] == oracle.OK and 1 <= r["rr_count"] <= 8
    A = a.to_scipy()
    assert np.linalg.norm(b - A @ out["x"]) <= 1e-8 * np.linalg.norm(b)
    assert rel(out["x"], classic["x"]) < 1e-6
    # before the first breakdown the two runs are the same computation
    k = plain["result"]["iters"] - 5
    assert np.array_equal(oracle.pipecg(a, b, tol=0.0, maxit=k, max_restarts=0, gap_theta=0.0)["x"],
                          oracle.pipecg(a, b, tol=0.0, maxit=k, gap_theta=0.0)["x"])


def test_gap_replacement():
    """Measured-gap residual replacement (the accuracy criterion of the pipelined-CG
    literature, not in the paper).  In exact arithmetic Alg. 2 and Alg. 1 are the same
    iteration, so Alg. 1's count is the reference:
      * on the system where Alg. 2 breaks down, replacing the residuals while their
        deviation from b - A x is still below 1e-6 ||r|| keeps the alpha/beta recurrences
        consistent: no breakdown even with restarts off, the true residual at the bar, and
        Alg. 1's iteration count within 2 -- where the late replacement and the beta = 0
        restart cost more than a hundred iterations;
      * the count no longer depends on the order of the dot products' sums (it does, by
        tens of iterations, without the trigger);
      * on a well-conditioned system the deviation never reaches 1% of ||r||, so a 1e-2
        threshold never replaces and the run is bit for bit the run without the trigger (a
        gap formed with a wrong sign or a dropped term would reach ||r|| and replace)."""
    a, b = _breakdown_system()
    A = a.to_scipy()
    classic = oracle.pcg(a, b, tol=1e-8, maxit=20000)["result"]["iters"]
    runs = {m: oracle.pipecg(a, b, tol=1e-8, maxit=20000, max_restarts=0, sum_mode=m) for m in (0, 1)}
    for m, out in runs.items():
        r = out["result"]
        assert r["status"] == oracle.OK and r["rr_count"] >= 1, (m, r)
        assert np.linalg.norm(b - A @ out["x"]) <= 1e-8 * np.linalg.norm(b)
        assert abs(r["iters"] - classic) <= 2, (m, r["iters"], classic)
    assert abs(runs[0]["result"]["iters"] - runs[1]["result"]["iters"]) <= 2
    off = [oracle.pipecg(a, b, tol=1e-8, maxit=20000, gap_theta=0.0, sum_mode=m)["result"]["iters"] for m in (0, 1)]
    assert min(off) > classic + 100 and abs(off[0] - off[1]) > 10, (off, classic)
    p = synth.poisson2d(64)
    bp = p.to_scipy() @ synth.xtrue_uniform(p.n, 1)
    loose = oracle.pipecg(p, bp, tol=1e-10, maxit=10000, gap_theta=1e-2)
    none = oracle.pipecg(p, bp, tol=1e-10, maxit=10000, gap_theta=0.0)
    assert loose["result"]["rr_count"] == 0 and loose["result"] == none["result"]
    assert np.array_equal(loose["x"], none["x"])
    # every check replaces (gap_fall 0: a check at every iteration): r is b - A x at exit
    st = oracle.pipecg(p, bp, tol=0.0, maxit=30, gap_theta=1e-300, gap_fall=0.0, state=True)
    assert st["result"]["rr_count"] == 30        # iterations 1..30, the last before the maxit exit
    assert rel(st["state"]["r"], bp - p.to_scipy() @ st["state"]["x"]) < 1e-14


# ---------------------------------------------------------------- Jacobi elimination -----

def test_jacobi_elimination_variant():
    """The variant that computes q = M^-1 s and u = M^-1 r instead of carrying them: exact
    termination on k distinct eigenvalues like Alg. 2, the same iterates as Alg. 2 to
    rounding in early iterations, the invariants u = M^-1 r, q = M^-1 s hold to the last
    bit, and the full solve converges in the same number of iterations (+-2)."""
    n = 64
    eigs = np.repeat(np.array([1.0, 3.0, 7.0, 20.0, 50.0, 100.0]), [11, 11, 11, 11, 10, 10])
    a, dense = synth.hadamard_spd(n, eigs, seed=11)
    b = synth.rhs_uniform(n, 12)
    xs = np.linalg.solve(dense, b)
    assert rel(oracle.pipecg(a, b, tol=0.0, maxit=5, jacobi_elim=True)["x"], xs) > 1e-2
    assert rel(oracle.pipecg(a, b, tol=0.0, maxit=6, jacobi_elim=True)["x"], xs) < 1e-11
    a = synth.varcoeff3d(24, seed=2)
    b = synth.rhs_uniform(a.n, 3)
    for k in (5, 20):
        x1 = oracle.pipecg(a, b, tol=0.0, maxit=k)["x"]
        x2 = oracle.pipecg(a, b, tol=0.0, maxit=k, jacobi_elim=True)["x"]
        assert rel(x2, x1) < 1e-11
    st = oracle.pipecg(a, b, tol=0.0, maxit=20, jacobi_elim=True, state=True)["state"]
    dinv = 1.0 / a.to_scipy().diagonal()
    assert np.array_equal(st["u"], st["r"] / (1.0 / dinv)) or rel(st["u"], dinv * st["r"]) < 1e-15
    f1 = oracle.pipecg(a, b, tol=1e-8, maxit=5000)
    f2 = oracle.pipecg(a, b, tol=1e-8, maxit=5000, jacobi_elim=True)
    assert f2["result"]["status"] == oracle.OK
    assert abs(f1["result"]["iters"] - f2["result"]["iters"]) <= 2


def test_openmp_build_is_bitwise_identical():
    """The OpenMP build of the oracle (timed as the all-core CPU baseline) spreads only rows
    over threads and keeps the dot products sequential, so it must return the plain build's
    iterates bit for bit: Algorithm 2 with residual replacement, the Jacobi-eliminated
    variant, and Algorithm 1."""
    a = synth.varcoeff3d(20, 5)
    b = synth.rhs_uniform(a.n, 5)
    for kw in ({"rr_period": 7}, {"jacobi_elim": True}, {"norm": oracle.NORM_PAPER_U_ABS, "tol": 1e-9}):
        kw = {"tol": 1e-10, "maxit": 400, **kw}
        plain = oracle.pipecg(a, b, history=True, state=True, **kw)
        omp = oracle.pipecg(a, b, history=True, state=True, openmp=True, **kw)
        assert plain["result"] == omp["result"]
        assert np.array_equal(plain["alpha"], omp["alpha"]) and np.array_equal(plain["beta"], omp["beta"])
        for k in oracle.STATE_NAMES:
            assert np.array_equal(plain["state"][k], omp["state"][k]), k
    p1 = oracle.pcg(a, b, tol=1e-10, history=True)
    p2 = oracle.pcg(a, b, tol=1e-10, history=True, openmp=True)
    assert p1["result"] == p2["result"] and np.array_equal(p1["x"], p2["x"])
    assert np.array_equal(oracle.spmv(a, b), oracle.spmv(a, b, openmp=True))
    assert oracle.threads() == 1 and oracle.threads(openmp=True) >= 1
