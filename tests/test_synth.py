"""Generators: structure pinned by the nnz formulas (including the paper's Table II) and by
the public SplitMix64 test vectors.  CPU only."""
import os

import numpy as np
import pytest

import synth
from synth.rng import GOLDEN, mix64

GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN_DIR, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_reference_vectors():
    want = [int(r[0], 16) for r in _rows("splitmix64_seed0.txt")]
    got = mix64(np.array([(i * GOLDEN) % 2 ** 64 for i in (1, 2, 3)], dtype=np.uint64))
    assert [int(v) for v in got] == want


def test_streams_are_counter_based():
    a = synth.uniform(7, 3, 1000)
    b = synth.uniform(7, 3, 400, offset=600)
    assert np.array_equal(a[600:], b)
    assert not np.array_equal(a, synth.uniform(7, 4, 1000))
    g = synth.normal(1, 0, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01


@pytest.mark.parametrize("n", [2, 5, 64])
def test_poisson2d_nnz(n):
    a = synth.poisson2d(n)
    assert a.n == n * n and a.nnz == 5 * n * n - 4 * n


@pytest.mark.parametrize("n", [2, 7, 16])
def test_stencil3d_nnz(n):
    assert synth.poisson3d(n).nnz == 7 * n ** 3 - 6 * n ** 2
    assert synth.varcoeff3d(n, 1).nnz == 7 * n ** 3 - 6 * n ** 2


def test_config_sizes():
    """2-D 64x64: N = 4096, nnz = 20,224.  3-D 256^3: N = 16,777,216, nnz = 117,047,296."""
    assert synth.poisson2d(64).nnz == 20224
    n = 256
    assert n ** 3 == 16777216 and 7 * n ** 3 - 6 * n ** 2 == 117047296


@pytest.mark.parametrize("n", [5, 6, 7, 9])
def test_box125_structure(n):
    a = synth.box125(n)
    assert a.nnz == synth.box125_nnz(n) == (5 * n - 6) ** 3
    A = a.to_scipy()
    assert abs(A - A.T).max() == 0
    assert (A.diagonal() == 124).all()


@pytest.mark.parametrize("n,slab", [(3, 1), (4, 3), (6, 8), (7, 2)])
def test_box125_matches_brute_force(n, slab):
    """Every pair of cells within Chebyshev distance 2 is an entry (124 on the diagonal,
    -1 off it), and the slab-wise construction does not depend on the slab height."""
    a = synth.box125(n, slab=slab)
    N = n ** 3
    idx = np.arange(N)
    zyx = np.stack([idx // (n * n), (idx // n) % n, idx % n], axis=1)
    cheb = np.abs(zyx[:, None, :] - zyx[None, :, :]).max(axis=2)
    expect = np.where(cheb <= 2, -1.0, 0.0)
    np.fill_diagonal(expect, 124.0)
    assert np.array_equal(a.dense(), expect)
    assert np.all(np.diff(a.col[a.row_ptr[0]:a.row_ptr[1]]) > 0)


@pytest.mark.parametrize("n,R", [(4, 1), (5, 1), (7, 3)])
def test_box_stencil_matches_brute_force(n, R):
    a = synth.box_stencil(n, R, 2.0 * (2 * R + 1) ** 3, -0.5)
    idx = np.arange(n ** 3)
    zyx = np.stack([idx // (n * n), (idx // n) % n, idx % n], axis=1)
    cheb = np.abs(zyx[:, None, :] - zyx[None, :, :]).max(axis=2)
    expect = np.where(cheb <= R, -0.5, 0.0)
    np.fill_diagonal(expect, 2.0 * (2 * R + 1) ** 3)
    assert np.array_equal(a.dense(), expect)


def test_box125_reproduces_table2():
    for name, N, nnz in _rows("table2_poisson125.txt"):
        n = round(int(N) ** (1 / 3))
        assert n ** 3 == int(N), name
        assert synth.box125_nnz(n) == int(nnz), name


@pytest.mark.parametrize("gen", ["varcoeff2d", "varcoeff3d", "rgg", "box125"])
def test_spd_and_symmetric(gen):
    if gen == "varcoeff2d":
        a = synth.varcoeff2d(12, 3)
    elif gen == "varcoeff3d":
        a = synth.varcoeff3d(6, 3)
    elif gen == "rgg":
        a = synth.rgg_laplacian(600, 0.18, 1e-3, 3)
    else:
        a = synth.box125(6)
    A = a.to_scipy().toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    assert np.all(np.diff(a.row_ptr) > 0)
    for i in range(a.n):
        c = a.col[a.row_ptr[i]:a.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_varcoeff_lognormal_faces():
    """Off-diagonals are -exp(g) with g ~ N(0,1): log(-a_ij) has mean ~0, std ~1."""
    a = synth.varcoeff3d(24, 5)
    A = a.to_scipy().tocoo()
    off = A.data[A.row != A.col]
    g = np.log(-off)
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1) < 0.03


def test_rgg_degree():
    npts = 100000
    r = (3 * 14.0 / (4 * np.pi * npts)) ** (1 / 3)
    a = synth.rgg_laplacian(npts, r, 1e-3, 1)
    deg = np.diff(a.row_ptr) - 1
    assert 12.5 < deg.mean() < 14.2
    A = a.to_scipy()
    assert abs(A - A.T).max() == 0
    assert np.allclose(A.diagonal(), deg + 1e-3)


def test_batch_mix_sizes():
    specs = synth.batch_mix(1024, 1)
    sizes = np.array([n * n if f == "varcoeff2d" else n ** 3 for f, n, _, _ in specs])
    assert sizes.min() >= 900 and sizes.max() <= 2.1e5
    assert 0.4 < np.mean([f == "varcoeff2d" for f, *_ in specs]) < 0.6
    assert 8e3 < np.median(sizes) < 2.2e4


def test_fullsize_golden_matches_the_generators():
    """The stored full-size oracle record (tests/golden/fullsize_oracle.json) belongs to the
    inputs the generators make today: the batch's 1024 system sizes, the 256^3 grid and the
    RGG parameters; its calibrated fixed k meets the 1e-12 rounding-sensitivity rule."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_oracle.json")) as f:
        gold = json.load(f)
    specs = synth.batch_mix(gold["batch_1024"]["count"], gold["batch_1024"]["seed"])
    assert len(specs) == len(gold["batch_1024"]["systems"]) == 1024
    for (fam, size, _, _), rec in zip(specs, gold["batch_1024"]["systems"]):
        assert rec["n"] == (size ** 2 if fam == "varcoeff2d" else size ** 3)
        assert rec["status"] == 0 and rec["rel_res_true"] <= 1e-8
    vc = gold["varcoeff3d_256"]
    assert vc["grid"] == 256 and vc["iters"] > 0 and vc["rel_res_true"] <= 1e-8
    for rec in (vc, gold["rgg_4M"]):
        assert rec["fixed_k"] in (5, 10, 20) and rec["fixed_k_rel_diff_seq_vs_pairwise"] <= 1e-12
    assert gold["rgg_4M"]["iters_1e-10"] > gold["rgg_4M"]["iters_1e-08"]
