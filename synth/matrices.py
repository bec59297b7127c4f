"""Seeded sparse SPD matrices in CSR form (row_ptr int64, col int32, val float64).

Families:
  * ``poisson2d``    -- 5-point Laplacian on an n x n grid (diag 4, off-diag -1).
  * ``poisson3d``    -- 7-point Laplacian on an n^3 grid (diag 6, off-diag -1).
  * ``varcoeff2d/3d``-- cell-centred finite-volume diffusion with log-normal face
                        coefficients k_f = exp(g), g ~ N(0, 1); boundary faces are
                        Dirichlet and only add to the diagonal (an SPD M-matrix).
  * ``rgg_laplacian``-- graph Laplacian of a random geometric graph in the unit cube,
                        unit weights, plus a diagonal shift; rows in cell-list order.
  * ``box125``       -- the 125-point (5x5x5 box) stencil of the paper's Table II
                        matrices, truncated at the boundary; diag 124, off-diag -1.
  * ``hadamard_spd`` -- dense SPD matrices with a prescribed spectrum for the
                        preconditioned operator (pins for the oracle).

Rows are numbered lexicographically with x fastest; columns are ascending in each row.
"""
from dataclasses import dataclass

import numpy as np

from .rng import uniform, uniform_pm1, normal

# stream ids: one per independent use of a seed
_S_FACE, _S_XTRUE, _S_RHS, _S_POINTS, _S_SCALE, _S_PERM, _S_SIGN, _S_SIZES, _S_FAMILY = range(9)


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray   # int64, n + 1
    col: np.ndarray       # int32, nnz
    val: np.ndarray       # float64, nnz
    name: str = ""

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def dense(self):
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        a[rows, self.col] = self.val
        return a


def _compress(cols, vals, mask, name):
    """Dense (n, k) candidate table -> CSR keeping entries where ``mask`` holds.

    Candidates of a row must already be in ascending column order."""
    n = cols.shape[0]
    lens = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    return CSR(n, row_ptr, cols[mask].astype(np.int32), vals[mask].astype(np.float64), name)


def _stencil(dims, offsets, value_fn, name):
    """Generic structured stencil.  ``dims`` = (nz, ny, nx); ``offsets`` = list of
    (dz, dy, dx) in ascending linear-offset order; ``value_fn(k, z, y, x)`` returns the
    value of candidate k for the given broadcast cell coordinates."""
    nz, ny, nx = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    n = nz * ny * nx
    k = len(offsets)
    cols = np.empty((n, k), dtype=np.int64)
    vals = np.empty((n, k), dtype=np.float64)
    mask = np.empty((n, k), dtype=bool)
    for j, (dz, dy, dx) in enumerate(offsets):
        zz, yy, xx = z + dz, y + dy, x + dx
        mask[:, j] = (zz >= 0) & (zz < nz) & (yy >= 0) & (yy < ny) & (xx >= 0) & (xx < nx)
        cols[:, j] = (zz * ny + yy) * nx + xx
        vals[:, j] = value_fn(j, z, y, x)
    cols[~mask] = 0
    return _compress(cols, vals, mask, name)


def poisson2d(n):
    """5-point Poisson on an n x n grid: diag 4, off-diag -1; nnz = 5n^2 - 4n."""
    offs = [(0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0)]
    return _stencil((1, n, n), offs, lambda j, z, y, x: np.full(z.shape, 4.0 if j == 2 else -1.0),
                    f"poisson2d_{n}")


def poisson3d(n):
    """7-point Poisson on an n^3 grid: diag 6, off-diag -1; nnz = 7n^3 - 6n^2."""
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    return _stencil((n, n, n), offs, lambda j, z, y, x: np.full(z.shape, 6.0 if j == 3 else -1.0),
                    f"poisson3d_{n}")


def _face_coeffs(seed, count):
    return np.exp(normal(seed, _S_FACE, count))


def varcoeff3d(n, seed):
    """Cell-centred 7-point diffusion on n^3 cells with k_f = exp(N(0,1)) on all 3n^2(n+1)
    faces.  Face ids: x-faces (z, y, fx) first, then y-faces (z, fy, x), then z-faces
    (fz, y, x), each in C order; face id i takes normal i of the face stream."""
    nf = n * n * (n + 1)
    k = _face_coeffs(seed, 3 * nf)
    kx = k[:nf].reshape(n, n, n + 1)
    ky = k[nf:2 * nf].reshape(n, n + 1, n)
    kz = k[2 * nf:].reshape(n + 1, n, n)
    west, east = kx[:, :, :-1].ravel(), kx[:, :, 1:].ravel()
    south, north = ky[:, :-1, :].ravel(), ky[:, 1:, :].ravel()
    bottom, top = kz[:-1, :, :].ravel(), kz[1:, :, :].ravel()
    diag = west + east + south + north + bottom + top
    by_slot = [bottom, south, west, diag, east, north, top]
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    return _stencil((n, n, n), offs,
                    lambda j, z, y, x: by_slot[j] if j == 3 else -by_slot[j], f"varcoeff3d_{n}")


def varcoeff2d(n, seed):
    """2-D analogue of :func:`varcoeff3d` on n x n cells (2n(n+1) faces: x-faces then y-faces)."""
    nf = n * (n + 1)
    k = _face_coeffs(seed, 2 * nf)
    kx = k[:nf].reshape(n, n + 1)
    ky = k[nf:].reshape(n + 1, n)
    west, east = kx[:, :-1].ravel(), kx[:, 1:].ravel()
    south, north = ky[:-1, :].ravel(), ky[1:, :].ravel()
    diag = west + east + south + north
    by_slot = [south, west, diag, east, north]
    offs = [(0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0)]
    return _stencil((1, n, n), offs,
                    lambda j, z, y, x: by_slot[j] if j == 2 else -by_slot[j], f"varcoeff2d_{n}")


def box125_nnz(n):
    """nnz of the boundary-truncated 5x5x5 box stencil, counted row by row from the
    per-axis neighbour counts (a cell at index i has min(i,2) + min(n-1-i,2) + 1 axis
    neighbours within distance 2, and the box is the product of three axes)."""
    i = np.arange(n)
    c = np.minimum(i, 2) + np.minimum(n - 1 - i, 2) + 1
    return int(c.sum()) ** 3


def box125(n, slab=8):
    """125-point box stencil on an n^3 grid: every cell within Chebyshev distance 2,
    diag 124, off-diag -1 (irreducibly diagonally dominant, so SPD).  Built `slab`
    z-planes at a time straight into arrays of the final size (n = 185 has 776M nonzeros),
    so the peak host memory is the CSR itself plus one slab of candidates."""
    return box_stencil(n, 2, 124.0, -1.0, slab=slab, name=f"box125_{n}")


def box_stencil(n, R, cd, co, slab=8, name=None):
    """Constant-coefficient box stencil on an n^3 grid: cd on the diagonal, co for every
    other cell within Chebyshev distance R (truncated at the boundary); rows in grid order,
    x fastest.  SPD when cd > 0 and cd >= ((2R+1)^3 - 1) |co| with co < 0."""
    offs = np.array([(dz, dy, dx) for dz in range(-R, R + 1) for dy in range(-R, R + 1) for dx in range(-R, R + 1)])
    i = np.arange(n)
    nnz = int((np.minimum(i, R) + np.minimum(n - 1 - i, R) + 1).sum()) ** 3
    N = n ** 3
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    is_diag = np.all(offs == 0, axis=1)
    pos = 0
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        z, y, x = np.meshgrid(np.arange(z0, z1), np.arange(n), np.arange(n), indexing="ij")
        z, y, x = z.ravel(), y.ravel(), x.ravel()
        nz_ = z[:, None] + offs[None, :, 0]
        ny_ = y[:, None] + offs[None, :, 1]
        nx_ = x[:, None] + offs[None, :, 2]
        ok = (nz_ >= 0) & (nz_ < n) & (ny_ >= 0) & (ny_ < n) & (nx_ >= 0) & (nx_ < n)
        # with every coordinate inside [0, n) the (dz, dy, dx) order is ascending column order
        cols = ((nz_ * n + ny_) * n + nx_)[ok]
        vals = np.where(np.broadcast_to(is_diag[None, :], ok.shape), cd, co)[ok]
        r0 = z0 * n * n
        np.cumsum(ok.sum(axis=1), out=row_ptr[r0 + 1:r0 + 1 + ok.shape[0]])
        row_ptr[r0 + 1:r0 + 1 + ok.shape[0]] += pos
        col[pos:pos + cols.size] = cols
        val[pos:pos + vals.size] = vals
        pos += cols.size
    assert pos == nnz
    return CSR(N, row_ptr, col, val, name or f"box{2 * R + 1}_{n}")


def rgg_laplacian(npts, radius, shift, seed, chunk=1 << 22):
    """Random geometric graph Laplacian + shift*I.

    Points are U[0,1)^3 from the seed; an edge joins points closer than ``radius``.
    Points are renumbered in cell-list order (cells of side >= radius, cell id
    (cz*nc + cy)*nc + cx, ties by original index).  A = L + shift*I with unit weights."""
    pts = uniform(seed, _S_POINTS, 3 * npts).reshape(npts, 3)
    nc = max(1, int(np.floor(1.0 / radius)))
    cell3 = np.minimum((pts * nc).astype(np.int64), nc - 1)
    cid = (cell3[:, 2] * nc + cell3[:, 1]) * nc + cell3[:, 0]
    order = np.argsort(cid, kind="stable")
    pts = pts[order]
    cell3 = cell3[order]
    cid = cid[order]
    counts = np.bincount(cid, minlength=nc ** 3)
    start = np.zeros(nc ** 3 + 1, dtype=np.int64)
    np.cumsum(counts, out=start[1:])
    r2 = radius * radius
    rows_l, cols_l = [], []
    # The distance test is symmetric to the last bit ((a - b)^2 == (b - a)^2 in IEEE
    # arithmetic), so only the point's own cell and the 13 neighbour cells with a positive
    # offset (in (dz, dy, dx) order) are searched, and each pair found across cells is kept in
    # both orientations: the same edge set as searching all 27 cells, at half the work.
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) < (0, 0, 0):
                    continue
                mirror = (dz, dy, dx) != (0, 0, 0)
                for lo in range(0, npts, chunk):
                    hi = min(npts, lo + chunk)
                    c = cell3[lo:hi]
                    nx_, ny_, nz_ = c[:, 0] + dx, c[:, 1] + dy, c[:, 2] + dz
                    ok = (nx_ >= 0) & (nx_ < nc) & (ny_ >= 0) & (ny_ < nc) & (nz_ >= 0) & (nz_ < nc)
                    src = np.nonzero(ok)[0] + lo
                    nb = ((nz_[ok] * nc + ny_[ok]) * nc + nx_[ok])
                    cnt = counts[nb]
                    tot = int(cnt.sum())
                    if tot == 0:
                        continue
                    i_rep = np.repeat(src, cnt)
                    base = np.repeat(start[nb] - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt)
                    j = base + np.arange(tot)
                    d = pts[i_rep] - pts[j]
                    keep = (np.einsum("ij,ij->i", d, d) < r2) & (i_rep != j)
                    rows_l.append(i_rep[keep])
                    cols_l.append(j[keep])
                    if mirror:
                        rows_l.append(cols_l[-1])
                        cols_l.append(rows_l[-2])
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    deg = np.bincount(rows, minlength=npts).astype(np.float64)
    diag_idx = np.arange(npts)
    rows = np.concatenate([rows, diag_idx])
    cols = np.concatenate([cols, diag_idx])
    vals = np.concatenate([np.full(len(rows) - npts, -1.0), deg + shift])
    o = np.argsort(rows * np.int64(npts) + cols, kind="stable")   # (row, col) pairs are unique
    rows, cols, vals = rows[o], cols[o], vals[o]
    row_ptr = np.zeros(npts + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=npts), out=row_ptr[1:])
    return CSR(npts, row_ptr, cols.astype(np.int32), vals, f"rgg_{npts}")


def _hadamard(n):
    h = np.ones((1, 1))
    while h.shape[0] < n:
        h = np.block([[h, h], [h, -h]])
    return h


def hadamard_spd(n, eigs, seed, scale_spread=1.0):
    """Dense SPD matrix A = S B S with B = Q diag(eigs) Q^T, Q a randomly signed and
    permuted normalised Hadamard matrix (n a power of 2) and S a positive diagonal.

    Every entry of Q is +-1/sqrt(n), so diag(B) = mean(eigs) for all rows and the
    Jacobi-preconditioned operator diag(A)^-1/2 A diag(A)^-1/2 equals B / mean(eigs):
    its spectrum is exactly eigs / mean(eigs)."""
    assert n & (n - 1) == 0
    eigs = np.asarray(eigs, dtype=np.float64)
    assert eigs.shape == (n,)
    h = _hadamard(n) / np.sqrt(n)
    perm = np.argsort(uniform(seed, _S_PERM, n))
    signs = np.where(uniform(seed, _S_SIGN, n) < 0.5, -1.0, 1.0)
    q = signs[:, None] * h[perm]
    b = (q * eigs) @ q.T
    b = 0.5 * (b + b.T)
    s = np.exp(scale_spread * uniform_pm1(seed, _S_SCALE, n))
    a = s[:, None] * b * s[None, :]
    a = 0.5 * (a + a.T)
    row_ptr = np.arange(0, n * n + 1, n, dtype=np.int64)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    return CSR(n, row_ptr, col, a.ravel().copy(), f"hadamard_spd_{n}"), a


def rhs_uniform(n, seed):
    """b ~ U[-1, 1) from the right-hand-side stream of ``seed``."""
    return uniform_pm1(seed, _S_RHS, n)


def xtrue_uniform(n, seed):
    """x_true ~ U[-1, 1) from the solution stream of ``seed``."""
    return uniform_pm1(seed, _S_XTRUE, n)


def batch_mix(count, seed, lo=1e3, hi=2e5):
    """Specs of a ragged batch: sizes log-uniform in [lo, hi], half 2-D (n = round(sqrt R))
    and half 3-D (n = round(cbrt R)) variable-coefficient stencils.  Returns a list of
    (family, n, matrix_seed, rhs_seed)."""
    u = uniform(seed, _S_SIZES, count)
    f = uniform(seed, _S_FAMILY, count)
    specs = []
    for i in range(count):
        r = np.exp(np.log(lo) + u[i] * (np.log(hi) - np.log(lo)))
        if f[i] < 0.5:
            specs.append(("varcoeff2d", max(2, int(round(np.sqrt(r)))), seed * 7919 + 2 * i, seed * 7919 + 2 * i + 1))
        else:
            specs.append(("varcoeff3d", max(2, int(round(np.cbrt(r)))), seed * 7919 + 2 * i, seed * 7919 + 2 * i + 1))
    return specs


def serving_mix(count, seed, lo=1e3, hi=4e6, rgg_radius_deg=14.0):
    """Specs of a serving request stream: sizes log-uniform in [lo, hi], family uniform
    over {varcoeff2d, varcoeff3d, rgg}.  RGG radius keeps the expected interior degree
    at ``rgg_radius_deg``.  Returns (family, size_param, matrix_seed, rhs_seed)."""
    u = uniform(seed, _S_SIZES, count)
    f = uniform(seed, _S_FAMILY, count)
    specs = []
    for i in range(count):
        r = np.exp(np.log(lo) + u[i] * (np.log(hi) - np.log(lo)))
        ms, rs = seed * 104729 + 2 * i, seed * 104729 + 2 * i + 1
        if f[i] < 1.0 / 3.0:
            specs.append(("varcoeff2d", max(2, int(round(np.sqrt(r)))), ms, rs))
        elif f[i] < 2.0 / 3.0:
            specs.append(("varcoeff3d", max(2, int(round(np.cbrt(r)))), ms, rs))
        else:
            specs.append(("rgg", int(round(r)), ms, rs))
    return specs


def build_spec(spec, rgg_degree=14.0, rgg_shift=1e-3):
    """Materialise one (family, size, matrix_seed, rhs_seed) spec -> (CSR, b)."""
    fam, size, ms, rs = spec
    if fam == "varcoeff2d":
        a = varcoeff2d(size, ms)
    elif fam == "varcoeff3d":
        a = varcoeff3d(size, ms)
    elif fam == "rgg":
        radius = (3.0 * rgg_degree / (4.0 * np.pi * size)) ** (1.0 / 3.0)
        a = rgg_laplacian(size, radius, rgg_shift, ms)
    else:
        raise ValueError(fam)
    return a, rhs_uniform(a.n, rs)
