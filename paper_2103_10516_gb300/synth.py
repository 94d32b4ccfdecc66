"""Seeded synthetic inputs shaped like the workloads of Hallman & Troester, Section 5.

This module only builds matrices (CSR arrays) from a seed.  It holds none of the
estimator's arithmetic, so both the CUDA path and the CPU oracle may take their
inputs from it.  Every generator is deterministic for a given seed (numpy PCG64).

CSR convention used everywhere in this project:
  rowptr : int64[nrows + 1]
  col    : int32[nnz], sorted ascending inside each row, no duplicates
  val    : float64[nnz] or None (pattern-only 0/1 matrix)
"""
from __future__ import annotations

import numpy as np


class CSR:
    """A plain CSR matrix (host numpy arrays)."""

    def __init__(self, nrows, ncols, rowptr, col, val=None):
        self.nrows = int(nrows)
        self.ncols = int(ncols)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = None if val is None else np.ascontiguousarray(val, dtype=np.float64)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self):
        a = np.zeros((self.nrows, self.ncols))
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        a[rows, self.col] = 1.0 if self.val is None else self.val
        return a


def _sorted_unique(key):
    """Sorted distinct values of an int64 array (sort + adjacent compare)."""
    key = np.sort(key)
    if key.size == 0:
        return key
    keep = np.empty(key.size, dtype=bool)
    keep[0] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    return key[keep]


def _from_coo(nrows, ncols, r, c, v=None):
    """Sort COO entries by (row, col) and build a CSR.  Duplicates must already be gone."""
    key = r.astype(np.int64) * np.int64(ncols) + c.astype(np.int64)
    order = np.argsort(key, kind="stable")
    r = r[order]
    c = c[order]
    counts = np.bincount(r, minlength=nrows).astype(np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(nrows, ncols, rowptr, c.astype(np.int32), None if v is None else v[order])


def grid_laplacian_2d(nx: int, ny: int | None = None, shift: float = 0.0) -> CSR:
    """5-point Dirichlet Laplacian on an nx-by-ny grid, stencil [4, -1], plus shift*I.

    Row index of grid point (x, y) is y*nx + x.  The log-det workload of Section 5.3
    (Table of log-determinant estimates) uses SPD matrices of this kind; the 64x64
    grid with shift 0.1 has d = 4096 and nnz = 20,224.
    """
    ny = nx if ny is None else ny
    d = nx * ny
    idx = np.arange(d, dtype=np.int64)
    x = idx % nx
    y = idx // nx
    rows = [idx]
    cols = [idx]
    vals = [np.full(d, 4.0 + shift)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + dy * nx)
        vals.append(np.full(int(ok.sum()), -1.0))
    return _from_coo(d, d, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def rmat_edges(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed=0):
    """Directed R-MAT edge list (Chakrabarti, Zhan, Faloutsos 2004), no noise.

    2**scale vertices, edge_factor * 2**scale edges; at every one of the `scale`
    recursion levels each edge picks quadrant (0,0), (0,1), (1,0), (1,1) with
    probabilities a, b, c, 1-a-b-c.  Generated in chunks to bound host memory.
    """
    rng = np.random.default_rng(seed)
    m = edge_factor << scale
    src = np.empty(m, dtype=np.int64)
    dst = np.empty(m, dtype=np.int64)
    chunk = 1 << 22
    ab = a + b
    abc = a + b + c
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        u = np.zeros(e - s, dtype=np.int64)
        v = np.zeros(e - s, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(e - s)
            bit_u = r >= ab                       # quadrants c, d
            bit_v = ((r >= a) & (r < ab)) | (r >= abc)  # quadrants b, d
            u = (u << 1) | bit_u
            v = (v << 1) | bit_v
        src[s:e] = u
        dst[s:e] = v
    return src, dst


def rmat_adjacency(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed=0) -> CSR:
    """Symmetric 0/1 adjacency (pattern-only CSR) of an R-MAT graph.

    Edges are symmetrised, self-loops and duplicate edges removed, as for the
    triangle-counting workload of Section 5.4.
    """
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, a, b, c, seed)
    keep = src != dst
    src = src[keep]
    dst = dst[keep]
    key = np.concatenate([src * n + dst, dst * n + src])
    del src, dst
    key = _sorted_unique(key)
    r = key // n
    cc = key % n
    counts = np.bincount(r, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, n, rowptr, cc.astype(np.int32), None)


def random_graph(d: int, p: float, seed=0) -> CSR:
    """Erdos-Renyi G(d, p) symmetric 0/1 adjacency without self-loops."""
    rng = np.random.default_rng(seed)
    upper = np.triu(rng.random((d, d)) < p, 1)
    adj = upper | upper.T
    r, c = np.nonzero(adj)
    return _from_coo(d, d, r, c, None)


def complete_graph(d: int) -> CSR:
    adj = ~np.eye(d, dtype=bool)
    r, c = np.nonzero(adj)
    return _from_coo(d, d, r, c, None)


def random_symmetric(d: int, density: float, seed=0, diag_shift=0.0) -> CSR:
    """Random sparse symmetric matrix with N(0,1) entries plus diag_shift*I (small tests)."""
    rng = np.random.default_rng(seed)
    m = rng.random((d, d)) < density
    vals = rng.standard_normal((d, d))
    a = np.where(m, vals, 0.0)
    a = np.triu(a, 1)
    a = a + a.T + np.diag(rng.standard_normal(d) + diag_shift)
    r, c = np.nonzero(a)
    return _from_coo(d, d, r, c, a[r, c])


def sparse_gaussian(nrows: int, ncols: int, density: float, seed=0) -> CSR:
    """Rectangular X with uniformly placed nonzeros (positions drawn without
    replacement, count Binomial(nrows*ncols, density)) and N(0,1) values; the
    nuclear-norm workload of Section 5.3 applies A = X^T X."""
    rng = np.random.default_rng(seed)
    total = nrows * ncols
    k = int(rng.binomial(total, density))
    pos = _sorted_unique(rng.integers(0, total, size=k, dtype=np.int64))
    while pos.size < k:
        extra = rng.integers(0, total, size=k - pos.size, dtype=np.int64)
        pos = _sorted_unique(np.concatenate([pos, extra]))
    vals = rng.standard_normal(pos.size)
    r = pos // ncols
    c = pos % ncols
    counts = np.bincount(r, minlength=nrows).astype(np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(nrows, ncols, rowptr, c.astype(np.int32), vals)


def diffusion_3d(s: int, sigma: float = 1.0, shift: float = 0.0, seed=0) -> CSR:
    """7-point 3D diffusion operator on an s^3 grid with lognormal cell
    coefficients kappa = exp(sigma * N(0,1)), face coefficients the harmonic mean
    of the two cells, Dirichlet boundary (boundary faces use the cell's own
    kappa), plus shift*I.  SPD; used for the batched log-det workload."""
    rng = np.random.default_rng(seed)
    d = s * s * s
    kap = np.exp(sigma * rng.standard_normal(d))
    idx = np.arange(d, dtype=np.int64)
    x = idx % s
    y = (idx // s) % s
    z = idx // (s * s)
    diag = np.full(d, float(shift))
    rows = []
    cols = []
    vals = []
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        nb_ok = (x + dx >= 0) & (x + dx < s) & (y + dy >= 0) & (y + dy < s) & (z + dz >= 0) & (z + dz < s)
        nb = idx + dx + dy * s + dz * s * s
        face = np.where(nb_ok, 2.0 * kap * kap[np.where(nb_ok, nb, idx)] /
                        (kap + kap[np.where(nb_ok, nb, idx)]), kap)
        diag += face
        rows.append(idx[nb_ok])
        cols.append(nb[nb_ok])
        vals.append(-face[nb_ok])
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return _from_coo(d, d, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))

