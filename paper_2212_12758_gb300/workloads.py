"""Seeded synthetic inputs shaped like the test problems of arXiv 2212.12758 §5.

This module only builds inputs (sparse matrices in CSR form, starting vectors,
batch and arrival descriptors). It holds none of the f(A)b method's
arithmetic, imports only numpy, and is shared by the CUDA path's tests and
benchmarks and by the CPU oracle's callers.

Matrices (the paper's §5 uses convection-diffusion operators, graph
Laplacians and a 3D Laplacian; the exact discretisations it cites are not in
the paper, so the schemes below are this library's stated choice):

* ``convdiff``: scaled finite differences on the unit square/cube, h = 1/(N+1),
  homogeneous Dirichlet boundary, A = -d*Laplace_h + c . grad_h with first-order
  upwind differences for c > 0 (backward difference in each direction).
  Unknowns are in lexicographic order with x fastest. Row r has, in increasing
  column order, the entries (down, south, west, diag, east, north, up):
  diag = 2*dim*d/h^2 + sum(c)/h, west/south/down = -d/h^2 - c_axis/h,
  east/north/up = -d/h^2.
* ``chung_lu_laplacian``: unweighted symmetric Chung-Lu graph with power-law
  expected degrees, A = L + shift*I with L = D - W.
* ``laplacian3d``: T_N (x) I (x) I + I (x) T_N (x) I + I (x) I (x) T_N with
  T_N = tridiag(-1, 2, -1) (the 3D Laplacian of §5.1.4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A square sparse matrix in CSR form (int64 row pointers, int32 columns,
    float64 values, columns sorted within each row)."""

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _stencil_csr(n: int, offsets, coeffs, valid_masks) -> CSR:
    """Assemble CSR from per-row stencil entries given in increasing column order."""
    width = len(offsets)
    idx = np.arange(n, dtype=np.int64)
    cols = np.empty((n, width), dtype=np.int32)
    vals = np.empty((n, width), dtype=np.float64)
    mask = np.empty((n, width), dtype=bool)
    for e, (off, coef, valid) in enumerate(zip(offsets, coeffs, valid_masks)):
        cols[:, e] = (idx + off).astype(np.int32, copy=False) if valid is not None else idx.astype(np.int32)
        vals[:, e] = coef  # a scalar or one value per row
        mask[:, e] = True if valid is None else valid
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[mask]
    values = vals[mask]
    return CSR(n=n, rowptr=rowptr, colind=np.ascontiguousarray(colind), vals=np.ascontiguousarray(values))


def convdiff(dim: int, N: int, d: float = 1.0, c=None) -> CSR:
    """Upwind convection-diffusion matrix on an N^dim grid (see module docstring)."""
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if c is None:
        c = (10.0,) * dim
    c = tuple(float(x) for x in c)
    if len(c) != dim or min(c) < 0:
        raise ValueError("c must have dim non-negative entries")
    h = 1.0 / (N + 1)
    n = N ** dim
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    diag = 2 * dim * d / h**2 + sum(c) / h
    lower = [-d / h**2 - ca / h for ca in c]  # west, south, down
    upper = -d / h**2  # east, north, up
    if dim == 2:
        offsets = (-N, -1, 0, 1, N)
        coeffs = (lower[1], lower[0], diag, upper, upper)
        masks = (iy > 0, ix > 0, None, ix < N - 1, iy < N - 1)
    else:
        iz = idx // (N * N)
        NN = N * N
        offsets = (-NN, -N, -1, 0, 1, N, NN)
        coeffs = (lower[2], lower[1], lower[0], diag, upper, upper, upper)
        masks = (iz > 0, iy > 0, ix > 0, None, ix < N - 1, iy < N - 1, iz < N - 1)
    return _stencil_csr(n, offsets, coeffs, masks)


def convdiff_skew(N: int, Pe: float = 200.0, d_in: float = 1000.0) -> CSR:
    """The convection-diffusion operator of the paper's first experiment (§5.1.1),
    on an N x N interior grid of the unit square (h = 1/(N+1), Dirichlet):
    L[u] = -(D1 u_x)_x - (D2 u_y)_y + Pe (1/2 (v1 u_x + v2 u_y) + 1/2 ((v1 u)_x + (v2 u)_y)),
    D1 = d_in on [0.25, 0.75]^2 and 1 elsewhere, D2 = D1 / 2, v = (x + y, x - y).

    Discretisation (not given in the paper; this module's choice): diffusion by
    the conservative 5-point scheme with D evaluated at the cell-face midpoints;
    convection in the printed skew-symmetric form with central differences, which
    makes the convection part of the matrix exactly skew-symmetric:
    A[i, i+1] = Pe (v_i + v_{i+1}) / (4h) = -A[i+1, i] along each axis.
    Rows in lexicographic order, x fastest, columns sorted."""
    h = 1.0 / (N + 1)
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = idx // N
    x = (ix + 1) * h
    y = (iy + 1) * h

    def D1(px, py):
        inside = (px >= 0.25) & (px <= 0.75) & (py >= 0.25) & (py <= 0.75)
        return np.where(inside, d_in, 1.0)

    dxp = D1(x + h / 2, y)
    dxm = D1(x - h / 2, y)
    dyp = D1(x, y + h / 2) / 2
    dym = D1(x, y - h / 2) / 2
    v1 = x + y
    v2 = x - y
    v1p, v1m = v1 + h, v1 - h  # v1 at the east / west neighbours
    v2p, v2m = v2 - h, v2 + h  # v2 at the north / south neighbours (v2 = x - y)
    c = Pe / (4 * h)
    diag = (dxp + dxm + dyp + dym) / h**2
    east = -dxp / h**2 + c * (v1 + v1p)
    west = -dxm / h**2 - c * (v1 + v1m)
    north = -dyp / h**2 + c * (v2 + v2p)
    south = -dym / h**2 - c * (v2 + v2m)
    offsets = (-N, -1, 0, 1, N)
    coeffs = (south, west, diag, east, north)
    masks = (iy > 0, ix > 0, None, ix < N - 1, iy < N - 1)
    return _stencil_csr(n, offsets, coeffs, masks)


def sine_vector(N: int) -> np.ndarray:
    """sin(pi x) sin(pi y) on the N x N interior grid, normalised (§5.1.1)."""
    h = 1.0 / (N + 1)
    t = np.sin(np.pi * h * np.arange(1, N + 1))
    b = np.outer(t, t).ravel()  # row iy, column ix: x fastest
    return b / np.linalg.norm(b)


def convdiff_nnz(dim: int, N: int) -> int:
    """Closed-form nonzero count of ``convdiff``: 5N^2-4N (2D), 7N^3-6N^2 (3D)."""
    return 5 * N * N - 4 * N if dim == 2 else 7 * N**3 - 6 * N * N


def laplacian3d(N: int) -> CSR:
    """3D Laplacian with T_N = tridiag(-1, 2, -1) in each direction."""
    n = N**3
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    iz = idx // (N * N)
    NN = N * N
    offsets = (-NN, -N, -1, 0, 1, N, NN)
    coeffs = (-1.0, -1.0, -1.0, 6.0, -1.0, -1.0, -1.0)
    masks = (iz > 0, iy > 0, ix > 0, None, ix < N - 1, iy < N - 1, iz < N - 1)
    return _stencil_csr(n, offsets, coeffs, masks)


def chung_lu_laplacian(n: int, exponent: float = 2.5, mean_degree: float = 10.0,
                       shift: float = 0.1, seed: int = 2) -> CSR:
    """Shifted Laplacian L + shift*I of a Chung-Lu graph with power-law degrees.

    Expected degrees w_i proportional to (i+1)^(-1/(exponent-1)), scaled to the
    requested mean and capped at sqrt(sum w). round(n*mean/2) edges are drawn
    with both endpoints chosen proportionally to w; self-loops and duplicate
    edges are dropped; the graph is unweighted and symmetric.
    """
    rng = np.random.default_rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    w *= mean_degree / w.mean()
    w = np.minimum(w, math.sqrt(w.sum()))
    p = w / w.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    E = int(round(n * mean_degree / 2))
    a = np.searchsorted(cdf, rng.random(E), side="right").astype(np.int64)
    b = np.searchsorted(cdf, rng.random(E), side="right").astype(np.int64)
    np.minimum(a, n - 1, out=a)
    np.minimum(b, n - 1, out=b)
    keep = a != b
    a, b = a[keep], b[keep]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = np.unique(lo * n + hi)
    lo = key // n
    hi = key % n
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    deg = np.bincount(rows, minlength=n).astype(np.float64)
    # add the diagonal entries
    rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    vals = np.concatenate([-np.ones(2 * len(lo)), deg + shift])
    order = np.argsort(rows * n + cols)  # (row, col) pairs are distinct: row-major order
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n=n, rowptr=rowptr, colind=cols.astype(np.int32), vals=vals.astype(np.float64))


def random_vector(n: int, seed: int = 0, normalize: bool = True) -> np.ndarray:
    """b ~ N(0, 1) from numpy's default generator with the given seed."""
    b = np.random.default_rng(seed).standard_normal(n)
    if normalize:
        b /= np.linalg.norm(b)
    return b


def diagonal(d: np.ndarray) -> CSR:
    """Diagonal matrix diag(d) in CSR form."""
    n = len(d)
    return CSR(n=n, rowptr=np.arange(n + 1, dtype=np.int64), colind=np.arange(n, dtype=np.int32),
               vals=np.asarray(d, dtype=np.float64).copy())


def from_dense(M: np.ndarray) -> CSR:
    """CSR of the nonzeros of a dense square matrix."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    rows, cols = np.nonzero(M)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n=n, rowptr=rowptr, colind=cols.astype(np.int32), vals=M[rows, cols].copy())


def to_scipy(A: CSR):
    """scipy.sparse view of a CSR (for callers that hold scipy)."""
    import scipy.sparse as sp

    return sp.csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n))


@dataclass
class BatchItem:
    N: int
    t: float
    m: int


def batch_specs(count: int = 256, seed: int = 3, n_lo: float = 1e4, n_hi: float = 1e6,
                t_lo: float = 1e-4, t_hi: float = 1e-2, m_lo: int = 20, m_hi: int = 80):
    """Uneven batch of 2D convection-diffusion solves: n log-uniform on
    [n_lo, n_hi] (grid side N = round(sqrt(n))), t log-uniform on [t_lo, t_hi]
    (f = exp(-tA)), m uniform on {m_lo..m_hi}."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))
    ts = np.exp(rng.uniform(math.log(t_lo), math.log(t_hi), count))
    ms = rng.integers(m_lo, m_hi + 1, count)
    return [BatchItem(N=int(round(math.sqrt(nv))), t=float(tv), m=int(mv)) for nv, tv, mv in zip(ns, ts, ms)]


def poisson_arrivals(rate_per_s: float, count: int, seed: int = 4) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given mean rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))
