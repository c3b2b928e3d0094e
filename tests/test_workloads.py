"""Seeded input generators (no GPU): structure the method's inputs must have."""
import numpy as np
import scipy.sparse as sp

from paper_2212_12758_gb300 import workloads as W


def test_convdiff_stencil_and_nnz_closed_form():
    for dim, N in ((2, 7), (2, 30), (3, 5), (3, 11)):
        A = W.convdiff(dim, N)
        assert A.n == N**dim and A.nnz == W.convdiff_nnz(dim, N)
        S = W.to_scipy(A)
        h = 1.0 / (N + 1)
        diag = 2 * dim / h**2 + 10.0 * dim / h
        assert np.allclose(S.diagonal(), diag)
        # an interior row: 2 dim/h^2 + sum(c)/h on the diagonal, -1/h^2 - c_i/h below and
        # -1/h^2 above in each direction, so the row sums to zero
        r = (N // 2) * (1 + (N if dim >= 2 else 0) + (N * N if dim == 3 else 0))
        assert abs(S[r].sum()) < 1e-6 * diag
        # columns sorted within every row
        for i in range(0, A.n, max(1, A.n // 50)):
            c = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
            assert np.all(np.diff(c) > 0)


def test_chung_lu_laplacian_is_shifted_laplacian():
    A = W.chung_lu_laplacian(5000, seed=2)
    S = W.to_scipy(A)
    assert (S != S.T).nnz == 0  # symmetric
    assert np.allclose(S @ np.ones(A.n), 0.1)  # L 1 = 0, so A 1 = 0.1 * 1
    off = S - sp.diags(S.diagonal())
    assert np.all(off.data == -1.0)  # unweighted, no self-loops off the diagonal
    deg = -off.sum(axis=1).A.ravel()
    assert 6.0 < deg.mean() <= 10.0  # duplicates and self-loops dropped from the mean-10 draw
    assert deg[:50].mean() > 20 * np.median(deg)  # power-law head


def test_batch_specs_and_arrivals_ranges():
    specs = W.batch_specs(256, seed=3)
    ns = np.array([it.N**2 for it in specs])
    assert ns.min() >= 0.9e4 and ns.max() <= 1.01e6
    assert all(1e-4 <= it.t <= 1e-2 and 20 <= it.m <= 80 for it in specs)
    assert W.batch_specs(256, seed=3) == specs  # seeded
    arr = W.poisson_arrivals(2000.0, 20000, seed=4)
    assert np.all(np.diff(arr) > 0)
    assert abs(20000 / arr[-1] - 2000.0) < 60.0
