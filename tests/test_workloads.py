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


def test_bench_algorithmic_cost_of_the_basis_kernels():
    """The per-launch algorithmic bytes and FP64 flops that bench.py divides by the
    measured launch time, for the 3D convection-diffusion 200^3 workload (m = 100,
    k = 4, SRHT s = 400): SpMV + window dots 12 nnz + 4(n+1) + 8 n k + 8 n bytes and
    2 nnz + 2 n k flops; window update + sketch 8 n (k + 2) + 8 s chunks bytes and
    2 n k + 2 n flops."""
    import bench

    n, nnz = 8_000_000, 55_760_000
    assert W.convdiff_nnz(3, 200) == nnz
    cost = bench.algorithmic_cost(n, nnz, 100, 4, 400)
    sp_b, sp_f = cost["spmv_dots"]
    up_b, up_f = cost["update"]
    assert sp_b == 12 * nnz + 4 * (n + 1) + 8 * n * 4 + 8 * n == 1_021_120_004
    assert sp_f == 2 * nnz + 2 * n * 4 == 175_520_000
    chunks = (n + 4095) // 4096
    assert up_b == 8 * n * 6 + 8 * 400 * chunks
    assert up_f == 2 * n * 4 + 2 * n == 80_000_000
