"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: relative 2-norm <= 1e-10 for f(A)b (the library's FP64 target);
H, the sketch and y are compared element-wise at the precision their
arithmetic allows (a sketch entry carries the int64 block-transform rounding,
relative 2^-49 of a 4096-row chunk's largest entry, so 1e-13 relative to the
column norm). Sketch supports and signs are compared exactly.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import krylov, matfun
from oracle import sketch as osk
from paper_2212_12758_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


@pytest.fixture(scope="module")
def torch():
    import torch as t

    assert t.cuda.is_available()
    return t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --------------------------------------------------------------- sketches
@pytest.mark.parametrize("n", [300, 4096, 9000])
@pytest.mark.parametrize("kind,s", [(osk.SPARSE_SIGN, 48), (osk.SRHT, 40)])
def test_sketch_matrix_bit_exact(fab, torch, n, kind, s):
    """Theta e_j for every j reveals the sketch: supports and signs exactly, values to rounding."""
    cols = np.arange(n) if n <= 4096 else np.r_[np.arange(0, 4200), np.arange(n - 700, n)]
    V = torch.zeros((len(cols), n), dtype=torch.float64, device="cuda")
    V[torch.arange(len(cols)), torch.from_numpy(cols).cuda()] = 1.0
    out = fab.sketch_apply(V, s, sketch=kind, zeta=8, seed=5).cpu().numpy().T  # s x ncols
    th = osk.make(kind, n, s, 5, 8)
    ref = th.dense()[:, cols]
    assert np.array_equal(np.sign(out), np.sign(ref))
    assert np.array_equal(out != 0, ref != 0)
    assert np.allclose(out, ref, rtol=1e-15, atol=0)


@pytest.mark.parametrize("zeta,s", [(1, 300), (16, 20), (5, 97)])
def test_sparse_table_sketch_of_the_basis(fab, torch, zeta, s):
    """A solve's sparse-sign sketch comes from the transposed per-chunk table (gather):
    Theta v_j of the library's own basis (n = 4900: a full and a partial chunk) against
    the oracle's sketch of the same vectors, for short and long lists."""
    A = W.convdiff(2, 70)
    b = W.random_vector(A.n, 3)
    m = 12
    M = fab.Matrix.from_csr(A)
    M.apply(torch.from_numpy(b).cuda(), fab.params(f=fab.EXP, t=-0.01, m=m, k=2, s=s, zeta=zeta,
                                                   sketch=fab.SPARSE_SIGN, seed=9, method=fab.SKETCHED_FAST))
    V = M.last_basis()  # n x (m+1), v_j = sigma_j W_j
    SV = M.last_state().SV  # s x (m+1)
    ref = osk.make(osk.SPARSE_SIGN, A.n, s, 9, zeta).apply(V)
    for j in range(m + 1):
        assert np.max(np.abs(SV[:, j] - ref[:, j])) <= 1e-13 * np.linalg.norm(V[:, j]), j


@pytest.mark.parametrize("n", [1000, 12345, 70000])
@pytest.mark.parametrize("kind,s", [(osk.SPARSE_SIGN, 160), (osk.SRHT, 400)])
def test_sketch_random_vectors(fab, torch, n, kind, s):
    rng = np.random.default_rng(n)
    Vh = rng.standard_normal((3, n)) * np.array([[1.0], [1e-7], [3e5]])
    Vh[2, ::3] *= 1e-9  # wide dynamic range inside chunks
    out = fab.sketch_apply(torch.from_numpy(Vh).cuda(), s, sketch=kind, zeta=8, seed=2).cpu().numpy()
    th = osk.make(kind, n, s, 2, 8)
    ref = th.apply(Vh.T).T
    for j in range(3):
        assert np.max(np.abs(out[j] - ref[j])) <= 1e-13 * np.linalg.norm(Vh[j])


# ---------------------------------------------------------- whole methods
def _c1():
    A = W.convdiff(2, 100)
    return A, W.random_vector(A.n, 0)


def _run_gpu(fab, torch, A, b, **kw):
    M = fab.Matrix.from_csr(A)
    p = fab.params(**kw)
    x, st = M.apply(torch.from_numpy(b).cuda(), p, stats=True)
    return M, x.cpu().numpy(), st


METHODS = [(krylov.ARNOLDI, "arnoldi"), (krylov.SKETCHED_LS, "sketched_ls"), (krylov.SKETCHED_FAST, "sketched_fast"),
           (krylov.NOPROJ, "noproj")]


@pytest.mark.parametrize("method,name", METHODS)
def test_c1_convdiff_exp_all_methods(fab, torch, method, name):
    """2D convection-diffusion 100x100, exp(-0.01 A) b, m = 40, k = 2, sparse sign s = 160, zeta = 8."""
    A, b = _c1()
    As = W.to_scipy(A)
    m, k, s, t = 40, 2, 160, -0.01
    th = osk.make(osk.SPARSE_SIGN, A.n, s, 1, 8)
    ref = krylov.run(method, As, b, m, k, matfun.EXP, th, t, tol=1e-14)
    M, x, st = _run_gpu(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, s=s, zeta=8, sketch=fab.SPARSE_SIGN, seed=1,
                        method=method, lsqr_tol=1e-14)
    assert st.m_used == m
    assert _rel(x, ref.x) <= TOL, name
    ls = M.last_state()
    B = ref.basis
    assert np.allclose(ls.H, B.H, rtol=0, atol=1e-11 * np.abs(B.H).max())
    if method in (krylov.SKETCHED_FAST, krylov.SKETCHED_LS):
        SVref = th.apply(B.V)
        assert np.max(np.abs(ls.SV - SVref)) <= 1e-12
        assert _rel(ls.y, ref.y) <= 1e-9
    assert _rel(ls.coeffs, ref.coeffs) <= TOL


@pytest.mark.parametrize("method", [krylov.SKETCHED_FAST, krylov.SKETCHED_LS, krylov.NOPROJ, krylov.ARNOLDI])
def test_ragged_3d_srht_k4(fab, torch, method):
    """3D convection-diffusion 23^3 (n = 12167, not a multiple of the 4096-row chunk), k = 4, SRHT."""
    A = W.convdiff(3, 23)
    b = W.random_vector(A.n, 3)
    m, k, s, t = 30, 4, 90, -1e-3
    th = osk.make(osk.SRHT, A.n, s, 7, 8)
    ref = krylov.run(method, W.to_scipy(A), b, m, k, matfun.EXP, th, t, tol=1e-14)
    _, x, st = _run_gpu(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=7, method=method,
                        lsqr_tol=1e-14)
    assert _rel(x, ref.x) <= TOL


@pytest.mark.parametrize("method", [krylov.SKETCHED_FAST, krylov.NOPROJ])
def test_wide_window_k8_h_and_sketch(fab, torch, method):
    """Window k = 8, the largest: the first steps run every window width 1..8, so the
    SpMV's in-warp reduction of the kw window dots runs both with and without zero
    padding (kw = 3, 5, 6, 7 are padded). H and the sketch of the basis against the
    oracle; 3D convection-diffusion 23^3 (ragged last chunk), SRHT."""
    A = W.convdiff(3, 23)
    b = W.random_vector(A.n, 5)
    m, k, s, t = 24, 8, 100, -1e-3
    th = osk.make(osk.SRHT, A.n, s, 3, 8)
    ref = krylov.run(method, W.to_scipy(A), b, m, k, matfun.EXP, th, t, tol=1e-14)
    M, x, st = _run_gpu(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=3, method=method)
    assert st.m_used == m
    assert _rel(x, ref.x) <= TOL
    ls = M.last_state()
    B = ref.basis
    assert np.allclose(ls.H, B.H, rtol=0, atol=1e-11 * np.abs(B.H).max())
    if method == krylov.SKETCHED_FAST:
        assert np.max(np.abs(ls.SV - th.apply(B.V))) <= 1e-12


@pytest.mark.parametrize("f", [matfun.SQRT, matfun.INVSQRT])
@pytest.mark.parametrize("method", [krylov.SKETCHED_FAST, krylov.ARNOLDI, krylov.NOPROJ])
def test_graph_laplacian_sqrt(fab, torch, f, method):
    """Shifted Chung-Lu Laplacian (power-law degrees), f = sqrt and inverse sqrt, m = 30, k = 2."""
    A = W.chung_lu_laplacian(20000, seed=2)
    b = W.random_vector(A.n, 0)
    m, k, s = 30, 2, 120
    th = osk.make(osk.SRHT, A.n, s, 1, 8)
    ref = krylov.run(method, W.to_scipy(A), b, m, k, f, th, 1.0)
    _, x, _ = _run_gpu(fab, torch, A, b, f=f, m=m, k=k, s=s, sketch=fab.SRHT, seed=1, method=method)
    assert _rel(x, ref.x) <= TOL


def test_breakdown_invariant_subspace(fab, torch):
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 5.0], 40)
    A = W.diagonal(d)
    b = W.random_vector(len(d), 2)
    for method in (fab.ARNOLDI, fab.SKETCHED_FAST, fab.SKETCHED_LS, fab.NOPROJ):
        _, x, st = _run_gpu(fab, torch, A, b, f=fab.EXP, t=-0.3, m=8, k=2, s=16, sketch=fab.SRHT, seed=1,
                            method=method)
        assert st.m_used == 5
        assert _rel(x, np.exp(-0.3 * d) * b) <= 1e-9


def test_zero_rhs_and_invalid_params(fab, torch):
    A, _ = _c1()
    M = fab.Matrix.from_csr(A)
    x = M.apply(np.zeros(A.n), fab.params(m=10, s=40))
    assert not np.any(x)
    with pytest.raises(fab.FabError) as e:
        M.apply(np.ones(A.n), fab.params(m=10, s=5))  # s < m + 1
    assert e.value.code == fab.FAB_EINVAL
    with pytest.raises(fab.FabError):
        M.apply(np.ones(A.n), fab.params(m=10, k=0))
    with pytest.raises(fab.FabError):
        M.apply(np.ones(A.n), fab.params(m=10, precision=7))
    with pytest.raises(fab.FabError):  # the Gaussian sketch needs the mixed-precision path
        M.apply(np.ones(A.n), fab.params(m=10, sketch=fab.GAUSSIAN))
    bad = np.ones(A.n)
    bad[7] = np.nan
    with pytest.raises(fab.FabError) as e:
        M.apply(bad, fab.params(m=10, s=40))
    assert e.value.code == fab.FAB_ENUMERIC


def test_host_and_device_buffers_agree_and_are_deterministic(fab, torch):
    A, b = _c1()
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=fab.EXP, t=-0.01, m=40, k=2, s=160, sketch=fab.SPARSE_SIGN, seed=1)
    x1 = M.apply(b, p)
    x2 = M.apply(torch.from_numpy(b).cuda(), p).cpu().numpy()
    x3 = M.apply(b, p)
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)


def test_mgs_vs_cgs_window_reading(fab, torch):
    """The library orthogonalises the window by one classical pass; the modified
    sequence printed in Alg. 2 agrees to rounding (reported, loose bound)."""
    A, b = _c1()
    th = osk.make(osk.SPARSE_SIGN, A.n, 160, 1, 8)
    mgs = krylov.sketched_fast(W.to_scipy(A), b, 40, 2, matfun.EXP, th, -0.01, orth="mgs", form="sketch_solve")
    _, x, _ = _run_gpu(fab, torch, A, b, f=fab.EXP, t=-0.01, m=40, k=2, s=160, sketch=fab.SPARSE_SIGN, seed=1)
    assert _rel(x, mgs.x) <= 1e-8


# ------------------------------------------------ full-size (bench) workload
def _golden_c2():
    """The oracle's C2 solve as stored by tests/golden/make_c2_reference.py."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_sketched_fast.txt")
    out = {"x": {}}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        if key == "x":
            out["x"][int(vals[0])] = float(vals[1])
        elif key == "coeffs":
            out["coeffs"] = np.array([float(v) for v in vals])
        else:
            out[key] = float(vals[0])
    return out


@pytest.mark.slow
def test_c2_full_size_against_the_oracle(fab, torch):
    """The bench workload at full size: 3D convection-diffusion 200^3 (n = 8.0M,
    nnz = 55.76M), exp(-1e-3 A) b, m = 100, k = 4, SRHT s = 400, sketched_fast (Remark
    after eq. sFOM), FP64. The oracle runs the whole solve on the host: x at 1e-10
    relative 2-norm, the coefficient vector c and H element by element; the stored
    oracle solve (coefficients and sampled entries, tests/golden/) agrees too; the
    Arnoldi-like relation A V_m = V_{m+1} H_m (eq. arnoldilike) holds on sampled rows."""
    A = W.convdiff(3, 200)
    assert A.nnz == W.convdiff_nnz(3, 200)
    b = W.random_vector(A.n, 0)
    As = W.to_scipy(A)
    m, k, s, t = 100, 4, 400, -1e-3
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=1, method=fab.SKETCHED_FAST)
    bd = torch.from_numpy(b).cuda()
    x, st = M.apply(bd, p, stats=True)
    x = x.cpu().numpy()
    assert st.m_used == m
    ls = M.last_state()
    gold = _golden_c2()
    idx = np.array(sorted(gold["x"]))
    xs = np.array([gold["x"][i] for i in idx])
    assert _rel(x[idx], xs) <= TOL
    assert _rel(ls.coeffs, gold["coeffs"]) <= TOL
    ref = krylov.sketched_fast(As, b, m, k, matfun.EXP, osk.SRHT_(A.n, s, 1), t, form="sketch_solve")
    print(f"\nC2 full size: rel err vs oracle {_rel(x, ref.x):.3e}, kappa_est {st.kappa_est:.3e}")
    assert _rel(x, ref.x) <= TOL
    assert _rel(ls.coeffs, ref.coeffs) <= TOL
    H_ref = ref.basis.H
    assert np.max(np.abs(ls.H - H_ref)) <= 1e-11 * np.abs(H_ref).max()
    del ref
    # Arnoldi-like relation on sampled rows of the GPU basis
    V = torch.empty((m + 1, A.n), dtype=torch.float64, device="cuda")
    assert fab.lib.fab_last_basis(M._h, V.data_ptr(), 1) == 0
    rows = np.random.default_rng(0).choice(A.n, 64, replace=False)
    res = []
    for r in rows:
        e0, e1 = A.rowptr[r], A.rowptr[r + 1]
        cols = torch.from_numpy(A.colind[e0:e1].astype(np.int64)).cuda()
        AV = (torch.from_numpy(A.vals[e0:e1]).cuda()[None, :] * V[:m, cols]).sum(1).cpu().numpy()
        VH = V[:, r].cpu().numpy() @ ls.H
        res.append(np.abs(AV - VH).max())
    assert max(res) <= 1e-12 * np.abs(A.vals).max()


# ------------------------------------------------------- SpMV tilings
@pytest.mark.parametrize("tiling", [(256, 2048, 1), (256, 2048, 0), (64, 512, 1), (16, 128, 1), (1, 2048, 1),
                                    (256, 2048, 2), (200, 1500, 2), (16, 128, 2)])
def test_spmv_tilings_power_law_graph(fab, torch, tiling):
    """Every tiling (rows per tile, nonzeros per tile, staging) gives the oracle's result:
    (1, ., .) puts the whole block on each row, (16, 128) mixes 16..256 lanes per row;
    staging 2 processes tiles of at least 32 rows by nonzeros (200 rows: tiles cut by the
    nonzero cap keep any row count), and tiles of fewer rows by lanes."""
    A = W.chung_lu_laplacian(20000, seed=2)
    b = W.random_vector(A.n, 0)
    m, k, s = 30, 2, 120
    th = osk.make(osk.SRHT, A.n, s, 1, 8)
    ref = krylov.run(krylov.SKETCHED_FAST, W.to_scipy(A), b, m, k, matfun.INVSQRT, th, 1.0)
    M = fab.Matrix.from_csr(A)
    M.set_tiling(*tiling)
    x = M.apply(b, fab.params(f=fab.INVSQRT, m=m, k=k, s=s, sketch=fab.SRHT, seed=1))
    assert _rel(x, ref.x) <= TOL


def _uneven_rows(n, seed):
    """Rows of 0..60 nonzeros (one in eight empty, a few of 300) at random columns,
    with a dominant diagonal on the non-empty rows; CSR with sorted columns."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 61, n)
    lens[rng.random(n) < 0.125] = 0
    lens[rng.choice(n, 5, replace=False)] = 300
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    cols, vals = [], []
    for i, L in enumerate(lens):
        if L == 0:
            continue
        c = np.sort(rng.choice(n, L, replace=False))
        v = rng.standard_normal(L) / np.sqrt(L)
        if i not in c:
            c[0] = i
            c = np.sort(c)
        v[np.searchsorted(c, i)] = 3.0
        cols.append(c)
        vals.append(v)
    return W.CSR(n=n, rowptr=rowptr, colind=np.concatenate(cols).astype(np.int32), vals=np.concatenate(vals))


@pytest.mark.parametrize("tiling", [(256, 2048, 2), (97, 700, 2), (256, 2048, 1)])
@pytest.mark.parametrize("k", [1, 3])
def test_nonzero_parallel_tiles_empty_and_long_rows(fab, torch, tiling, k):
    """Tiles processed by nonzeros with empty rows (their sums are 0), rows spread over
    many threads (a row of 300 nonzeros in a staged tile) and rows cut at thread and tile
    boundaries: sketched_fast against the oracle at 1e-10."""
    A = _uneven_rows(6000, 12)
    b = W.random_vector(A.n, 3)
    m, s = 25, 100
    th = osk.make(osk.SPARSE_SIGN, A.n, s, 2, 8)
    ref = krylov.run(krylov.SKETCHED_FAST, W.to_scipy(A), b, m, k, matfun.EXP, th, -0.2)
    M = fab.Matrix.from_csr(A)
    M.set_tiling(*tiling)
    x = M.apply(b, fab.params(f=fab.EXP, t=-0.2, m=m, k=k, s=s, sketch=fab.SPARSE_SIGN, zeta=8, seed=2))
    assert _rel(x, ref.x) <= TOL


def test_dense_rows_and_autotune(fab, torch):
    """Rows longer than a staged tile (a dense first row and column, 5000 entries) take the
    direct path with the whole block on the row; the autotuned tiling keeps parity."""
    n = 5000
    rng = np.random.default_rng(4)
    D = np.diag(4.0 + rng.random(n))
    D[0, :] += 0.001 * rng.standard_normal(n)
    D[:, 0] += 0.001 * rng.standard_normal(n)
    i = np.arange(n - 1)
    D[i, i + 1] -= 0.5
    D[i + 1, i] -= 0.7
    A = W.from_dense(D)
    b = W.random_vector(n, 1)
    m, k = 25, 3
    ref = krylov.run(krylov.NOPROJ, W.to_scipy(A), b, m, k, matfun.EXP, None, -0.05)
    M = fab.Matrix.from_csr(A)
    x = M.apply(b, fab.params(f=fab.EXP, t=-0.05, m=m, k=k, method=fab.NOPROJ))
    assert _rel(x, ref.x) <= TOL
    choice = M.tune(fab.FP64, k=k)
    assert choice[0] in (256, 128, 64) and choice[1] in (2048, 1024, 512) and choice[2] in (0, 1, 2)
    x2 = M.apply(b, fab.params(f=fab.EXP, t=-0.05, m=m, k=k, method=fab.NOPROJ))
    assert _rel(x2, ref.x) <= TOL
    with pytest.raises(fab.FabError) as e:
        M.set_tiling(0, 2048, 1)
    assert e.value.code == fab.FAB_EINVAL


# ------------------------------------------------------ Alg. 3 (Alg. 1 basis)
@pytest.mark.parametrize("kind,s", [(osk.SRHT, 160), (osk.SPARSE_SIGN, 160)])
def test_bg_ls_convdiff_exp(fab, torch, kind, s):
    """Alg. 3 on the 2D convection-diffusion problem: f(A)b, H (= R without its first
    column) and the orthonormal sketched basis S = Theta V against the oracle."""
    A, b = _c1()
    m, t = 40, -0.01
    th = osk.make(kind, A.n, s, 1, 8)
    ref = krylov.run(krylov.BG_LS, W.to_scipy(A), b, m, 0, matfun.EXP, th, t, tol=1e-14)
    M, x, st = _run_gpu(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=2, s=s, zeta=8, sketch=kind, seed=1,
                        method=fab.BG_LS, lsqr_tol=1e-14)
    assert st.m_used == m and st.lsqr_iters > 0
    assert st.beta == pytest.approx(ref.basis.beta, rel=1e-12)  # gamma_b = r_11 = ||Theta b||
    assert _rel(x, ref.x) <= TOL
    ls = M.last_state()
    B = ref.basis
    # One classical Gram-Schmidt pass per step (Alg. 1) loses orthogonality at
    # O(eps kappa^2) (1.7e-10 in the oracle itself here), so two correct
    # implementations' coefficients agree to about that times the growth over m
    # steps; f(A)b, what the method delivers, is held to 1e-10 above.
    errH = np.linalg.norm(ls.H - B.H) / np.linalg.norm(B.H)
    errS = np.linalg.norm(ls.SV - B.S) / np.linalg.norm(B.S)
    print(f"\nAlg. 1 basis vs oracle: H {errH:.2e}, S {errS:.2e}")
    assert errH <= 1e-8 and errS <= 1e-8


def test_bg_ls_laplacian3d_invsqrt_s_105m(fab, torch):
    """The paper's Alg. 3 setting (§5.1.4): 3D Laplacian, inverse square root, s = floor(1.05 m)."""
    A = W.laplacian3d(24)
    b = W.random_vector(A.n, 4)
    m = 40
    s = int(1.05 * m)
    th = osk.make(osk.SRHT, A.n, s, 2, 8)
    ref = krylov.run(krylov.BG_LS, W.to_scipy(A), b, m, 0, matfun.INVSQRT, th, 1.0, tol=1e-14)
    _, x, _ = _run_gpu(fab, torch, A, b, f=fab.INVSQRT, m=m, k=2, s=s, sketch=fab.SRHT, seed=2, method=fab.BG_LS,
                       lsqr_tol=1e-14)
    assert _rel(x, ref.x) <= TOL


def test_bg_ls_graph_sqrt_and_breakdown(fab, torch):
    A = W.chung_lu_laplacian(20000, seed=2)
    b = W.random_vector(A.n, 0)
    th = osk.make(osk.SRHT, A.n, 120, 1, 8)
    ref = krylov.run(krylov.BG_LS, W.to_scipy(A), b, 30, 0, matfun.SQRT, th, 1.0, tol=1e-14)
    _, x, _ = _run_gpu(fab, torch, A, b, f=fab.SQRT, m=30, k=2, s=120, sketch=fab.SRHT, seed=1, method=fab.BG_LS,
                       lsqr_tol=1e-14)
    assert _rel(x, ref.x) <= TOL
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 5.0], 40)
    bd = W.random_vector(len(d), 2)
    _, xd, std = _run_gpu(fab, torch, W.diagonal(d), bd, f=fab.EXP, t=-0.3, m=8, k=2, s=16, sketch=fab.SRHT,
                          seed=1, method=fab.BG_LS)
    assert std.m_used == 5
    assert _rel(xd, np.exp(-0.3 * d) * bd) <= 1e-9
    M = fab.Matrix.from_csr(W.diagonal(d))
    with pytest.raises(fab.FabError) as e:  # Alg. 1 sketches every new vector: no tensor-core Gaussian sketch
        M.apply(bd, fab.params(m=8, s=16, sketch=fab.GAUSSIAN, method=fab.BG_LS, precision=fab.MIXED))
    assert e.value.code == fab.FAB_EINVAL


# ------------------------------------------------------------ sign(A) b, §5.1.1
def _shifted_convdiff(N=16):
    A = W.to_scipy(W.convdiff(2, N, c=(2.0, 1.0)))
    ev = np.linalg.eigvals(A.toarray())
    mu = float(np.median(ev.real)) + 0.37  # spectrum on both sides of the imaginary axis
    As = (A - mu * __import__("scipy").sparse.identity(A.shape[0])).tocsr()
    As.sort_indices()
    return As


@pytest.mark.parametrize("method", [krylov.ARNOLDI, krylov.SKETCHED_FAST, krylov.NOPROJ, krylov.BG_LS])
def test_sign_via_inverse_sqrt_of_square(fab, torch, method):
    """sign(A) b = (A^2)^{-1/2} (A b): the library forms A^2 on the host with its own
    summation order, a relative perturbation of about (nonzeros per row) eps that the
    inverse square root amplifies by about kappa(A^2)/2, so the bar is that bound or
    1e-10, whichever is larger."""
    As = _shifted_convdiff(16)
    A = W.CSR(n=As.shape[0], rowptr=As.indptr.astype(np.int64), colind=As.indices.astype(np.int32),
              vals=As.data.astype(np.float64))
    b = W.random_vector(A.n, 5)
    m, k, s = 40, 2, 120
    th = osk.make(osk.SRHT, A.n, s, 3, 8)
    ref = krylov.run(method, As, b, m, k, matfun.SIGN, th, 1.0, tol=1e-14)
    A2 = (As @ As).toarray()
    tol = max(TOL, 5 * np.finfo(float).eps * 13 * np.linalg.cond(A2) / 2)
    _, x, st = _run_gpu(fab, torch, A, b, f=fab.SIGN, m=m, k=k, s=s, sketch=fab.SRHT, seed=3, method=method,
                        lsqr_tol=1e-14)
    err = _rel(x, ref.x)
    print(f"\nsign method={method}: rel err {err:.2e} (bar {tol:.1e})")
    assert err <= tol


@pytest.mark.parametrize("method", [krylov.ARNOLDI, krylov.SKETCHED_FAST, krylov.SKETCHED_LS, krylov.NOPROJ,
                                    krylov.BG_LS])
def test_skew_convdiff_exp_all_methods(fab, torch, method):
    """The §5.1.1 operator (skew-form convection, discontinuous diffusion, Pe = 200) with
    the sine start vector, exp(t A), every method against the oracle."""
    A = W.convdiff_skew(48)
    b = W.sine_vector(48)
    m, k, s, t = 40, 2, 160, -1e-5
    th = osk.make(osk.SRHT, A.n, s, 1, 8)
    ref = krylov.run(method, W.to_scipy(A), b, m, k, matfun.EXP, th, t, tol=1e-14)
    _, x, _ = _run_gpu(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=1, method=method,
                       lsqr_tol=1e-14)
    assert _rel(x, ref.x) <= TOL


# ------------------------------------------- exp(t H) e_1: Pade [13/13] scaling
@pytest.mark.parametrize("method", [krylov.NOPROJ, krylov.SKETCHED_FAST])
@pytest.mark.parametrize("t", [-1e-4, -3e-3, -2e-2])
def test_exp_pade_scaling_across_norms(fab, torch, method, t):
    """exp(t Hhat) e_1 by scaling and squaring with the [13/13] Pade approximant: for
    ||t Hhat||_1 from 0.9 (no squaring) to 238 (6 squarings), the solve matches
    the oracle (scipy's expm, a different scaling-and-squaring scheme) at 1e-10, and the
    number of squarings is the smallest sq with ||t Hhat||_1 / 2^sq <= theta_13 (Higham
    2005), computed from the oracle's Hhat."""
    A = W.convdiff(2, 30)
    b = W.random_vector(A.n, 4)
    m, k, s = 30, 4, 120
    th = osk.make(osk.SRHT, A.n, s, 2, 8) if method == krylov.SKETCHED_FAST else None
    ref = krylov.run(method, W.to_scipy(A), b, m, k, matfun.EXP, th, t)
    M = fab.Matrix.from_csr(A)
    meth = fab.NOPROJ if method == krylov.NOPROJ else fab.SKETCHED_FAST
    x, st = M.apply(torch.from_numpy(b).cuda(), fab.params(f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=2,
                                                        method=meth), stats=True)
    assert _rel(x.cpu().numpy(), ref.x) <= TOL
    theta13 = 5.371920351148152
    nrm = float(np.abs(t * ref.Hhat).sum(axis=0).max())
    ratio = math.log2(nrm / theta13) if nrm > theta13 else 0.0
    if abs(ratio - round(ratio)) > 1e-6:  # away from a power-of-two boundary
        assert st.fh_iters == max(0, math.ceil(ratio))
    if t == -2e-2:
        assert st.fh_iters >= 4
