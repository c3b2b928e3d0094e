"""GPU: edge cases of the path, against closed forms or the FP64 oracle.

A 1 x 1 matrix (the Krylov space ends after one column), rows without nonzeros
(at the start, the end and inside a row tile), the largest Krylov dimension
(m = 1024) and the largest sketch (s = 4096, with the sketch-and-solve QR on
the cluster path and on the one-block fallback).
"""
import math

import numpy as np
import pytest

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


def _run(fab, torch, A, b, **kw):
    M = fab.Matrix.from_csr(A)
    x, st = M.apply(torch.from_numpy(b).cuda(), fab.params(**kw), stats=True)
    return x.cpu().numpy(), st


def test_one_by_one_matrix(fab, torch):
    """A = (2), b = (3): A v_1 = 2 v_1, so h_21 = 0 ends the basis at one column and
    every method returns exp(2t) 3."""
    A = W.from_dense(np.array([[2.0]]))
    b = np.array([3.0])
    t = -0.7
    for method, kw in ((fab.ARNOLDI, {}), (fab.NOPROJ, {}),
                       (fab.SKETCHED_FAST, dict(s=4, zeta=2, sketch=fab.SPARSE_SIGN))):
        x, st = _run(fab, torch, A, b, f=fab.EXP, t=t, m=3, k=2, method=method, **kw)
        assert st.m_used == 1, method
        assert abs(x[0] - 3.0 * math.exp(2.0 * t)) <= 1e-14 * 3.0, method


def _without_rows(A, empty):
    """A with the rows marked in `empty` left without nonzeros."""
    counts = np.diff(A.rowptr)
    keep = np.repeat(~empty, counts)
    rowptr = np.zeros(A.n + 1, dtype=np.int64)
    np.cumsum(np.where(empty, 0, counts), out=rowptr[1:])
    return W.CSR(n=A.n, rowptr=rowptr, colind=np.ascontiguousarray(A.colind[keep]),
                 vals=np.ascontiguousarray(A.vals[keep]))


@pytest.mark.parametrize("method", [krylov.SKETCHED_FAST, krylov.SKETCHED_LS, krylov.NOPROJ, krylov.ARNOLDI])
def test_rows_without_nonzeros(fab, torch, method):
    """2D convection-diffusion 50^2 with its first row, its last row and rows 100..199
    (inside one 256-row tile and across the next) emptied: A v is zero there."""
    A0 = W.convdiff(2, 50)
    empty = np.zeros(A0.n, dtype=bool)
    empty[[0, A0.n - 1]] = True
    empty[100:200] = True
    A = _without_rows(A0, empty)
    assert np.all(np.diff(A.rowptr)[empty] == 0)
    b = W.random_vector(A.n, 4)
    m, k, s, t = 30, 2, 120, -0.01
    th = osk.make(osk.SRHT, A.n, s, 5, 8)
    ref = krylov.run(method, W.to_scipy(A), b, m, k, matfun.EXP, th, t, tol=1e-14)
    x, st = _run(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=5, method=method,
                 lsqr_tol=1e-14)
    assert st.m_used == m
    assert _rel(x, ref.x) <= TOL


@pytest.mark.parametrize("method,N", [(krylov.ARNOLDI, 11), (krylov.NOPROJ, 22)])
def test_largest_krylov_dimension(fab, torch, method, N):
    """m = 1024, the largest the library takes, on the symmetric 3D Laplacian N^3,
    exp(-0.5 A) b: Arnoldi (full orthogonalization; N = 11, n = 1331 keeps the oracle's
    modified Gram-Schmidt short) and Alg. 5 with k = 2 (N = 22; the window recurrence
    is then Lanczos', whose Ritz values stay in the spectrum)."""
    A = W.laplacian3d(N)
    b = W.random_vector(A.n, 6)
    m, k, t = 1024, 2, -0.5
    ref = krylov.run(method, W.to_scipy(A), b, m, k, matfun.EXP, None, t)
    x, st = _run(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, method=method)
    assert st.m_used == m
    assert _rel(x, ref.x) <= TOL


@pytest.mark.parametrize("f,m", [(matfun.SQRT, 40), (matfun.SQRT, 200), (matfun.INVSQRT, 200), (matfun.EXP, 300)])
def test_small_stage_past_the_staged_lu(fab, torch, f, m):
    """The LU solves of Denman-Beavers and of the Pade approximant stage the factors in
    shared memory for m <= 160 and read them from global memory above; one process runs
    both sizes (m = 40 first), so a launch attribute set for the smaller must not
    constrain the larger. Alg. 5, k = 2, on the 3D Laplacian 12^3."""
    A = W.laplacian3d(12)
    b = W.random_vector(A.n, 8)
    k, t = 2, -0.05
    ref = krylov.run(krylov.NOPROJ, W.to_scipy(A), b, m, k, f, None, t)
    fe = {matfun.SQRT: fab.SQRT, matfun.INVSQRT: fab.INVSQRT, matfun.EXP: fab.EXP}[f]
    x, st = _run(fab, torch, A, b, f=fe, t=t, m=m, k=k, method=krylov.NOPROJ)
    assert st.m_used == m
    assert _rel(x, ref.x) <= TOL


@pytest.mark.parametrize("kind", [osk.SPARSE_SIGN, osk.SRHT])
def test_largest_sketch_of_vectors(fab, torch, kind):
    """s = 4096, the largest sketch, on vectors with a wide dynamic range (n = 12345,
    padded to 16384 for the SRHT)."""
    n, s = 12345, 4096
    rng = np.random.default_rng(9)
    Vh = rng.standard_normal((3, n)) * np.array([[1.0], [1e-7], [3e5]])
    Vh[2, ::3] *= 1e-9
    out = fab.sketch_apply(torch.from_numpy(Vh).cuda(), s, sketch=kind, zeta=8, seed=4).cpu().numpy()
    ref = osk.make(kind, n, s, 4, 8).apply(Vh.T).T
    for j in range(3):
        assert np.max(np.abs(out[j] - ref[j])) <= 1e-13 * np.linalg.norm(Vh[j])


@pytest.mark.parametrize("m", [40, 100])
def test_largest_sketch_in_a_solve(fab, torch, m):
    """sketched_fast with s = 4096 on the 2D convection-diffusion 100^2: the QR of the
    4096 x (m+1) sketch runs on the cluster (m = 40) and on the one-block fallback
    (m = 100, too large for the cluster's shared memory)."""
    A = W.convdiff(2, 100)
    b = W.random_vector(A.n, 0)
    s, k, t = 4096, 2, -0.01
    th = osk.make(osk.SRHT, A.n, s, 1, 8)
    ref = krylov.run(krylov.SKETCHED_FAST, W.to_scipy(A), b, m, k, matfun.EXP, th, t)
    x, st = _run(fab, torch, A, b, f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=1,
                 method=fab.SKETCHED_FAST)
    assert st.m_used == m
    assert _rel(x, ref.x) <= TOL


def test_failed_growth_invalidates_the_last_state():
    """A solve that fails while its workspace grows (FAB_FAULT=alloc:1 set after a
    successful solve: the next growing buffer is freed and not reallocated, as when
    cudaMalloc fails) leaves nothing to inspect: fab_last_state and fab_last_basis
    return FAB_EINVAL instead of reading freed or stale buffers. With the fault
    cleared the same solve succeeds and matches the oracle. The variable is re-read
    at every allocation, so one child process runs all three phases."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import ctypes, os, numpy as np\n"
        "from oracle import krylov, matfun\n"
        "from oracle import sketch as osk\n"
        "from paper_2212_12758_gb300 import fab, workloads as W\n"
        "A = W.convdiff(2, 30); b = W.random_vector(A.n, 0)\n"
        "M = fab.Matrix.from_csr(A)\n"
        "p1 = fab.params(f=fab.EXP, t=-0.01, m=10, k=2, s=40, sketch=fab.SRHT, method=fab.SKETCHED_FAST)\n"
        "x = M.apply(b, p1)\n"
        "assert fab.lib.fab_last_state(M._h, None, None, None, None) == fab.FAB_OK\n"
        "p2 = fab.params(f=fab.EXP, t=-0.01, m=60, k=2, s=240, sketch=fab.SRHT, method=fab.SKETCHED_FAST)\n"
        "os.environ['FAB_FAULT'] = 'alloc:1'\n"
        "rc = fab.lib.fab_apply(M._h, ctypes.byref(p2), b.ctypes.data, x.ctypes.data, 0, None)\n"
        "assert rc == fab.FAB_ENOMEM, rc\n"
        "V = np.zeros((61, A.n))\n"
        "assert fab.lib.fab_last_state(M._h, None, None, None, None) == fab.FAB_EINVAL\n"
        "assert fab.lib.fab_last_basis(M._h, V.ctypes.data, 0) == fab.FAB_EINVAL\n"
        "os.environ['FAB_FAULT'] = ''\n"
        "x2 = M.apply(b, p2)\n"
        "th = osk.make(osk.SRHT, A.n, 240, 1, 8)\n"
        "ref = krylov.run(krylov.SKETCHED_FAST, W.to_scipy(A), b, 60, 2, matfun.EXP, th, -0.01).x\n"
        "err = np.linalg.norm(x2 - ref) / np.linalg.norm(ref)\n"
        "assert err <= 1e-10, err\n"
        "print('ok')\n")
    env = dict(os.environ)
    env.pop("FAB_FAULT", None)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


@pytest.mark.parametrize("method", ["SKETCHED_FAST", "SKETCHED_LS"])
def test_kappa_estimate_of_the_sketched_basis(fab, torch, method):
    """fab_stats.kappa_est is max|r_ii| / min|r_ii| of the QR of Theta V_m. The |r_ii|
    of a Householder QR are unique (|r_ii| = dist(column i, span of the columns
    before it)), so the oracle's QR of its own sketched basis gives the same value
    up to the basis's rounding; it lower-bounds the oracle's exact kappa_2."""
    A = W.convdiff(2, 60)
    b = W.random_vector(A.n, 0)
    m, s = 30, 120
    x, st = _run(fab, torch, A, b, f=fab.EXP, t=-0.005, m=m, k=2, s=s, sketch=fab.SRHT, seed=1,
                 method=getattr(fab, method), lsqr_tol=1e-12)
    th = osk.make(osk.SRHT, A.n, s, 1, 8)
    r = krylov.run(getattr(krylov, method), W.to_scipy(A), b, m, 2, matfun.EXP, th, -0.005, tol=1e-12)
    d = np.abs(np.diag(np.linalg.qr(r.SV[:, :m], mode="r")))
    kap = d.max() / d.min()
    assert kap > 1.0
    assert abs(st.kappa_est - kap) <= 1e-6 * kap, (st.kappa_est, kap)
    sv = np.linalg.svd(r.SV[:, :m], compute_uv=False)
    assert st.kappa_est <= sv[0] / sv[-1] * (1 + 1e-6)
    _, st0 = _run(fab, torch, A, b, f=fab.EXP, t=-0.005, m=m, k=2, method=fab.NOPROJ)
    assert st0.kappa_est == 0.0


def test_fma_peak_is_plausible(fab, torch):
    """fab_fma_peak: the fastest of its operand patterns lies between half and all of
    the device's nominal FP64 rate (2 FMAs per clock per SM at GB300's 2.07 GHz
    maximum clock, 5 % slack) and FP32 runs at least 20 times faster than FP64."""
    p = torch.cuda.get_device_properties(0)
    f64, ms64 = fab.fma_peak(fab.FP64)
    f32, _ = fab.fma_peak(fab.MIXED)
    nominal64 = p.multi_processor_count * 2 * 2 * 2.07
    assert 0.5 * nominal64 <= f64 <= 1.05 * nominal64, (f64, nominal64)
    assert ms64 >= 40.0
    assert f32 >= 20 * f64, (f32, f64)
