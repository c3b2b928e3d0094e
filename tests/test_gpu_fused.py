"""GPU: one-pass basis steps of the FP32 basis (fab_set_fusion; fused.cu).

A pass updates, normalizes and sketches column c-1 and multiplies it by A with the
window dots of step c (Alg. 2); a value of column c-1 outside a block's 4096-row
chunk is recomputed from the previous SpMV output and the window by the FMAs its
owner runs. Checked, on matrices with at most 8 nonzeros per row and every kind of
chunk (a single partial chunk, exact multiples of 4096, a ragged last chunk):

* the FP32 basis and H satisfy the Arnoldi-like relation A V_m = V_{m+1} H_m
  (eq. arnoldilike) within the componentwise rounding bound of FP32 arithmetic;
* the sketch the passes accumulate is the sketch of the stored basis (exact int64
  sums: 1e-13 of the column norm);
* f(A)b against the FP64 oracle at the bar of the stated rounding model, as the
  two-pass FP32 loop is (test_gpu_mixed), and the two forms against each other;
* breakdown, growing m (each run of passes restarts from a finished column), and
  every window width k = 1..8.
"""
import numpy as np
import pytest

from oracle import krylov, matfun
from oracle import sketch as osk
from paper_2212_12758_gb300 import workloads as W
from rounding_model import TAIL, U32, model_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


MATS = {
    "cd2_10000": lambda: W.convdiff(2, 100),   # 3 chunks, the last one partial
    "cd3_27000": lambda: W.convdiff(3, 30),    # 7 chunks, ragged
    "cd2_4096": lambda: W.convdiff(2, 64),     # exactly one chunk
    "cd2_1600": lambda: W.convdiff(2, 40),     # one partial chunk
    "cd2_16384": lambda: W.convdiff(2, 128),   # exactly four chunks
}


def _solve(fab, M, b, fuse, **kw):
    M.set_fusion(fuse)
    x, st = M.apply(b, fab.params(precision=fab.MIXED, **kw), stats=True)
    return x, st, M.last_state(), M.last_basis()


def _relation_ok(As, V, H, k):
    """|A V_m - V_{m+1} H| <= gamma (|A_32||V_m| + |V_{m+1}||H|), gamma = (max row nnz + k + 2) u_32."""
    m = H.shape[1]
    gam = (int(np.diff(As.indptr).max()) + k + 2) * U32
    F = np.abs(As @ V[:, :m] - V @ H)
    B = gam * (abs(As) @ np.abs(V[:, :m]) + np.abs(V) @ np.abs(H))
    return float((F / (B + 1e-300)).max())


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("method,sk", [(krylov.SKETCHED_FAST, osk.SRHT), (krylov.SKETCHED_FAST, osk.SPARSE_SIGN),
                                       (krylov.SKETCHED_LS, osk.SRHT), (krylov.NOPROJ, None)])
def test_fused_steps_against_oracle(fab, name, method, sk):
    A = MATS[name]()
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    m, k, s, t = 30, 2, 120, -0.004
    M = fab.Matrix.from_csr(A)
    kw = dict(f=fab.EXP, t=t, m=m, k=k, s=s, sketch=sk if sk is not None else fab.SRHT, zeta=8, seed=3,
              method=method, lsqr_tol=1e-10)
    xf, stf, lsf, Vf = _solve(fab, M, b, True, **kw)
    x2, st2, ls2, V2 = _solve(fab, M, b, False, **kw)
    assert stf.m_used == st2.m_used == m
    # the relation of the one-pass basis, within FP32 rounding
    assert _relation_ok(As, Vf, lsf.H, k) <= 1.0
    # the accumulated sketch is the sketch of the stored basis
    if sk is not None:
        th = osk.make(sk, A.n, s, 3, 8)
        SVo = th.apply(Vf)
        assert np.max(np.abs(lsf.SV - SVo)) <= 1e-13 * np.linalg.norm(Vf, axis=0).max()
    # f(A) b against the FP64 oracle at the rounding model's bar, both forms
    th = osk.make(sk, A.n, s, 3, 8) if sk is not None else None
    ref = krylov.run(method, As, b, m, k, matfun.EXP, th, t, tol=1e-10)
    rms, _ = model_rms(As, b, m, k, matfun.EXP, th, t, method, ref.x, False)
    ef, e2 = _rel(xf, ref.x), _rel(x2, ref.x)
    print(f"\nFUSED {name} method={method} sk={sk}: one-pass {ef:.3e}, two-pass {e2:.3e}, bar {TAIL * rms:.3e}")
    assert ef <= TAIL * rms and e2 <= TAIL * rms
    assert _rel(xf, x2) <= 2 * TAIL * rms  # both within the bar of the same FP64 result


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8])
def test_fused_every_window_width(fab, k):
    A = W.convdiff(3, 24)  # n = 13,824: 4 chunks, the last one partial
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 1)
    m, s, t = 24, 100, -0.002
    M = fab.Matrix.from_csr(A)
    xf, stf, lsf, Vf = _solve(fab, M, b, True, f=fab.EXP, t=t, m=m, k=k, s=s, sketch=fab.SRHT, seed=2,
                              method=fab.SKETCHED_FAST)
    assert stf.m_used == m
    assert _relation_ok(As, Vf, lsf.H, k) <= 1.0
    # window structure: column c-1 of H has entries only in rows max(0, c-k) .. c
    H = lsf.H
    for c in range(1, m + 1):
        j0 = max(0, c - k)
        assert np.all(H[:j0, c - 1] == 0.0) and np.all(H[c + 1:, c - 1] == 0.0)
    th = osk.make(osk.SRHT, A.n, s, 2, 8)
    ref = krylov.run(krylov.SKETCHED_FAST, As, b, m, k, matfun.EXP, th, t)
    rms, _ = model_rms(As, b, m, k, matfun.EXP, th, t, krylov.SKETCHED_FAST, ref.x, False)
    assert _rel(xf, ref.x) <= TAIL * rms


def test_fused_breakdown(fab):
    """A diagonal matrix with 5 distinct eigenvalues: the Krylov space is invariant at
    dimension 5. The breakdown threshold is relative to the FP64 unit roundoff
    (64 eps ||A v||), which an FP32 basis does not reach, so the loop continues with
    rounding-level directions; the result stays exact up to the FP32 basis, on the
    one-pass and on the two-pass loop."""
    n = 9000
    d = np.array([1.0, 2.0, 3.0, 5.0, 8.0])[np.arange(n) % 5]
    A = W.diagonal(d)
    b = W.random_vector(n, 3)
    M = fab.Matrix.from_csr(A)
    t = -0.3
    for method in (fab.NOPROJ, fab.SKETCHED_FAST):
        for fuse in (True, False):
            x, st, _, _ = _solve(fab, M, b, fuse, f=fab.EXP, t=t, m=12, k=2, s=60, sketch=fab.SRHT, seed=1,
                                 method=method)
            assert st.m_used >= 5, (method, fuse, st.m_used)
            assert _rel(x, np.exp(t * d) * b) <= 1e-5, (method, fuse)


def test_fused_growing_m(fab):
    """Growing m restarts the one-pass loop from the last finished column; the result
    at the dimension reached agrees with a fixed-m solve within FP32 rounding."""
    A = W.convdiff(2, 90)
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    M = fab.Matrix.from_csr(A)
    kw = dict(f=fab.EXP, t=-0.003, m=10, k=2, s=300, sketch=fab.SRHT, seed=1, method=fab.SKETCHED_FAST)
    M.set_fusion(True)
    xg, stg = M.apply(b, fab.params(precision=fab.MIXED, target_rel_err=1e-5, m_step=10, m_max=120, **kw), stats=True)
    mu = stg.m_used
    assert 10 < mu <= 120
    kw["m"] = mu
    x1, st1, ls1, V1 = _solve(fab, M, b, True, **kw)
    th = osk.make(osk.SRHT, A.n, 300, 1, 8)
    ref = krylov.run(krylov.SKETCHED_FAST, As, b, mu, 2, matfun.EXP, th, -0.003)
    rms, _ = model_rms(As, b, mu, 2, matfun.EXP, th, -0.003, krylov.SKETCHED_FAST, ref.x, False)
    assert _rel(xg, ref.x) <= TAIL * rms and _rel(x1, ref.x) <= TAIL * rms
    assert _relation_ok(As, V1, ls1.H, 2) <= 1.0


def test_bounded_wait_expires_and_the_handle_recovers(fab):
    """Failure detection without a GPU fault: fab_inject_wait_timeout makes the SpMV
    tasks of one one-pass step wait for a chunk flag that no task sets, with a short
    poll limit. The wait runs out, the kernel records FAB_ETIMEOUT and returns, and
    fab_apply reports it; the next solve on the same handle is correct."""
    import ctypes

    A = W.convdiff(2, 100)
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    M = fab.Matrix.from_csr(A)
    M.set_fusion(True)
    p = fab.params(f=fab.EXP, t=-0.004, m=20, k=2, s=80, sketch=fab.SRHT, seed=3, method=fab.SKETCHED_FAST,
                   precision=fab.MIXED)
    x = np.empty(A.n)
    assert fab.lib.fab_inject_wait_timeout(M._h, 5, 2000) == fab.FAB_OK
    rc = fab.lib.fab_apply(M._h, ctypes.byref(p), b.ctypes.data, x.ctypes.data, 0, None)
    assert rc == fab.FAB_ETIMEOUT, rc
    assert fab.lib.fab_inject_wait_timeout(M._h, -1, 1) == fab.FAB_EINVAL
    assert fab.lib.fab_inject_wait_timeout(M._h, 3, 0) == fab.FAB_EINVAL
    x2 = M.apply(b, p)  # the hook was one-shot: a normal solve
    th = osk.make(osk.SRHT, A.n, 80, 3, 8)
    ref = krylov.run(krylov.SKETCHED_FAST, As, b, 20, 2, matfun.EXP, th, -0.004)
    rms, _ = model_rms(As, b, 20, 2, matfun.EXP, th, -0.004, krylov.SKETCHED_FAST, ref.x, False)
    assert _rel(x2, ref.x) <= TAIL * rms
