"""GPU: growing m to a target accuracy (fab_params.target_rel_err, serving).

The basis is extended by m_step columns until the sketched relative change of
two successive solutions is at most the target. The solution at the dimension
reached must be the oracle's at that dimension (FP64, 1e-10); the true change
of the last step is bounded by the embedding distortion of the sketch: for an
embedding with distortion eps the sketched and true norms of a vector agree
within factors (1 +- eps), so the true relative change is at most
(1 + eps) / (1 - eps) times the estimate (3x covers eps <= 1/2).
"""
import ctypes

import numpy as np
import pytest

from oracle import krylov, matfun
from oracle import sketch as osk
from paper_2212_12758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem():
    A = W.convdiff(2, 60)
    return A, W.random_vector(A.n, 0)


def _oracle_x(A, b, m, s, seed=1, t=-0.005):
    th = osk.make(osk.SRHT, A.n, s, seed, 8)
    return krylov.run(krylov.SKETCHED_FAST, W.to_scipy(A), b, m, 2, matfun.EXP, th, t).x


def test_grows_to_target_and_matches_oracle(fab):
    A, b = _problem()
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=fab.EXP, t=-0.005, m=10, k=2, s=300, sketch=fab.SRHT, seed=1, target_rel_err=1e-8, m_step=10,
                   m_max=200)
    x, st = M.apply(b, p, stats=True)
    mu = st.m_used
    assert 10 < mu <= 200 and (mu - 10) % 10 == 0
    assert 0 < st.err_est <= 1e-8
    x_ref = _oracle_x(A, b, mu, 300)
    assert _rel(x, x_ref) <= 1e-10
    x_prev = _oracle_x(A, b, mu - 10, 300)
    assert _rel(x_prev, x_ref) <= 3 * 1e-8


def test_cap_before_target_returns_best_solution(fab):
    A, b = _problem()
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=fab.EXP, t=-0.005, m=10, k=2, s=300, sketch=fab.SRHT, seed=1, target_rel_err=1e-30, m_step=15,
                   m_max=40)
    x = np.empty(A.n)
    st = fab.Stats()
    rc = fab.lib.fab_apply(M._h, ctypes.byref(p), b.ctypes.data, x.ctypes.data, 0, ctypes.byref(st))
    assert rc == fab.FAB_ENOTCONV
    assert st.m_used == 40
    assert _rel(x, _oracle_x(A, b, 40, 300)) <= 1e-10


def test_server_request_with_target_equals_single_solve(fab):
    A, b = _problem()
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=fab.EXP, t=-0.005, m=10, k=2, s=300, sketch=fab.SRHT, seed=1, target_rel_err=1e-8, m_step=10,
                   m_max=200)
    x1, st1 = M.apply(b, p, stats=True)
    srv = fab.Server(slots=2)
    t = srv.submit(M, b, p)
    x2, st2, _ = srv.poll(t, timeout_ms=60000)
    srv.close()
    assert st2.m_used == st1.m_used
    assert np.array_equal(x1, x2)


def test_target_parameter_checks(fab):
    A, b = _problem()
    M = fab.Matrix.from_csr(A)
    bad = [dict(method=fab.NOPROJ), dict(m_max=5), dict(s=100), dict(m_step=0), dict(target_rel_err=-1.0)]
    for kw in bad:
        base = dict(f=fab.EXP, t=-0.005, m=10, k=2, s=300, sketch=fab.SRHT, seed=1, target_rel_err=1e-8, m_step=10,
                    m_max=200)
        base.update(kw)
        with pytest.raises(fab.FabError) as e:
            M.apply(b, fab.params(**base))
        assert e.value.code == fab.FAB_EINVAL, kw
    with pytest.raises(fab.FabError) as e:  # batches run a fixed m
        fab.Batch([M], [fab.params(f=fab.EXP, t=-0.005, m=10, s=300, sketch=fab.SRHT, target_rel_err=1e-8, m_step=10,
                                   m_max=200)])
    assert e.value.code == fab.FAB_EINVAL


@pytest.mark.parametrize("method", ["SKETCHED_LS", "BG_LS"])
def test_growing_m_with_lsqr_methods(fab, method):
    """Every growth pass runs its own LSQR loop; the solution at the dimension reached is
    the single solve's at that dimension."""
    A, b = _problem()
    M = fab.Matrix.from_csr(A)
    meth = getattr(fab, method)
    p = fab.params(f=fab.EXP, t=-0.005, m=10, k=2, s=300, sketch=fab.SRHT, seed=1, method=meth, lsqr_tol=1e-12,
                   target_rel_err=1e-8, m_step=10, m_max=200)
    x, st = M.apply(b, p, stats=True)
    assert 10 < st.m_used <= 200 and st.err_est <= 1e-8
    x1 = M.apply(b, fab.params(f=fab.EXP, t=-0.005, m=st.m_used, k=2, s=300, sketch=fab.SRHT, seed=1, method=meth,
                               lsqr_tol=1e-12))
    assert _rel(x, x1) <= 1e-12
