"""GPU: the serving runtime (continuous batching).

A mix of requests (different matrices, sizes, functions, methods and
precisions) is solved once alone (fab_apply) and once submitted all together to
a server whose slots run them concurrently on separate streams. Every reduction
in the library has a fixed order that depends only on the problem size (launch
shapes come from the occupancy of the kernel, not from co-running work), so the
results must be bit-identical: the stated tolerance is 0.
"""
import numpy as np
import pytest

from paper_2212_12758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def _mix(fab):
    mats = {
        "cd2": W.convdiff(2, 70),
        "cd3": W.convdiff(3, 18),
        "graph": W.chung_lu_laplacian(12000, seed=2),
    }
    M = {k: fab.Matrix.from_csr(v) for k, v in mats.items()}
    reqs = []
    rng = np.random.default_rng(5)
    specs = [
        ("cd2", dict(f=fab.EXP, t=-0.002, m=30, k=2, s=120, sketch=fab.SRHT, method=fab.SKETCHED_FAST)),
        ("cd3", dict(f=fab.EXP, t=-0.001, m=40, k=4, s=160, sketch=fab.SRHT, method=fab.SKETCHED_LS)),
        ("graph", dict(f=fab.INVSQRT, m=30, k=2, s=120, sketch=fab.SRHT, method=fab.SKETCHED_FAST)),
        ("graph", dict(f=fab.SQRT, m=25, k=2, s=100, sketch=fab.GAUSSIAN, method=fab.SKETCHED_FAST,
                       precision=fab.MIXED)),
        ("cd2", dict(f=fab.EXP, t=-0.002, m=30, k=2, method=fab.ARNOLDI)),
        ("cd3", dict(f=fab.EXP, t=-0.001, m=20, k=2, s=80, zeta=8, sketch=fab.SPARSE_SIGN, method=fab.NOPROJ,
                     precision=fab.MIXED)),
        ("graph", dict(f=fab.SQRT, m=30, k=2, method=fab.NOPROJ)),
        ("cd2", dict(f=fab.EXP, t=-0.004, m=35, k=3, s=140, zeta=4, sketch=fab.SPARSE_SIGN,
                     method=fab.SKETCHED_FAST)),
    ]
    for i, (name, kw) in enumerate(specs * 2):
        b = rng.standard_normal(mats[name].n)
        reqs.append((M[name], b, fab.params(seed=1 + i % 3, **kw)))
    return M, reqs


def test_results_identical_alone_and_in_the_mix(fab):
    M, reqs = _mix(fab)
    alone = [Mx.apply(b, p) for Mx, b, p in reqs]
    srv = fab.Server(slots=4)
    tickets = [srv.submit(Mx, b, p) for Mx, b, p in reqs]
    lat = []
    for t, ref in zip(tickets, alone):
        x, st, ms = srv.poll(t, timeout_ms=120000)
        assert np.array_equal(x, ref)
        lat.append(ms)
    s = srv.stats()
    assert s.completed == len(reqs) and s.queued == 0
    assert s.bytes_in_use <= s.bytes_budget
    srv.close()
    assert min(lat) > 0


def test_admission_budget_and_poll(fab):
    A = W.convdiff(2, 120)
    Mx = fab.Matrix.from_csr(A)
    p = fab.params(f=fab.EXP, t=-0.002, m=40, k=2, s=160, sketch=fab.SRHT)
    b = W.random_vector(A.n, 1)
    ref = Mx.apply(b, p)
    budget = 8 << 20  # one request's workspace is about 6 MB: one slot at a time may hold one
    srv = fab.Server(hbm_budget_bytes=budget, slots=3)
    tickets = [srv.submit(Mx, b, p) for _ in range(6)]
    peak = 0.0
    for t in tickets:
        while True:
            s = srv.stats()
            peak = max(peak, s.bytes_in_use)
            r = srv.poll(t, timeout_ms=5)
            if r is not None:
                assert np.array_equal(r[0], ref)
                break
    assert peak <= budget
    with pytest.raises(fab.FabError) as e:  # a request larger than the whole budget
        srv.submit(Mx, b, fab.params(f=fab.EXP, t=-0.002, m=400, k=2, s=800, sketch=fab.SRHT))
    assert e.value.code == fab.FAB_ENOMEM
    assert fab.lib.fab_server_poll(srv._s, 10**9, None, None, None, 0) == fab.FAB_EINVAL  # unknown ticket
    srv.close()
