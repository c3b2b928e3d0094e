"""GPU: batched solves (fab_batch_*), many uneven solves as one persistent launch
in a CUDA graph.

A batched solve runs the same phase bodies on the same data as fab_apply, with its
SpMV tiles grouped into fewer blocks and its small stage in one CTA, so only
the grouping of partial sums differs: FP64 results agree with the solve alone
to 1e-11 and with the oracle to the library's FP64 target (1e-10); with the
FP32 basis both the batched and the single result are within the mixed-precision
bar of the FP64 oracle (4 x the RMS of the rounding model, as in test_gpu_mixed).
"""
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


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


MATS = {
    "cd2a": lambda: W.convdiff(2, 40),
    "cd2b": lambda: W.convdiff(2, 71),
    "cd3": lambda: W.convdiff(3, 19),
    "graph": lambda: W.chung_lu_laplacian(6000, seed=2),
}

# (matrix, f, t, m, k, s, zeta, sketch, method, seed)
SPECS = [
    ("cd2a", matfun.EXP, -0.01, 30, 2, 120, 8, osk.SPARSE_SIGN, krylov.SKETCHED_FAST, 1),
    ("cd2b", matfun.EXP, -0.004, 41, 2, 164, 4, osk.SPARSE_SIGN, krylov.SKETCHED_FAST, 2),
    ("cd3", matfun.EXP, -0.001, 25, 4, 100, 8, osk.SRHT, krylov.SKETCHED_FAST, 3),
    ("cd2a", matfun.EXP, -0.02, 18, 2, 0, 8, osk.SRHT, krylov.NOPROJ, 1),
    ("graph", matfun.SQRT, 1.0, 22, 2, 88, 8, osk.SRHT, krylov.SKETCHED_FAST, 4),
    ("graph", matfun.INVSQRT, 1.0, 30, 2, 120, 8, osk.SPARSE_SIGN, krylov.SKETCHED_FAST, 5),
    ("cd3", matfun.EXP, -0.002, 35, 3, 0, 8, osk.SRHT, krylov.NOPROJ, 1),
    ("graph", matfun.INVSQRT, 1.0, 12, 2, 0, 8, osk.SRHT, krylov.NOPROJ, 1),
    ("cd2b", matfun.EXP, -0.001, 41, 2, 123, 8, osk.SRHT, krylov.SKETCHED_FAST, 6),
]


def _setup(fab, precision):
    A = {k: v() for k, v in MATS.items()}
    M = {k: fab.Matrix.from_csr(v) for k, v in A.items()}
    mats, ps, bs, refs = [], [], [], []
    for i, (name, f, t, m, k, s, zeta, sk, method, seed) in enumerate(SPECS):
        kw = dict(f=f, t=t, m=m, k=k, zeta=zeta, sketch=sk, method=method, seed=seed, precision=precision)
        kw["s"] = s if s else 4 * m
        mats.append(M[name])
        ps.append(fab.params(**kw))
        bs.append(W.random_vector(A[name].n, 10 + i))
        refs.append((name, kw))
    return A, M, mats, ps, bs, refs


def _oracle(A, name, kw, b):
    As = W.to_scipy(A[name])
    th = osk.make(kw["sketch"], A[name].n, kw["s"], kw["seed"], kw["zeta"]) if kw["method"] == krylov.SKETCHED_FAST else None
    return krylov.run(kw["method"], As, b, kw["m"], kw["k"], kw["f"], th, kw["t"]).x


def test_batch_fp64_matches_oracle_and_alone(fab):
    A, M, mats, ps, bs, refs = _setup(fab, fab.FP64)
    bt = fab.Batch(mats, ps)
    xs, sts = bt.run(bs, stats=True)
    assert bt.kernels > 0
    for i, ((name, kw), b, x, st) in enumerate(zip(refs, bs, xs, sts)):
        assert st.m_used == kw["m"], i
        alone = mats[i].apply(b, ps[i])
        assert _rel(x, alone) <= 1e-11, i
        assert _rel(x, _oracle(A, name, kw, b)) <= TOL, i
    bt.close()


def test_batch_mixed_matches_alone(fab):
    """FP32 basis: batched and single results both within the mixed-precision bar of the
    FP64 oracle (TAIL x the RMS change of the oracle's f_m under the stated rounding model
    of the FP32 products), and so within twice that of each other."""
    from rounding_model import TAIL, model_rms

    A, M, mats, ps, bs, refs = _setup(fab, fab.MIXED)
    bt = fab.Batch(mats, ps)
    xs = bt.run(bs)
    for i, ((name, kw), b, x) in enumerate(zip(refs, bs, xs)):
        alone = mats[i].apply(b, ps[i])
        ref = _oracle(A, name, kw, b)
        As = W.to_scipy(A[name])
        th = osk.make(kw["sketch"], A[name].n, kw["s"], kw["seed"], kw["zeta"]) \
            if kw["method"] == krylov.SKETCHED_FAST else None
        rms, _ = model_rms(As, b, kw["m"], kw["k"], kw["f"], th, kw["t"], kw["method"], ref, False)
        bar = TAIL * rms
        assert _rel(x, ref) <= bar, (i, _rel(x, ref), bar)  # FP32 basis against the FP64 oracle
        assert _rel(alone, ref) <= bar, (i, _rel(alone, ref), bar)
        assert _rel(x, alone) <= 2 * bar, i
    bt.close()


def test_batch_replay_device_inputs_deterministic(fab):
    import torch

    A, M, mats, ps, bs, refs = _setup(fab, fab.FP64)
    bt = fab.Batch(mats, ps)
    bd = [torch.from_numpy(b).cuda() for b in bs]
    x1 = [torch.empty_like(b) for b in bd]
    x2 = [torch.empty_like(b) for b in bd]
    bt.run(bd, x1)
    bt.run(None, x2)  # inputs left in the batch's staging vectors by the first run
    for a, c in zip(x1, x2):
        assert torch.equal(a, c)
    bt.close()


def test_batch_breakdown_zero_rhs_and_rejects(fab):
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 5.0], 40)
    D = fab.Matrix.from_csr(W.diagonal(d))
    C = fab.Matrix.from_csr(W.convdiff(2, 30))
    b1 = W.random_vector(len(d), 2)
    ps = [fab.params(f=fab.EXP, t=-0.3, m=8, k=2, s=16, sketch=fab.SRHT, seed=1),
          fab.params(f=fab.EXP, t=-0.3, m=8, k=2, method=fab.NOPROJ),
          fab.params(f=fab.EXP, t=-0.01, m=20, k=2, s=80)]
    bt = fab.Batch([D, D, C], ps)
    xs, sts = bt.run([b1, b1, np.zeros(C.n)], stats=True)
    for i in (0, 1):
        assert sts[i].m_used == 5
        assert _rel(xs[i], np.exp(-0.3 * d) * b1) <= 1e-9
    assert sts[2].m_used == 0 and not np.any(xs[2])
    bt.close()
    for bad in (fab.params(m=10, s=40, method=fab.ARNOLDI), fab.params(m=10, s=40, method=fab.SKETCHED_LS),
                fab.params(m=10, s=40, sketch=fab.GAUSSIAN, precision=fab.MIXED)):
        with pytest.raises(fab.FabError) as e:
            fab.Batch([C], [bad])
        assert e.value.code == fab.FAB_EINVAL
    with pytest.raises(fab.FabError) as e:  # one precision per batch
        fab.Batch([C, C], [fab.params(m=10, s=40), fab.params(m=10, s=40, precision=fab.MIXED)])
    assert e.value.code == fab.FAB_EINVAL


@pytest.mark.slow
def test_batch_fp64_many_blocks_per_wave(fab):
    """Solves large enough that a phase gives each of them many blocks (a batched solve
    takes at least 32 SpMV tiles of 256 rows and 4 update chunks of 4096 rows per
    block: n = 360,000 gives 44 SpMV and 22 update blocks): the cross-block partial
    sums, the last-block reductions, the item search and the per-solve phase counters
    of the persistent launch run with several solves of different sizes, windows and
    sketches in it. Every result against
    the FP64 oracle at the library's FP64 target, and against the solve alone."""
    specs = [  # (grid side, f, t, m, k, sketch, s, zeta, method, seed)
        (600, matfun.EXP, -1e-4, 40, 2, osk.SPARSE_SIGN, 160, 8, krylov.SKETCHED_FAST, 1),
        (450, matfun.EXP, -2e-4, 33, 2, osk.SRHT, 132, 8, krylov.SKETCHED_FAST, 2),
        (520, matfun.EXP, -1e-4, 28, 3, osk.SRHT, 0, 8, krylov.NOPROJ, 1),
        (300, matfun.EXP, -5e-4, 36, 2, osk.SPARSE_SIGN, 144, 4, krylov.SKETCHED_FAST, 3),
    ]
    A = [W.convdiff(2, g) for g, *_ in specs]
    assert A[0].n == 360000
    mats = [fab.Matrix.from_csr(a) for a in A]
    ps, bs, refs = [], [], []
    for i, (g, f, t, m, k, sk, s, zeta, method, seed) in enumerate(specs):
        kw = dict(f=f, t=t, m=m, k=k, zeta=zeta, sketch=sk, method=method, seed=seed, precision=fab.FP64,
                  s=s if s else 4 * m)
        ps.append(fab.params(**kw))
        b = W.random_vector(A[i].n, 40 + i)
        bs.append(b)
        th = osk.make(sk, A[i].n, kw["s"], seed, zeta) if method == krylov.SKETCHED_FAST else None
        refs.append(krylov.run(method, W.to_scipy(A[i]), b, m, k, f, th, t).x)
    bt = fab.Batch(mats, ps)
    xs = [np.empty(a.n) for a in A]
    bt.run(bs, xs)
    bt.close()
    for i in range(len(specs)):
        assert _rel(xs[i], refs[i]) <= TOL, i
        alone = mats[i].apply(bs[i], ps[i])
        assert _rel(xs[i], alone) <= 1e-11, i


def test_batch_many_small_solves_in_one_launch(fab):
    """240 small solves (2D convection-diffusion, n from 100 to 3600; m from 4 to 30;
    windows 1, 2 and 3; SRHT, sparse sign and Alg. 5), FP64: every phase of every solve
    runs as work items of the one persistent launch, claimed in plan order with many
    solves in each phase. Each result equals the solve run alone to 1e-11, twice in a
    row (the phase counters and the ticket start from zero in every replay)."""
    rng = np.random.default_rng(21)
    grids = [10, 17, 23, 31, 44, 60]
    A = {N: W.convdiff(2, N) for N in grids}
    M = {N: fab.Matrix.from_csr(a) for N, a in A.items()}
    mats, ps, bs = [], [], []
    for i in range(240):
        N = grids[int(rng.integers(len(grids)))]
        m = int(rng.integers(4, 31))
        k = int(rng.integers(1, 4))
        kind = i % 3
        sk = fab.SRHT if kind == 0 else fab.SPARSE_SIGN
        method = fab.NOPROJ if kind == 2 else fab.SKETCHED_FAST
        mats.append(M[N])
        ps.append(fab.params(f=fab.EXP, t=-0.05 / N, m=m, k=k, s=4 * m, zeta=4, sketch=sk, seed=1 + i % 5,
                             method=method))
        bs.append(W.random_vector(A[N].n, 300 + i))
    bt = fab.Batch(mats, ps)
    for _ in range(2):
        xs, sts = bt.run(bs, stats=True)
        for i, (b, x, st) in enumerate(zip(bs, xs, sts)):
            assert st.m_used == ps[i].m, i
            alone = mats[i].apply(b, ps[i])
            assert _rel(x, alone) <= 1e-11, (i, _rel(x, alone))
    bt.close()


def test_batch_wide_windows(fab):
    """Windows of 5 to 8 columns (the persistent kernel's widest instantiation), FP64,
    against each solve run alone at 1e-11 and against the oracle at 1e-10."""
    A = {"cd3": W.convdiff(3, 19), "cd2": W.convdiff(2, 50)}
    M = {k: fab.Matrix.from_csr(v) for k, v in A.items()}
    specs = [("cd3", 5, 30, krylov.SKETCHED_FAST, osk.SRHT), ("cd2", 8, 40, krylov.SKETCHED_FAST, osk.SPARSE_SIGN),
             ("cd3", 6, 25, krylov.NOPROJ, osk.SRHT), ("cd2", 7, 33, krylov.SKETCHED_FAST, osk.SRHT)]
    mats, ps, bs, refs = [], [], [], []
    for i, (name, k, m, method, sk) in enumerate(specs):
        kw = dict(f=matfun.EXP, t=-0.003, m=m, k=k, s=4 * m, zeta=8, sketch=sk, method=method, seed=2 + i)
        mats.append(M[name])
        ps.append(fab.params(**kw))
        bs.append(W.random_vector(A[name].n, 40 + i))
        refs.append((name, kw))
    bt = fab.Batch(mats, ps)
    xs = bt.run(bs)
    for i, ((name, kw), b, x) in enumerate(zip(refs, bs, xs)):
        assert _rel(x, mats[i].apply(b, ps[i])) <= 1e-11, i
        assert _rel(x, _oracle(A, name, kw, b)) <= TOL, i
    bt.close()
