"""Pins of the oracle's generator and sketch operators against their definitions.

The sketches are defined in the docstring of oracle/sketch.py (SRHT of §2.1.1,
sparse sign of Martinsson-Tropp §9.2, Gaussian); every check here is either a
published value, a brute-force evaluation of the entry formula on tiny sizes,
or a property the definition implies (orthogonality of a full SRHT, exactly
zeta distinct +-1/sqrt(zeta) entries per sparse-sign column, ...).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import rng, sketch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    state = 0
    for v in vals:
        state = (state + rng.GAMMA) & rng.MASK
        assert rng.mix64_int(state) == v


def test_vectorised_generator_matches_integer_generator():
    r = np.random.default_rng(7)
    for seed in [0, 1, 12345, 2**63 + 11]:
        for stream in range(1, 6):
            idx = r.integers(0, 2**40, 50)
            vec = rng.u(seed, stream, idx)
            ref = [rng.u_int(seed, stream, int(i)) for i in idx]
            assert [int(x) for x in vec] == ref


def test_mulhi32_range_reduction():
    r = np.random.default_rng(3)
    x = r.integers(0, 2**32, 1000, dtype=np.uint64)
    for s in [1, 7, 160, 400, 2**31 + 5]:
        got = rng.mulhi32(x, s)
        ref = [(int(v) * s) >> 32 for v in x]
        assert [int(g) for g in got] == ref
        assert int(got.max()) < s


# ---------------------------------------------------------------------------- SRHT
@pytest.mark.parametrize("n,s,seed", [(13, 8, 1), (16, 16, 5), (37, 10, 2), (1, 1, 0)])
def test_srht_apply_equals_entry_formula(n, s, seed):
    th = sketch.SRHT_(n, s, seed)
    V = np.random.default_rng(0).standard_normal((n, 3))
    assert np.allclose(th.apply(V), th.dense() @ V, rtol=0, atol=1e-13)


def test_srht_hadamard_is_sylvester():
    # Kronecker-factored application against scipy's Sylvester Hadamard matrix.
    for p in [1, 5, 9, 11]:
        X = np.random.default_rng(p).standard_normal((1 << p, 2))
        assert np.allclose(sketch._hadamard_apply(X), scipy.linalg.hadamard(1 << p) @ X, atol=1e-10)


def test_full_srht_is_orthogonal():
    n = 64
    th = sketch.SRHT_(n, n, 9)
    T = th.dense()
    assert np.allclose(T.T @ T, np.eye(n), atol=1e-13)
    assert np.array_equal(th.P, np.arange(n))


def test_srht_rows_floyd_properties():
    for npad, s, seed in [(16, 5, 1), (1 << 20, 400, 3), (8, 8, 4)]:
        P = sketch.srht_rows(npad, s, seed)
        assert len(P) == s and len(np.unique(P)) == s
        assert np.all(np.diff(P) > 0) and P[0] >= 0 and P[-1] < npad


def test_srht_rows_uniform_marginals():
    npad, s, trials = 16, 4, 4000
    counts = np.zeros(npad)
    for seed in range(trials):
        counts[sketch.srht_rows(npad, s, seed)] += 1
    expect = trials * s / npad
    assert np.all(np.abs(counts - expect) < 5 * math.sqrt(expect))


def test_srht_signs_bits():
    D = sketch.srht_signs(200, 11)
    for j in [0, 1, 63, 64, 65, 199]:
        word = rng.u_int(11, rng.STREAM_SRHT_D, j // 64)
        assert D[j] == (-1.0 if (word >> (j % 64)) & 1 else 1.0)
    assert abs(D.mean()) < 0.3


# --------------------------------------------------------------------- sparse sign
@pytest.mark.parametrize("n,s,zeta,seed", [(50, 16, 4, 1), (300, 160, 8, 2), (40, 8, 8, 3), (20, 3, 3, 4)])
def test_sparse_sign_structure(n, s, zeta, seed):
    th = sketch.SparseSign(n, s, zeta, seed)
    T = th.dense()
    nz = (T != 0).sum(axis=0)
    assert np.all(nz == zeta)
    assert np.allclose(np.abs(T[T != 0]), 1 / math.sqrt(zeta))
    assert np.allclose(np.linalg.norm(T, axis=0), 1.0)
    V = np.random.default_rng(1).standard_normal((n, 2))
    assert np.allclose(th.apply(V), T @ V, atol=1e-13)


def test_sparse_sign_rows_follow_draw_order():
    n, s, zeta, seed = 30, 160, 8, 77
    rows, signs = sketch.sparse_sign_rows(n, s, zeta, seed)
    for j in [0, 7, 29]:
        have = []
        t = 0
        while len(have) < zeta:
            h = rng.u_int(seed, rng.STREAM_SPARSE_ROWS, 128 * j + t // 2)
            half = (h & 0xFFFFFFFF) if t % 2 == 0 else h >> 32
            r = (half * s) >> 32
            if r not in have:
                have.append(r)
            t += 1
        assert list(rows[j]) == have
        word = rng.u_int(seed, rng.STREAM_SPARSE_SIGNS, j)
        assert list(signs[j]) == [(-1.0 if (word >> q) & 1 else 1.0) for q in range(zeta)]


def test_sparse_sign_subspace_embedding():
    n, d = 4096, 10
    Q = np.linalg.qr(np.random.default_rng(2).standard_normal((n, d)))[0]
    sv = np.linalg.svd(sketch.SparseSign(n, 8 * d, 8, 5).apply(Q), compute_uv=False)
    assert sv.min() > 0.4 and sv.max() < 1.6
    sv = np.linalg.svd(sketch.SRHT_(n, 8 * d, 5).apply(Q), compute_uv=False)
    assert sv.min() > 0.4 and sv.max() < 1.6


# ------------------------------------------------------------------------ Gaussian
def test_round_bf16_matches_torch_on_float32_values():
    torch = pytest.importorskip("torch")
    x32 = np.random.default_rng(5).standard_normal(20000).astype(np.float32)
    x32[:4] = [0.0, 1.0, -2.5, 3.0e-5]
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sketch.round_bf16(x32.astype(np.float64)), ref)


def test_round_bf16_nearest_for_float64_values():
    x = np.random.default_rng(6).standard_normal(5000)
    r = sketch.round_bf16(x)
    # neighbours at distance one bf16 ulp; the rounded value must be the closest
    e = np.floor(np.log2(np.abs(r)))
    ulp = 2.0 ** (e - 7)
    assert np.all(np.abs(x - r) <= ulp / 2 * (1 + 1e-12))


def test_gaussian_moments():
    G = sketch.gaussian_entries(40, 2000, 3, bf16=False)
    assert abs(G.mean()) < 0.01 / math.sqrt(40) * 5
    assert abs(G.var() * 40 - 1.0) < 0.03


def test_gaussian_subspace_embedding():
    """Theta = G with N(0, 1/s) entries (BF16-rounded) embeds a d-dimensional subspace:
    the singular values of G Q (Q orthonormal, n x d) lie in
    [1 - sqrt(d/s) - t, 1 + sqrt(d/s) + t] with probability >= 1 - 2 exp(-s t^2 / 2)
    (Davidson and Szarek's bound for Gaussian matrices). A wrong scale (say 1/sqrt(n)
    for 1/sqrt(s)) or correlated entries (a rank-deficient G) fall outside."""
    n = 4096
    for d, s, t in ((25, 100, 0.2), (8, 512, 0.1)):
        Q = np.linalg.qr(np.random.default_rng(3).standard_normal((n, d)))[0]
        sv = np.linalg.svd(sketch.Gaussian(n, s, 7).apply(Q), compute_uv=False)
        r = math.sqrt(d / s)
        assert sv.min() > 1 - r - t and sv.max() < 1 + r + t, (d, s, sv.min(), sv.max())
