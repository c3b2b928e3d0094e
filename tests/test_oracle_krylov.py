"""Pins of the oracle's Krylov bases and f(A)b methods against the paper's statements.

Each check is fixed by the mathematics, not by the oracle itself:
* eq. arnoldilike: A V_m = V_{m+1} H_m for every basis (residual ~ eps);
* Alg. 2 with k >= m and MGS is Arnoldi (identical operations);
* symmetric A, k = 2 gives Lanczos (orthonormal basis; Alg. 5 equals Arnoldi);
* Alg. 2: any k + 1 consecutive vectors are orthonormal, so ||A v_{c-1}||^2 is the sum
  of the squares of column c-1's window coefficients and h_{c,c-1};
* lemma:basis: with the LS solved exactly, Alg. 4 equals Arnoldi;
* thm:lastcol: every method is exact for polynomials of degree <= m-1;
* m = n and #distinct eigenvalues <= m give the exact f(A)b;
* an orthogonal sketch (full SRHT) makes the sketched variant equal to Arnoldi;
* eq. sFOM equals its sketch-and-solve form (Remark in §3.3);
* thm:convclassic, lemma:derivative and thm:lastcol bounds on small cases.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from oracle import krylov, matfun, sketch
from paper_2212_12758_gb300 import workloads as W

EXP, SQRT, INVSQRT, POLY = matfun.EXP, matfun.SQRT, matfun.INVSQRT, matfun.POLY


def _small_cd(N=12):
    A = W.to_scipy(W.convdiff(2, N))
    b = W.random_vector(A.shape[0], 0)
    return A, b


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sketch(n, kind=sketch.SPARSE_SIGN, s=None, m=10):
    s = s or 4 * m
    return sketch.make(kind, n, s, 1, 8)


@pytest.mark.parametrize("k,orth", [(2, "cgs"), (2, "mgs"), (4, "cgs"), (30, "mgs")])
def test_arnoldi_like_relation(k, orth):
    A, b = _small_cd()
    B = krylov.nt_basis(A, b, 25, k, orth)
    res = A @ B.V[:, :25] - B.V @ B.H
    assert np.linalg.norm(res) / (scipy.sparse.linalg.norm(A) * np.linalg.norm(B.V)) < 1e-14
    assert np.allclose(np.linalg.norm(B.V, axis=0), 1.0)


def test_nt_full_window_mgs_is_arnoldi():
    A, b = _small_cd()
    B1 = krylov.nt_basis(A, b, 20, 20, "mgs")
    B2 = krylov.arnoldi(A, b, 20)
    assert np.array_equal(B1.V, B2.V) and np.array_equal(B1.H, B2.H)


def test_arnoldi_orthonormal():
    A, b = _small_cd()
    B = krylov.arnoldi(A, b, 30, reorth=True)
    assert np.linalg.norm(B.V.T @ B.V - np.eye(31)) < 1e-13


def test_symmetric_k2_is_lanczos():
    A = W.to_scipy(W.laplacian3d(8))
    b = W.random_vector(A.shape[0], 1)
    B = krylov.nt_basis(A, b, 12, 2)
    assert np.linalg.norm(B.V.T @ B.V - np.eye(13)) < 1e-8
    r1 = krylov.noproj(A, b, 12, 2, INVSQRT)
    r2 = krylov.fm_arnoldi(A, b, 12, INVSQRT)
    assert _rel(r1.x, r2.x) < 1e-8


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_nt_window_orthonormal_pythagoras(k):
    """Alg. 2 orthogonalizes each new vector against the k before it, so any k + 1
    consecutive basis vectors are orthonormal (each pair is fewer than k + 1 apart), and
    A v_{c-1} = sum_{j in window} h_{j,c-1} v_j + h_{c,c-1} v_c gives
    ||A v_{c-1}||^2 = h_{c,c-1}^2 + sum_{window} h_{j,c-1}^2 (the breakdown test's norm).
    Checked on a nonsymmetric convection-diffusion matrix and a directed graph
    Laplacian, whose bases are far from orthonormal overall."""
    for A, b in ((W.to_scipy(W.convdiff(2, 40)), W.random_vector(1600, 1)),
                 (W.to_scipy(W.chung_lu_laplacian(3000, seed=2)), W.random_vector(3000, 7))):
        B = krylov.nt_basis(A, b, 40, k)
        V, H = B.V, B.H
        for c in range(1, V.shape[1]):
            j0 = max(0, c - k)
            Wn = V[:, j0:c + 1]
            assert np.linalg.norm(Wn.T @ Wn - np.eye(c + 1 - j0)) < 1e-12
            av = np.linalg.norm(A @ V[:, c - 1])
            est = math.sqrt(H[c, c - 1] ** 2 + np.sum(H[j0:c, c - 1] ** 2))
            assert abs(est - av) <= 1e-12 * av


def test_m_equals_n_is_exact():
    rng = np.random.default_rng(4)
    n = 12
    M = np.diag(np.linspace(1, 3, n)) + 0.2 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    for f in (EXP, SQRT, INVSQRT):
        exact = matfun.exact_fAb(M, b, f, -0.7 if f == EXP else 1.0)
        r = krylov.fm_arnoldi(M, b, n, f, -0.7 if f == EXP else 1.0)
        assert _rel(r.x, exact) < 1e-10


def test_diagonal_few_distinct_eigenvalues_exact():
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 5.0], 40)
    A = W.to_scipy(W.diagonal(d))
    b = W.random_vector(len(d), 2)
    exact = np.exp(-0.3 * d) * b  # f(A) b = f(a_ii) b_i
    assert np.allclose(matfun.exact_fAb(np.diag(d), b, EXP, -0.3), exact, atol=1e-14)
    th = _sketch(len(d), sketch.SRHT, s=16)
    for meth in (0, 1, 2, 3):
        r = krylov.run(meth, A, b, 8, 2, EXP, th, -0.3)
        assert r.m_used == 5  # the Krylov space is invariant after 5 steps
        assert _rel(r.x, exact) < 1e-9


@pytest.mark.parametrize("meth", [0, 1, 2, 3])
def test_polynomial_exactness(meth):
    """thm:lastcol and its corollary: all methods reproduce p(A) b for deg p <= m-1."""
    A, b = _small_cd()
    m = 8
    coef = np.random.default_rng(meth).standard_normal(m) / 10.0**np.arange(m)
    exact = matfun.exact_fAb(A.toarray() / 1000.0, b, POLY, coef=coef)
    As = A / 1000.0
    th = _sketch(A.shape[0], sketch.SPARSE_SIGN, s=4 * m, m=m)
    if meth == 0:
        r = krylov.fm_arnoldi(As, b, m, POLY, coef=coef)
    elif meth == 1:
        r = krylov.sketched_ls(As, b, m, 2, POLY, th, coef=coef)
    elif meth == 2:
        r = krylov.sketched_fast(As, b, m, 2, POLY, th, coef=coef, form="sketch_solve")
    else:
        r = krylov.noproj(As, b, m, 2, POLY, coef=coef)
    assert _rel(r.x, exact) < 1e-10


def test_lemma_basis_exact_ls_equals_arnoldi():
    A, b = _small_cd(16)
    th = _sketch(A.shape[0], m=20)
    for f, t in ((EXP, -0.01), (INVSQRT, 1.0)):
        r1 = krylov.sketched_ls(A, b, 20, 2, f, th, t, exact_ls=True)
        r2 = krylov.fm_arnoldi(A, b, 20, f, t)
        assert _rel(r1.x, r2.x) < 1e-10
        r3 = krylov.sketched_ls(A, b, 20, 2, f, th, t, tol=1e-14)
        assert _rel(r3.x, r2.x) < 1e-10


def test_orthogonal_sketch_gives_arnoldi():
    A = W.to_scipy(W.convdiff(2, 16))  # n = 256 = n'
    b = W.random_vector(256, 3)
    th = sketch.SRHT_(256, 256, 4)
    r1 = krylov.sketched_fast(A, b, 20, 2, EXP, th, -0.01, form="sketch_solve")
    r2 = krylov.fm_arnoldi(A, b, 20, EXP, -0.01)
    assert _rel(r1.x, r2.x) < 1e-10


def test_sfom_equals_sketch_and_solve():
    A, b = _small_cd(20)
    th = _sketch(A.shape[0], sketch.SRHT, s=60, m=25)
    for f, t in ((EXP, -0.01), (SQRT, 1.0)):
        r1 = krylov.sketched_fast(A, b, 25, 2, f, th, t, form="sfom", sav="direct")
        r2 = krylov.sketched_fast(A, b, 25, 2, f, th, t, form="sfom", sav="relation")
        r3 = krylov.sketched_fast(A, b, 25, 2, f, th, t, form="sketch_solve")
        assert _rel(r1.x, r3.x) < 1e-11 and _rel(r2.x, r3.x) < 1e-11


def test_lsqr_matches_lstsq():
    rng = np.random.default_rng(8)
    M = rng.standard_normal((300, 12)) @ np.diag(np.logspace(0, 1, 12))
    rhs = rng.standard_normal(300)
    res = krylov.lsqr(lambda z: M @ z, lambda u: M.T @ u, rhs, 12, 1e-14, 200)
    ref = np.linalg.lstsq(M, rhs, rcond=None)[0]
    assert res.converged and _rel(res.x, ref) < 1e-10


def test_exp_matches_expm_multiply_on_c1_shape():
    """exp(-0.01 A) b for the 2D convection-diffusion operator: Arnoldi with a large
    basis agrees with SciPy's expm_multiply (Al-Mohy and Higham 2011)."""
    A = W.to_scipy(W.convdiff(2, 40))
    b = W.random_vector(A.shape[0], 0)
    ref = scipy.sparse.linalg.expm_multiply(-0.01 * A, b)
    r = krylov.fm_arnoldi(A, b, 120, EXP, -0.01, reorth=True)
    assert _rel(r.x, ref) < 1e-9


def test_convclassic_bound_symmetric():
    """thm:convclassic on a symmetric case: W(A) = [lmin, lmax]; the minimax error
    is bounded by the Chebyshev interpolant's error."""
    A = W.to_scipy(W.laplacian3d(6))
    lam = np.linalg.eigvalsh(A.toarray())
    b = W.random_vector(A.shape[0], 5)
    exact = matfun.exact_fAb(A.toarray(), b, INVSQRT)
    for m in (3, 5, 8):
        r = krylov.fm_arnoldi(A, b, m, INVSQRT)
        lo, hi = lam[0], lam[-1]
        k = np.arange(m)
        nodes = (lo + hi) / 2 + (hi - lo) / 2 * np.cos((2 * k + 1) * np.pi / (2 * m))
        p = np.polynomial.Polynomial.fit(nodes, 1 / np.sqrt(nodes), m - 1)
        z = np.linspace(lo, hi, 20001)
        cheb_err = np.max(np.abs(1 / np.sqrt(z) - p(z)))
        assert np.linalg.norm(exact - r.x) <= 2 * (1 + math.sqrt(2)) * cheb_err * 1.0001


def _range_box(*mats):
    re_lo = min(np.linalg.eigvalsh((M + M.T) / 2)[0] for M in mats)
    re_hi = max(np.linalg.eigvalsh((M + M.T) / 2)[-1] for M in mats)
    im = max(np.abs(np.linalg.eigvalsh(((M - M.T) / 2j).astype(complex))).max() for M in mats)
    return re_lo, re_hi, im


def test_lemma_derivative_bound():
    """lemma:derivative for f = exp(tz): perturbing y changes f(.) by at most
    (1+sqrt2)^2 ||f'||_D ||h (y - y~)||."""
    A, b = _small_cd(10)
    t = -0.002
    B = krylov.nt_basis(A, b, 12, 2)
    m = 12
    Vm = B.V[:, :m]
    y = np.linalg.lstsq(Vm, B.V[:, m], rcond=None)[0]
    yt = y + 1e-3 * np.random.default_rng(1).standard_normal(m)
    C = B.H[:m, :m].copy(); C[:, -1] += B.H[m, m - 1] * y
    D = B.H[:m, :m].copy(); D[:, -1] += B.H[m, m - 1] * yt
    re_lo, re_hi, im = _range_box(C, D)
    fprime = abs(t) * math.exp(t * re_lo)  # sup of |t e^{tz}| on the box (t < 0)
    lhs = np.linalg.norm(scipy.linalg.expm(t * C) - scipy.linalg.expm(t * D), "fro")
    rhs = (1 + math.sqrt(2)) ** 2 * fprime * np.linalg.norm(B.H[m, m - 1] * (y - yt))
    assert lhs <= rhs


def test_lastcol_bound_disk():
    """thm:lastcol with a disk containing both numerical ranges: the minimax error
    is bounded by the Taylor remainder of exp(tz) about the disk centre."""
    A, b = _small_cd(10)
    t = -0.0004
    for m in (4, 6, 8):
        B = krylov.nt_basis(A, b, m, 2)
        Vm = B.V[:, :m]
        P = np.linalg.pinv(Vm) @ (A @ Vm)
        Hm = B.H[:m, :m]
        lhs = np.linalg.norm(scipy.linalg.expm(t * P)[:, 0] - scipy.linalg.expm(t * Hm)[:, 0])
        c = np.trace(Hm) / m
        r = max(np.linalg.norm(P - c * np.eye(m), 2), np.linalg.norm(Hm - c * np.eye(m), 2))
        x = abs(t) * r
        tail = sum(x**j / math.factorial(j) for j in range(m, m + 60))
        rhs = (2 + 2 * math.sqrt(2)) * math.exp(t * c) * tail
        assert lhs <= rhs * 1.0001


def test_matfun_against_eigendecomposition():
    rng = np.random.default_rng(9)
    n = 15
    X = rng.standard_normal((n, n))
    lam = np.linspace(0.5, 4.0, n)
    M = X @ np.diag(lam) @ np.linalg.inv(X)
    z = rng.standard_normal(n)
    for f, t in ((EXP, -0.4), (SQRT, 1.0), (INVSQRT, 1.0)):
        ref = X @ (matfun.f_scalar(lam, f, t) * np.linalg.solve(X, z))
        assert _rel(matfun.f_apply(M, z, f, t), ref) < 1e-8
    S = matfun.sqrtm(M)
    assert np.linalg.norm(S @ S - M) / np.linalg.norm(M) < 1e-10


# ------------------------------------------------ Alg. 1 basis and Alg. 3
def test_bg_basis_sketch_orthonormal_and_arnoldi_like():
    """Alg. 1 keeps S = Theta V orthonormal (the sketched Gram-Schmidt step) and the
    basis satisfies eq. arnoldilike with H_m = R(:, 2:m+1)."""
    A, b = _small_cd(14)
    th = sketch.make(sketch.SRHT, A.shape[0], 90, 3, 8)
    B = krylov.bg_basis(A, b, 30, th)
    assert B.m_used == 30
    # Theta v_i = s_i by linearity: the same coefficients act on both vectors (to the
    # rounding of the two recurrences, carried through m = 30 steps)
    assert np.linalg.norm(th.apply(B.V) - B.S) < 1e-9 * np.linalg.norm(B.S)
    # orthonormal in exact arithmetic; one classical Gram-Schmidt pass per step
    # loses orthogonality at O(eps kappa^2) of [S_{i-1}, p_i]
    assert np.linalg.norm(B.S.T @ B.S - np.eye(31)) < 1e-8
    res = A @ B.V[:, :30] - B.V @ B.H
    assert np.linalg.norm(res) / (scipy.sparse.linalg.norm(A) * np.linalg.norm(B.V)) < 1e-13
    assert B.beta == pytest.approx(np.linalg.norm(th.apply(b)))  # gamma_b = r_11
    assert np.allclose(B.V[:, 0] * B.beta, b)


def test_bg_with_orthogonal_sketch_is_arnoldi():
    """A full SRHT (s = n = 2^p) is an orthogonal map, so the sketched Gram-Schmidt
    step is exact Gram-Schmidt: the basis and H are Arnoldi's."""
    A = W.to_scipy(W.convdiff(2, 16))  # n = 256
    b = W.random_vector(256, 1)
    th = sketch.make(sketch.SRHT, 256, 256, 2, 8)
    B = krylov.bg_basis(A, b, 20, th)
    U = krylov.arnoldi(A, b, 20, reorth=True)
    assert np.linalg.norm(B.V - U.V) < 1e-10 * np.linalg.norm(U.V)
    assert np.linalg.norm(B.H - U.H) < 1e-10 * np.linalg.norm(U.H)
    assert B.beta == pytest.approx(np.linalg.norm(b))


@pytest.mark.parametrize("f,t", [(EXP, -0.01), (SQRT, 1.0), (INVSQRT, 1.0)])
def test_bg_ls_exact_equals_arnoldi_and_lsqr_converges(f, t):
    """lemma:basis: the compression onto K_m does not depend on the basis, so Alg. 3
    with the least-squares problem solved exactly equals Arnoldi; LSQR on the well
    conditioned basis reaches the exact solution."""
    A, b = _small_cd(12)
    if f != EXP:
        A = (A + A.T) / 2  # SPD: convdiff's symmetric part is -Laplace_h + diag
    th = sketch.make(sketch.SRHT, A.shape[0], 60, 5, 8)
    ref = krylov.fm_arnoldi(A, b, 18, f, t, reorth=True).x
    ex = krylov.bg_ls(A, b, 18, f, th, t, exact_ls=True)
    assert _rel(ex.x, ref) < 1e-10
    it = krylov.bg_ls(A, b, 18, f, th, t, tol=1e-14)
    assert _rel(it.x, ex.x) < 1e-10
    assert 0 < it.lsqr_iters <= 4 * 18
    assert krylov.run(krylov.BG_LS, A, b, 18, 0, f, th, t).x.tobytes() == it.x.tobytes()


def test_bg_ls_polynomial_exact_and_breakdown():
    """thm:lastcol-type exactness for a polynomial of degree <= m-1, and a diagonal
    matrix with 5 distinct eigenvalues stops at m_used = 5 with the exact f(A)b."""
    A, b = _small_cd(10)
    th = sketch.make(sketch.SRHT, A.shape[0], 50, 1, 8)
    coef = np.array([0.3, -1.2, 0.5, 2.0])  # degree 3 <= m - 1
    x = krylov.bg_ls(A, b, 8, POLY, th, 1.0, coef=coef, exact_ls=True).x
    Ad = A.toarray()
    ref = sum(c * np.linalg.matrix_power(Ad, i) @ b for i, c in enumerate(coef))
    assert _rel(x, ref) < 1e-10
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 5.0], 40)
    D = scipy.sparse.diags(d).tocsr()
    bd = W.random_vector(len(d), 2)
    thd = sketch.make(sketch.SRHT, len(d), 20, 1, 8)
    r = krylov.bg_ls(D, bd, 9, EXP, thd, -0.3)
    assert r.m_used == 5
    assert _rel(r.x, np.exp(-0.3 * d) * bd) < 1e-9


# ------------------------------------------------------------- sign(A) b
def _shifted(N=12, mu=None):
    """A 2D convection-diffusion matrix shifted so that its spectrum straddles the
    imaginary axis (eigenvalues on both sides): sign(A) is a nontrivial projector."""
    A = W.to_scipy(W.convdiff(2, N, c=(2.0, 1.0)))
    if mu is None:
        mu = float(np.median(np.linalg.eigvals(A.toarray()).real)) + 0.37
    return (A - mu * scipy.sparse.identity(A.shape[0])).tocsr()


def test_sign_formula_and_krylov_exactness():
    """sign(A) b = (A^2)^{-1/2} (A b) (Higham Ch. 5) on a dense shifted matrix, and the
    Krylov method on (A^2, A b) with m = n reproduces it."""
    A = _shifted(8)  # n = 64
    Ad = A.toarray()
    b = W.random_vector(64, 3)
    ref = matfun.exact_fAb(Ad, b, matfun.SIGN)
    via = matfun.f_apply(Ad @ Ad, Ad @ b, matfun.INVSQRT)
    assert _rel(via, ref) < 1e-10
    S = scipy.linalg.signm(Ad).real
    assert np.linalg.norm(S @ S - np.eye(64)) < 1e-8  # sign(A)^2 = I
    x = krylov.run(krylov.ARNOLDI, A, b, 64, 0, matfun.SIGN, None, 1.0, reorth=True).x
    assert _rel(x, ref) < 1e-8
    th = sketch.make(sketch.SRHT, 64, 64, 2, 8)
    # full window (k = m) and an orthogonal sketch: the sketched variant on (A^2, A b)
    # is Arnoldi on (A^2, A b)
    x3 = krylov.run(krylov.SKETCHED_FAST, A, b, 30, 30, matfun.SIGN, th, 1.0).x
    x4 = krylov.run(krylov.ARNOLDI, A @ A, A @ b, 30, 0, matfun.INVSQRT, None, 1.0).x
    assert _rel(x3, x4) < 1e-8


def test_convdiff_skew_structure():
    """The skew-form convection-diffusion operator: symmetric part = the diffusion
    operator (Pe = 0), skew part = the convection, spectrum in the right half plane."""
    S = W.to_scipy(W.convdiff_skew(16))
    D = W.to_scipy(W.convdiff_skew(16, Pe=0.0))
    assert abs((S + S.T) / 2 - D).max() < 1e-9 * abs(D).max()
    assert abs(D - D.T).max() == 0.0
    assert np.linalg.eigvals(S.toarray()).real.min() > 0
    b = W.sine_vector(16)
    assert abs(np.linalg.norm(b) - 1) < 1e-15 and np.all(b > 0)


# ------------------------------------------------ whitening (§2.1.2, §5.1.3)
def test_whiten_never_triggered_is_alg5():
    """A basis that stays below the threshold is Alg. 2's, and the method returns
    Alg. 5's approximation bit for bit."""
    A, b = _small_cd(12)
    th = sketch.make(sketch.SRHT, A.shape[0], 100, 3, 8)
    r = krylov.whiten(A, b, 25, 2, EXP, th, -0.01, kappa_max=np.inf)
    assert r.basis.wh == 0
    assert r.x.tobytes() == krylov.noproj(A, b, 25, 2, EXP, -0.01).x.tobytes()
    B = krylov.nt_basis(A, b, 25, 2)
    assert np.array_equal(r.basis.V, B.V) and np.array_equal(r.basis.H, B.H)


@pytest.mark.parametrize("kappa_max", [5.0, 20.0, 100.0])
def test_whiten_triggers_at_first_exceedance(kappa_max):
    """Whitening happens after the first column i with kappa_1(R_i) > kappa_max,
    R_i the triangular factor of the sketch of Alg. 2's basis V_i (recomputed here
    from the Alg. 2 basis and a library QR)."""
    A, b = _small_cd(14)
    th = sketch.make(sketch.SRHT, A.shape[0], 120, 3, 8)
    wb = krylov.nt_whiten_basis(A, b, 30, 2, th, kappa_max)
    i = wb.wh
    assert 2 <= i <= 31
    V = krylov.nt_basis(A, b, 30, 2).V
    SV = th.apply(V)

    def kap(j):
        return np.linalg.cond(np.linalg.qr(SV[:, :j], mode="r"), 1)

    assert kap(i) > kappa_max
    assert all(kap(j) <= kappa_max for j in range(2, i))


@pytest.mark.parametrize("kappa_max", [5.0, 20.0, 100.0])
def test_whitened_basis_is_alg1_basis(kappa_max):
    """Remark after Alg. 2: Alg. 1 is Alg. 2 followed by whitening. The whitened
    basis, its Hessenberg matrix (R H R^{-1}), its sketch (Q) and gamma_b = ||b|| r_11
    are Alg. 1's with the same Theta, to rounding (kappa <= 150 here)."""
    A, b = _small_cd(14)
    th = sketch.make(sketch.SRHT, A.shape[0], 120, 3, 8)
    wb = krylov.nt_whiten_basis(A, b, 30, 2, th, kappa_max)
    bg = krylov.bg_basis(A, b, 30, th)
    assert wb.wh > 0 and wb.m_used == bg.m_used == 30
    assert _rel(wb.V, bg.V) < 1e-10
    assert _rel(wb.H, bg.H) < 1e-10
    assert _rel(wb.S, bg.S) < 1e-10
    assert wb.beta == pytest.approx(bg.beta, rel=1e-14)
    # the Arnoldi-like relation holds for the whitened pair (eq. arnoldilike)
    res = A @ wb.V[:, :30] - wb.V @ wb.H
    assert np.linalg.norm(res) / (scipy.sparse.linalg.norm(A) * np.linalg.norm(wb.V)) < 1e-13
    assert np.linalg.norm(th.apply(wb.V) - wb.S) < 1e-9 * np.linalg.norm(wb.S)


def test_whitened_alg5_equals_sfom():
    """§3.3: Alg. 5 on the whitened Alg. 2 basis is eq. sFOM."""
    A, b = _small_cd(14)
    th = sketch.make(sketch.SRHT, A.shape[0], 120, 3, 8)
    r = krylov.whiten(A, b, 30, 2, EXP, th, -0.01, kappa_max=20.0, final="noproj")
    assert r.basis.wh > 0
    sf = krylov.sketched_fast(A, b, 30, 2, EXP, th, -0.01, form="sfom").x
    assert _rel(r.x, sf) < 1e-12


def test_whiten_e3_standin_equals_arnoldi():
    """§5.1.3 setting on a synthetic directed graph Laplacian: Alg. 2's sketch
    passes kappa_1 = 1000 near column 60 (as the paper reports for its graph),
    after which the method is Alg. 3 on an Alg. 1 continuation: with the
    least-squares problem solved exactly it is the Arnoldi approximation
    (lemma:basis), with LSQR to 1e-10 close to it."""
    A = W.to_scipy(W.chung_lu_laplacian(3000, seed=2))
    b = W.random_vector(3000, 7)
    th = sketch.make(sketch.SRHT, 3000, 400, 1, 8)
    ex = krylov.whiten(A, b, 80, 2, SQRT, th, 1.0, exact_ls=True)
    assert 50 <= ex.basis.wh <= 70
    ar = krylov.fm_arnoldi(A, b, 80, SQRT, 1.0, reorth=True).x
    assert _rel(ex.x, ar) < 1e-9
    it = krylov.whiten(A, b, 80, 2, SQRT, th, 1.0, tol=1e-12)
    assert 0 < it.lsqr_iters <= 4 * 80 and _rel(it.x, ex.x) < 1e-9
    assert krylov.run(krylov.WHITEN, A, b, 80, 2, SQRT, th, 1.0, tol=1e-12).x.tobytes() == it.x.tobytes()


def test_whiten_polynomial_exact_and_breakdown():
    """Exactness for a polynomial of degree <= m-1 through a whitened basis, and a
    diagonal matrix with 5 distinct eigenvalues: the Alg. 1 continuation stops at
    m_used = 5 with the exact f(A)b."""
    A, b = _small_cd(10)
    th = sketch.make(sketch.SRHT, A.shape[0], 50, 1, 8)
    coef = np.array([0.3, -1.2, 0.5, 2.0])
    r = krylov.whiten(A, b, 8, 2, POLY, th, 1.0, coef=coef, kappa_max=1.5, exact_ls=True)
    assert r.basis.wh > 0
    Ad = A.toarray()
    ref = sum(c * np.linalg.matrix_power(Ad, i) @ b for i, c in enumerate(coef))
    assert _rel(r.x, ref) < 1e-10
    d = np.repeat([0.5, 1.0, 2.0, 3.5, 5.0], 40)
    D = scipy.sparse.diags(d).tocsr()
    bd = W.random_vector(len(d), 2)
    thd = sketch.make(sketch.SRHT, len(d), 20, 1, 8)
    rd = krylov.whiten(D, bd, 9, 2, EXP, thd, -0.3, kappa_max=1.0)
    assert rd.basis.wh == 2 and rd.m_used == 5
    assert _rel(rd.x, np.exp(-0.3 * d) * bd) < 1e-9
