"""Krylov bases and f(A)b methods of arXiv 2212.12758, step by step in FP64.

Indices are 0-based in code: column c of V is the paper's v_{c+1}; H has shape
(m+1) x m and H[j, c-1] is the paper's h_{j+1,c}.

Readings of the paper taken here (where it is garbled or silent):
* Alg. 2: the window update is w <- w - h_{j,i-1} v_j and the subdiagonal is
  h_{i,i-1} = ||w_i||_2 (the printed lines index h_{j,i} v_i and ||w||).
* The window of Alg. 2 is orthogonalised either by one classical pass (all
  window dots of the unmodified w, then one update; ``orth="cgs"``) or by the
  modified sequence (``orth="mgs"``). They agree in exact arithmetic; the CUDA
  library uses the classical pass.
* gamma_b = ||b||_2 for the Alg. 2 based methods (eq. relationxx).
* Breakdown (the paper assumes none, §2): when the new norm satisfies
  h_{c,c-1} <= 64 eps ||w|| (w before orthogonalisation) or is zero, the basis
  stops with m_used = c columns.
* Alg. 4 reuses the basis sketch Theta for the Blendenpik preconditioner, and
  LSQR starts at zero.
* Alg. 1: gamma_b = r_11 (eq. relationxx); breakdown when r_ii <= 1e-12
  ||Theta w_i|| (the sketch, not the long vector, is orthogonalised); Alg. 3 runs
  LSQR on V_m itself.
* Whitening (§2.1.2, §5.1.3): the condition number checked after every new column
  is kappa_1(R_i) = ||R_i||_1 ||R_i^{-1}||_1 of the thin QR Theta V_i = Q_i R_i
  (diag(R_i) > 0), computed exactly (Matlab's condest estimates this 1-norm
  condition number and needs a square matrix); the first i with kappa_1 > 1000
  whitens V_i and H_{i-1}, and Alg. 1 continues with the same Theta. A basis that
  is never whitened returns Alg. 5's approximation, a whitened one Alg. 3's (the
  recommendation of §6). A QR column with r_ii <= 1e-12 ||Theta v_i|| is a
  breakdown (m_used = i - 1 columns), as for Alg. 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.sparse

from . import matfun

EPS = np.finfo(np.float64).eps
ARNOLDI, SKETCHED_LS, SKETCHED_FAST, NOPROJ, BG_LS, WHITEN = 0, 1, 2, 3, 4, 5
# whitening threshold on kappa_1(Theta V_i) (§5.1.3)
WHITEN_KAPPA = 1000.0
# Alg. 1 breakdown: the sketched residual r_ii below this fraction of ||Theta w_i||
# (far above the rounding of a sketch, far below a genuinely new direction)
BG_BREAKDOWN = 1e-12


def as_operator(A):
    """Accept a scipy sparse matrix, a dense array, or anything with ``@``."""
    return A


@dataclass
class Basis:
    V: np.ndarray      # n x (m_used+1) basis
    H: np.ndarray      # (m_used+1) x m_used Hessenberg
    beta: float        # ||b||_2
    m_used: int


def nt_basis(A, b, m: int, k: int, orth: str = "cgs") -> Basis:
    """Alg. 2 (truncated orthogonalization, §2.1.2): w_i = A v_{i-1} is
    orthogonalised against the last k basis vectors only."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return Basis(V[:, :1], H[:1, :0], 0.0, 0)
    V[:, 0] = b / beta
    for c in range(1, m + 1):
        w = A @ V[:, c - 1]
        wnorm = float(np.linalg.norm(w))
        win = list(range(max(0, c - k), c))
        if orth == "cgs":
            h = V[:, win].T @ w
            w = w - V[:, win] @ h
            H[win, c - 1] = h
        else:
            for j in win:
                H[j, c - 1] = V[:, j] @ w
                w = w - H[j, c - 1] * V[:, j]
        H[c, c - 1] = float(np.linalg.norm(w))
        if not H[c, c - 1] > 64 * EPS * wnorm:
            return _breakdown(V, H, beta, c)
        V[:, c] = w / H[c, c - 1]
    return Basis(V, H, beta, m)


@dataclass
class BGBasis(Basis):
    S: np.ndarray = None   # s x (m_used+1): Theta V, orthonormal columns
    R: np.ndarray = None   # (m_used+1) x (m_used+1) upper triangular coefficients


def bg_basis(A, b, m: int, sketch) -> BGBasis:
    """Alg. 1 (§2.1.1, from Balabanov and Grigori): a basis whose sketch
    S = Theta V keeps orthonormal columns. Step i forms w = A v_{i-1} and its
    sketch p = Theta w, does one classical Gram-Schmidt step on the sketches
    (r = S^T p, s = p - S r, r_ii = ||s||), and applies the same coefficients to
    the long vectors: v_i = (w - V r) / r_ii. H_m is R without its first column;
    gamma_b = r_11. Breakdown as for Alg. 2, on the sketched norms."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    p = np.asarray(sketch.apply(b), dtype=np.float64).ravel()
    s = p.shape[0]
    V = np.zeros((n, m + 1))
    S = np.zeros((s, m + 1))
    R = np.zeros((m + 1, m + 1))
    r11 = float(np.linalg.norm(p))
    if r11 == 0.0:
        return BGBasis(V[:, :1], np.zeros((1, 0)), 0.0, 0, S[:, :1], R[:1, :1])
    R[0, 0] = r11
    S[:, 0] = p / r11
    V[:, 0] = b / r11
    for c in range(1, m + 1):
        w = A @ V[:, c - 1]
        p = np.asarray(sketch.apply(w), dtype=np.float64).ravel()
        r = S[:, :c].T @ p
        sv = p - S[:, :c] @ r
        rcc = float(np.linalg.norm(sv))
        R[:c, c] = r
        R[c, c] = rcc
        if not rcc > BG_BREAKDOWN * float(np.linalg.norm(p)):
            Vb = np.zeros((n, c + 1))
            Vb[:, :c] = V[:, :c]
            Hb = np.zeros((c + 1, c))
            Hb[:c, :c] = R[:c, 1 : c + 1]
            return BGBasis(Vb, Hb, r11, c, S[:, : c + 1], R[: c + 1, : c + 1])
        S[:, c] = sv / rcc
        V[:, c] = (w - V[:, :c] @ r) / rcc
    return BGBasis(V, R[:, 1:].copy(), r11, m, S, R)


@dataclass
class WBasis(BGBasis):
    wh: int = 0            # columns of V when it was whitened (0: never)
    kappas: np.ndarray = None   # kappa_1(R_i) for i = 1 .. (checked columns)


def _qr_pos(X):
    """Thin QR with a positive diagonal in R (the Gram-Schmidt convention)."""
    Q, R = np.linalg.qr(X)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d, R * d[:, None]


def nt_whiten_basis(A, b, m: int, k: int, sketch, kappa_max: float = WHITEN_KAPPA, orth: str = "cgs") -> WBasis:
    """Alg. 2 with a sketched basis and whitening (§2.1.2).

    After each new column the sketch Theta V_i (i columns) is factored, Theta V_i =
    Q_i R_i. While kappa_1(R_i) <= kappa_max the basis grows by Alg. 2. The first
    time it exceeds kappa_max the basis becomes V_i R_i^{-1}, the Hessenberg matrix
    R_i H_{i-1} R_{i-1}^{-1} (i x (i-1)), the sketch Theta V_i R_i^{-1} = Q_i, and
    the remaining columns are built by Alg. 1 with the same Theta. b = ||b|| v_1
    and v_1 = (V R^{-1}) R e_1 give gamma_b = ||b|| r_11 once whitened.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    beta = float(np.linalg.norm(b))
    sk0 = np.asarray(sketch.apply(np.zeros(n)), dtype=np.float64).ravel()
    S = np.zeros((sk0.shape[0], m + 1))
    if beta == 0.0:
        return WBasis(V[:, :1], H[:1, :0], 0.0, 0, S[:, :1], np.zeros((1, 1)), 0, np.zeros(0))
    V[:, 0] = b / beta
    S[:, 0] = np.asarray(sketch.apply(V[:, 0]), dtype=np.float64).ravel()
    gamma = beta
    wh = 0
    Rw = None
    kappas = [1.0]

    def truncated(c):
        Vb = np.zeros((n, c + 1))
        Vb[:, :c] = V[:, :c]
        Hb = np.zeros((c + 1, c))
        Hb[:c, :c] = H[:c, :c]
        return WBasis(Vb, Hb, gamma, c, S[:, : c + 1], Rw, wh, np.array(kappas))

    for c in range(1, m + 1):
        w = A @ V[:, c - 1]
        if wh == 0:  # Alg. 2 step
            wnorm = float(np.linalg.norm(w))
            win = list(range(max(0, c - k), c))
            if orth == "cgs":
                h = V[:, win].T @ w
                w = w - V[:, win] @ h
                H[win, c - 1] = h
            else:
                for j in win:
                    H[j, c - 1] = V[:, j] @ w
                    w = w - H[j, c - 1] * V[:, j]
            H[c, c - 1] = float(np.linalg.norm(w))
            if not H[c, c - 1] > 64 * EPS * wnorm:
                return truncated(c)
            V[:, c] = w / H[c, c - 1]
            S[:, c] = np.asarray(sketch.apply(V[:, c]), dtype=np.float64).ravel()
            i = c + 1
            Q, R = _qr_pos(S[:, :i])
            if not R[c, c] > BG_BREAKDOWN * float(np.linalg.norm(S[:, c])):
                return truncated(c)
            kap = float(np.linalg.norm(R, 1) * np.linalg.norm(np.linalg.inv(R), 1))
            kappas.append(kap)
            if kap > kappa_max:  # whiten V_i, H_{i-1} and the sketch
                Rinv = scipy.linalg.solve_triangular(R, np.eye(i), lower=False)
                V[:, :i] = V[:, :i] @ Rinv
                H[:i, : i - 1] = R @ H[:i, : i - 1] @ Rinv[: i - 1, : i - 1]
                S[:, :i] = Q
                gamma = beta * R[0, 0]
                wh = i
                Rw = R
        else:  # Alg. 1 step on the whitened basis
            p = np.asarray(sketch.apply(w), dtype=np.float64).ravel()
            r = S[:, :c].T @ p
            sv = p - S[:, :c] @ r
            rcc = float(np.linalg.norm(sv))
            H[:c, c - 1] = r
            H[c, c - 1] = rcc
            if not rcc > BG_BREAKDOWN * float(np.linalg.norm(p)):
                return truncated(c)
            S[:, c] = sv / rcc
            V[:, c] = (w - V[:, :c] @ r) / rcc
    return WBasis(V, H, gamma, m, S, Rw, wh, np.array(kappas))


def _breakdown(V, H, beta, c):
    """Basis of dimension c: V_c spans an invariant subspace (in exact arithmetic)."""
    Vb = np.zeros((V.shape[0], c + 1))
    Vb[:, :c] = V[:, :c]
    Hb = np.zeros((c + 1, c))
    Hb[:c, :c] = H[:c, :c]
    return Basis(Vb, Hb, beta, c)


def arnoldi(A, b, m: int, reorth: bool = False) -> Basis:
    """Arnoldi with modified Gram-Schmidt (eq. arnoldi, §2): an orthonormal
    basis U_{m+1} and Hessenberg K. ``reorth`` adds a second MGS pass."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    U = np.zeros((n, m + 1))
    K = np.zeros((m + 1, m))
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return Basis(U[:, :1], K[:1, :0], 0.0, 0)
    U[:, 0] = b / beta
    for c in range(1, m + 1):
        w = A @ U[:, c - 1]
        wnorm = float(np.linalg.norm(w))
        for _ in range(2 if reorth else 1):
            for j in range(c):
                hj = U[:, j] @ w
                K[j, c - 1] += hj
                w = w - hj * U[:, j]
        K[c, c - 1] = float(np.linalg.norm(w))
        if not K[c, c - 1] > 64 * EPS * wnorm:
            return _breakdown(U, K, beta, c)
        U[:, c] = w / K[c, c - 1]
    return Basis(U, K, beta, m)


# ---------------------------------------------------------------------------- LSQR
@dataclass
class LSQRResult:
    x: np.ndarray
    iters: int
    converged: bool


def lsqr(matvec, rmatvec, rhs: np.ndarray, ncols: int, tol: float, maxit: int) -> LSQRResult:
    """LSQR (Paige and Saunders 1982) for min ||Op x - rhs||_2 from x = 0.

    Golub-Kahan bidiagonalisation with the QR update of the bidiagonal by plane
    rotations. Stops when ||Op^T r|| <= tol * ||Op||_F-estimate * ||r|| (the
    method's least-squares stopping rule) or after maxit iterations.
    """
    x = np.zeros(ncols)
    beta = float(np.linalg.norm(rhs))
    if beta == 0.0:
        return LSQRResult(x, 0, True)
    u = rhs / beta
    v = rmatvec(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return LSQRResult(x, 0, True)
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = 0.0
    for it in range(1, maxit + 1):
        u = matvec(v) - alpha * u
        beta = float(np.linalg.norm(u))
        anorm2 += alpha * alpha + beta * beta
        if beta > 0.0:
            u = u / beta
            v = rmatvec(u) - beta * v
            alpha = float(np.linalg.norm(v))
            if alpha > 0.0:
                v = v / alpha
        rho = math.hypot(rhobar, beta)
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        if phibar * alpha * abs(c) <= tol * math.sqrt(anorm2) * phibar or beta == 0.0 or alpha == 0.0:
            return LSQRResult(x, it, True)
    return LSQRResult(x, maxit, False)


# ------------------------------------------------------------------------- methods
@dataclass
class Result:
    x: np.ndarray
    m_used: int
    coeffs: np.ndarray          # c with x = gamma * V_m c (gamma = ||b||) where applicable
    Hhat: np.ndarray | None = None
    y: np.ndarray | None = None
    SV: np.ndarray | None = None
    R: np.ndarray | None = None
    lsqr_iters: int = 0
    basis: Basis | None = None


def fm_arnoldi(A, b, m: int, f: int, t: float = 1.0, coef=None, reorth: bool = False) -> Result:
    """Standard Krylov approximation f_m = ||b|| U_m f(K_m) e_1 (eq. standardfm)."""
    B = arnoldi(A, b, m, reorth=reorth)
    mu = B.m_used
    if mu == 0:
        return Result(np.zeros_like(b, dtype=np.float64), 0, np.zeros(0), basis=B)
    c = matfun.f_e1(B.H[:mu, :mu], f, t, coef)
    return Result(B.beta * (B.V[:, :mu] @ c), mu, c, Hhat=B.H[:mu, :mu], basis=B)


def noproj(A, b, m: int, k: int, f: int, t: float = 1.0, coef=None, orth: str = "cgs") -> Result:
    """Alg. 5: ||b|| V_m f(H_m) e_1, no least-squares solve (eq. noproj)."""
    B = nt_basis(A, b, m, k, orth)
    mu = B.m_used
    if mu == 0:
        return Result(np.zeros_like(b, dtype=np.float64), 0, np.zeros(0), basis=B)
    c = matfun.f_e1(B.H[:mu, :mu], f, t, coef)
    return Result(B.beta * (B.V[:, :mu] @ c), mu, c, Hhat=B.H[:mu, :mu], basis=B)


def _last_column_update(B: Basis, y: np.ndarray) -> np.ndarray:
    """H_m + h_{m+1,m} y e_m^T (eq. relationxx)."""
    return last_column_update(B.H[: B.m_used + 1, : B.m_used], y)


def last_column_update(H: np.ndarray, y: np.ndarray) -> np.ndarray:
    """H_m + h_{m+1,m} y e_m^T (eq. relationxx) for the (m+1) x m Hessenberg H."""
    mu = H.shape[1]
    Hhat = H[:mu, :mu].copy()
    Hhat[:, mu - 1] += H[mu, mu - 1] * y
    return Hhat


def sketch_solve_stage(H: np.ndarray, SV: np.ndarray, f: int, t: float = 1.0, coef=None):
    """The small stage of the sketch-and-solve form (Remark after eq. sFOM) from the
    (m+1) x m Hessenberg H and the sketched basis SV = Theta V_{m+1} (s x (m+1)):
    Theta V_m = S R (thin QR), y = R^{-1} S^T Theta v_{m+1} (the least-squares
    solution of min ||Theta (V_m z - v_{m+1})||), then c = f(H_m + h_{m+1,m} y e_m^T) e_1.
    Returns (y, Hhat, c, R)."""
    mu = H.shape[1]
    S, R = np.linalg.qr(SV[:, :mu])
    y = scipy.linalg.solve_triangular(R, S.T @ SV[:, mu], lower=False)
    Hhat = last_column_update(H, y)
    c = matfun.f_e1(Hhat, f, t, coef)
    return y, Hhat, c, R


def sketched_ls(A, b, m: int, k: int, f: int, sketch, t: float = 1.0, coef=None,
                tol: float = 1e-14, maxit: int | None = None, orth: str = "cgs",
                exact_ls: bool = False) -> Result:
    """Alg. 4: y = argmin ||V_m z - v_{m+1}|| by Blendenpik (QR of Theta V_m gives
    the preconditioner R; LSQR on V_m R^{-1}), then ||b|| V_m f(H_m + h y e_m^T) e_1.
    ``exact_ls`` solves the least-squares problem densely instead (for pins)."""
    B = nt_basis(A, b, m, k, orth)
    mu = B.m_used
    if mu == 0:
        return Result(np.zeros_like(b, dtype=np.float64), 0, np.zeros(0), basis=B)
    Vm, vlast = B.V[:, :mu], B.V[:, mu]
    SV = sketch.apply(Vm)
    R = np.linalg.qr(SV, mode="r")
    if exact_ls:
        y = np.linalg.lstsq(Vm, vlast, rcond=None)[0]
        iters = 0
    else:
        def mv(z):
            return Vm @ scipy.linalg.solve_triangular(R, z, lower=False)

        def rmv(u):
            return scipy.linalg.solve_triangular(R, Vm.T @ u, lower=False, trans="T")

        res = lsqr(mv, rmv, vlast, mu, tol, maxit if maxit is not None else 4 * mu)
        y = scipy.linalg.solve_triangular(R, res.x, lower=False)
        iters = res.iters
    Hhat = _last_column_update(B, y)
    c = matfun.f_e1(Hhat, f, t, coef)
    return Result(B.beta * (Vm @ c), mu, c, Hhat=Hhat, y=y, SV=SV, R=R, lsqr_iters=iters, basis=B)


def sketched_fast(A, b, m: int, k: int, f: int, sketch, t: float = 1.0, coef=None,
                  orth: str = "cgs", form: str = "sfom", sav: str = "direct") -> Result:
    """The sketched variant working on Theta V and Theta A V only.

    form="sfom": eq. sFOM, V_m R^{-1} f(S_m^T Theta A V_m R^{-1}) S_m^T Theta b with
                 Theta V_m = S_m R_m (thin QR).
    form="sketch_solve": the Remark after eq. sFOM, y = argmin ||Theta(V_m z - v_{m+1})||,
                 then ||b|| V_m f(H_m + h y e_m^T) e_1.
    sav="direct" sketches A V_m column by column; sav="relation" uses
    Theta V_{m+1} H_m (eq. arnoldilike).
    """
    B = nt_basis(A, b, m, k, orth)
    mu = B.m_used
    if mu == 0:
        return Result(np.zeros_like(b, dtype=np.float64), 0, np.zeros(0), basis=B)
    Vm = B.V[:, :mu]
    SVfull = sketch.apply(B.V[:, : mu + 1])
    if form == "sketch_solve":
        y, Hhat, c, R = sketch_solve_stage(B.H[: mu + 1, :mu], SVfull, f, t, coef)
        return Result(B.beta * (Vm @ c), mu, c, Hhat=Hhat, y=y, SV=SVfull, R=R, basis=B)
    SV = SVfull[:, :mu]
    S, R = np.linalg.qr(SV)
    if sav == "direct":
        SAV = sketch.apply(np.column_stack([A @ Vm[:, j] for j in range(mu)]))
    else:
        SAV = SVfull @ B.H[: mu + 1, :mu]
    # M = S^T (Theta A V_m) R^{-1}, i.e. M R = S^T Theta A V_m
    M = scipy.linalg.solve_triangular(R, (S.T @ SAV).T, lower=False, trans="T").T
    Sb = sketch.apply(np.asarray(b, dtype=np.float64))
    z = matfun.f_apply(M, S.T @ Sb, f, t, coef)
    c = scipy.linalg.solve_triangular(R, z, lower=False)
    return Result(Vm @ c, mu, c / B.beta, SV=SVfull, R=R, basis=B)


def bg_ls(A, b, m: int, f: int, sketch, t: float = 1.0, coef=None, tol: float = 1e-14, maxit: int | None = None,
          exact_ls: bool = False) -> Result:
    """Alg. 3: the basis of Alg. 1, y = argmin ||V_m z - v_{m+1}|| by LSQR without a
    preconditioner (the basis is well conditioned, §3.1.1), then
    r_11 V_m f(H_m + h_{m+1,m} y e_m^T) e_1. ``exact_ls`` solves densely (pins)."""
    B = bg_basis(A, b, m, sketch)
    mu = B.m_used
    if mu == 0:
        return Result(np.zeros_like(b, dtype=np.float64), 0, np.zeros(0), basis=B)
    Vm, vlast = B.V[:, :mu], B.V[:, mu]
    if mu < m:  # invariant subspace: v_{m+1} does not exist, Hhat = H_m
        y, iters = np.zeros(mu), 0
    elif exact_ls:
        y, iters = np.linalg.lstsq(Vm, vlast, rcond=None)[0], 0
    else:
        res = lsqr(lambda z: Vm @ z, lambda u: Vm.T @ u, vlast, mu, tol, maxit if maxit is not None else 4 * mu)
        y, iters = res.x, res.iters
    Hhat = _last_column_update(B, y)
    c = matfun.f_e1(Hhat, f, t, coef)
    return Result(B.beta * (Vm @ c), mu, c, Hhat=Hhat, y=y, SV=B.S, R=B.R, lsqr_iters=iters, basis=B)


def whiten(A, b, m: int, k: int, f: int, sketch, t: float = 1.0, coef=None, kappa_max: float = WHITEN_KAPPA,
           tol: float = 1e-14, maxit: int | None = None, exact_ls: bool = False, final: str = "auto",
           orth: str = "cgs") -> Result:
    """Alg. 2 with whitening and a switch to Alg. 1 (§2.1.2), finished as §6
    recommends: a basis that stayed well conditioned gives Alg. 5's
    ||b|| V_m f(H_m) e_1; a whitened one Alg. 3's gamma_b V_m f(H_m + h y e_m^T) e_1
    with y = argmin ||V_m z - v_{m+1}|| by LSQR (no preconditioner: Theta V is
    orthonormal). ``final="noproj"`` forces Alg. 5 on the whitened basis (which
    §3.3 shows equals eq. sFOM)."""
    B = nt_whiten_basis(A, b, m, k, sketch, kappa_max, orth)
    mu = B.m_used
    if mu == 0:
        return Result(np.zeros_like(b, dtype=np.float64), 0, np.zeros(0), basis=B)
    Vm, iters, y = B.V[:, :mu], 0, None
    if B.wh == 0 or final == "noproj" or mu < m:
        Hhat = B.H[:mu, :mu]
    else:
        vlast = B.V[:, mu]
        if exact_ls:
            y = np.linalg.lstsq(Vm, vlast, rcond=None)[0]
        else:
            res = lsqr(lambda z: Vm @ z, lambda u: Vm.T @ u, vlast, mu, tol, maxit if maxit is not None else 4 * mu)
            y, iters = res.x, res.iters
        Hhat = _last_column_update(B, y)
    c = matfun.f_e1(Hhat, f, t, coef)
    return Result(B.beta * (Vm @ c), mu, c, Hhat=Hhat, y=y, SV=B.S, R=B.R, lsqr_iters=iters, basis=B)


def run(method: int, A, b, m: int, k: int, f: int, sketch=None, t: float = 1.0, **kw) -> Result:
    """Dispatch on the library's method enum. f = SIGN runs the method on A^2 with
    the starting vector A b and f = inverse square root (§5.1.3)."""
    if f == matfun.SIGN:
        b = A @ np.asarray(b, dtype=np.float64)
        A = A @ A
        f = matfun.INVSQRT
    if method == ARNOLDI:
        return fm_arnoldi(A, b, m, f, t, reorth=kw.get("reorth", False))
    if method == NOPROJ:
        return noproj(A, b, m, k, f, t, orth=kw.get("orth", "cgs"))
    if method == SKETCHED_LS:
        return sketched_ls(A, b, m, k, f, sketch, t, tol=kw.get("tol", 1e-14), maxit=kw.get("maxit"),
                           orth=kw.get("orth", "cgs"))
    if method == SKETCHED_FAST:
        return sketched_fast(A, b, m, k, f, sketch, t, orth=kw.get("orth", "cgs"),
                             form=kw.get("form", "sketch_solve"))
    if method == BG_LS:
        return bg_ls(A, b, m, f, sketch, t, tol=kw.get("tol", 1e-14), maxit=kw.get("maxit"))
    if method == WHITEN:
        return whiten(A, b, m, k, f, sketch, t, kappa_max=kw.get("kappa_max", WHITEN_KAPPA),
                      tol=kw.get("tol", 1e-14), maxit=kw.get("maxit"), final=kw.get("final", "auto"))
    raise ValueError("unknown method")
