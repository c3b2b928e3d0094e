"""f(M) z for the small projected matrix, and exact f(A)b for small n.

The paper evaluates f on the compressed matrix with MATLAB ``expm`` and
``sqrtm`` (§5); the oracle uses SciPy's ``expm`` and ``sqrtm`` as the same
kind of library primitive. The functions are those of the library's ABI:
  EXP     f(z) = exp(t z)   (exp(tA) b; the Krylov space of A equals that of tA)
  SQRT    f(z) = z^{1/2}    (principal square root)
  INVSQRT f(z) = z^{-1/2}
POLY (oracle only) evaluates a polynomial sum_i coef[i] z^i, for the
polynomial-exactness pins of the paper's Theorem thm:lastcol.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

EXP, SQRT, INVSQRT, POLY = 0, 1, 2, 99
# sign(A) b, computed as (A^2)^{-1/2} (A b) (§5.1.3, after Higham's Chapter 5): a
# transformation of the problem (see krylov.run), not a function of the small H.
SIGN = 3


def _real(X: np.ndarray) -> np.ndarray:
    if np.iscomplexobj(X):
        scale = max(1.0, float(np.abs(X).max()))
        if float(np.abs(X.imag).max()) > 1e-8 * scale:
            raise ValueError("principal square root is not real for this matrix")
        X = X.real
    return np.asarray(X, dtype=np.float64)


def sqrtm(M: np.ndarray) -> np.ndarray:
    return _real(scipy.linalg.sqrtm(np.asarray(M, dtype=np.float64)))


def f_apply(M: np.ndarray, z: np.ndarray, f: int, t: float = 1.0, coef=None) -> np.ndarray:
    """f(M) @ z."""
    M = np.asarray(M, dtype=np.float64)
    if f == EXP:
        return scipy.linalg.expm(t * M) @ z
    if f == SQRT:
        return sqrtm(M) @ z
    if f == INVSQRT:
        return np.linalg.solve(sqrtm(M), z)
    if f == POLY:
        acc = np.zeros_like(np.asarray(z, dtype=np.float64))
        for cf in reversed(list(coef)):  # Horner
            acc = M @ acc + cf * z
        return acc
    raise ValueError("unknown f")


def f_e1(M: np.ndarray, f: int, t: float = 1.0, coef=None) -> np.ndarray:
    """f(M) e_1."""
    e1 = np.zeros(M.shape[0])
    e1[0] = 1.0
    return f_apply(M, e1, f, t, coef)


def f_scalar(lam, f: int, t: float = 1.0, coef=None):
    """f on scalars (eigenvalues)."""
    lam = np.asarray(lam)
    if f == EXP:
        return np.exp(t * lam)
    if f == SQRT:
        return np.sqrt(lam)
    if f == INVSQRT:
        return 1.0 / np.sqrt(lam)
    if f == POLY:
        return sum(cf * lam**i for i, cf in enumerate(coef))
    raise ValueError("unknown f")


def exact_fAb(A_dense: np.ndarray, b: np.ndarray, f: int, t: float = 1.0, coef=None) -> np.ndarray:
    """Dense f(A) b (small n): expm / sqrtm as in the paper's reference values (§5);
    sign by scipy's signm."""
    A_dense = np.asarray(A_dense, dtype=np.float64)
    if f == SIGN:
        return _real(scipy.linalg.signm(A_dense)) @ np.asarray(b, dtype=np.float64)
    return f_apply(A_dense, np.asarray(b, dtype=np.float64), f, t, coef)
