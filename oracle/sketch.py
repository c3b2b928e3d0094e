"""Sketch operators Theta in R^{s x n} (paper §2.1.1), written from their definitions.

SRHT (paper §2.1.1, Tropp 2011): Theta = s^{-1/2} P H D. The input is zero-padded
to n' = 2^ceil(log2 n); D = diag(+-1) Rademacher; H is the n' x n' Walsh-Hadamard
matrix in Sylvester order, H[r, j] = (-1)^popcount(r & j); P selects s distinct
rows of [0, n') drawn uniformly (Floyd's algorithm), sorted ascending.
  D_j  = -1 iff bit (j mod 64) of u(seed, 3, j div 64) is set.
  P    : for i = 0..s-1 with j = n' - s + i, t = floor(u(seed, 4, i) * (j+1) / 2^64);
         take t unless already taken, else take j.

Sparse sign (mentioned in §2.1.1; defined in Martinsson-Tropp 2020 §9.2): every
column j of Theta has zeta nonzeros +-1/sqrt(zeta) in distinct rows.
  Candidate rows for column j, in draw order t = 0..255: the low (t even) or high
  (t odd) 32-bit half x of u(seed, 1, 128*j + t div 2), row = floor(x * s / 2^32).
  The first zeta distinct candidates are the rows (q = 0..zeta-1 in that order);
  if fewer than zeta are distinct after 256 candidates, the smallest unused rows
  are appended in increasing order.
  The sign of the q-th row is -1 iff bit q of u(seed, 2, j) is set.

Gaussian (not in the paper; the dense sketch whose application is a GEMM): entry
(q, j) is g / sqrt(s) with g = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller), where for
idx = q*n + j, u1 = ((u(seed,5,2 idx) >> 11) + 1) 2^-53 and
u2 = (u(seed,5,2 idx+1) >> 11) 2^-53; optionally rounded to bfloat16 (nearest,
ties to even) directly from the FP64 value.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse

from . import rng

SPARSE_SIGN, SRHT, GAUSSIAN = 0, 1, 2


def next_pow2(n: int) -> int:
    return 1 << max(0, (int(n) - 1).bit_length())


# ----------------------------------------------------------------------------- SRHT
def srht_signs(npad: int, seed: int) -> np.ndarray:
    """Diagonal of D (length n'), entries +-1."""
    j = np.arange(npad, dtype=np.uint64)
    words = rng.u(seed, rng.STREAM_SRHT_D, j >> np.uint64(6))
    bits = (words >> (j & np.uint64(63))) & np.uint64(1)
    return 1.0 - 2.0 * bits.astype(np.float64)


def srht_rows(npad: int, s: int, seed: int) -> np.ndarray:
    """The sampled rows P (sorted, distinct) by Floyd's algorithm."""
    if s > npad:
        raise ValueError("SRHT needs s <= n' = next power of two >= n")
    chosen: set[int] = set()
    for i in range(s):
        j = npad - s + i
        t = rng.mulhi64_int(rng.u_int(seed, rng.STREAM_SRHT_P, i), j + 1)
        chosen.add(j if t in chosen else t)
    return np.array(sorted(chosen), dtype=np.int64)


def _hadamard_apply(X: np.ndarray) -> np.ndarray:
    """H_{n'} X for X of shape (n', c), n' a power of two, by the Kronecker
    factorisation H_{2^(a+b+..)} = H_{2^a} (x) H_{2^b} (x) ... of the Sylvester
    matrix (index bits split into contiguous fields)."""
    npad, c = X.shape
    p = npad.bit_length() - 1
    fields = []
    while p > 0:
        f = min(8, p)
        fields.append(f)
        p -= f
    if not fields:
        return X.copy()
    T = X.reshape([1 << f for f in fields] + [c])
    for ax, f in enumerate(fields):
        Hf = scipy.linalg.hadamard(1 << f).astype(np.float64)
        T = np.moveaxis(np.tensordot(Hf, T, axes=([1], [ax])), 0, ax)
    return np.ascontiguousarray(T).reshape(npad, c)


class SRHT_:
    def __init__(self, n: int, s: int, seed: int):
        self.n, self.s, self.seed = n, s, seed
        self.npad = next_pow2(n)
        self.D = srht_signs(self.npad, seed)
        self.P = srht_rows(self.npad, s, seed)

    def apply(self, V: np.ndarray, chunk: int = 8) -> np.ndarray:
        V = np.asarray(V, dtype=np.float64)
        one = V.ndim == 1
        V2 = V[:, None] if one else V
        out = np.empty((self.s, V2.shape[1]))
        for c0 in range(0, V2.shape[1], chunk):
            c1 = min(V2.shape[1], c0 + chunk)
            X = np.zeros((self.npad, c1 - c0))
            X[: self.n] = self.D[: self.n, None] * V2[:, c0:c1]
            out[:, c0:c1] = _hadamard_apply(X)[self.P] / math.sqrt(self.s)
        return out[:, 0] if one else out

    def dense(self) -> np.ndarray:
        """Theta as a dense s x n matrix, from the entry formula (tiny n only)."""
        r = self.P[:, None]
        j = np.arange(self.n)[None, :]
        pc = np.vectorize(lambda x: bin(int(x)).count("1"))(r & j)
        return ((-1.0) ** pc) * self.D[None, : self.n] / math.sqrt(self.s)


# ------------------------------------------------------------------------ sparse sign
def sparse_sign_rows(n: int, s: int, zeta: int, seed: int):
    """Rows (n x zeta, draw order) and signs (n x zeta, +-1) of a sparse sign sketch."""
    if not (1 <= zeta <= min(s, 64)):
        raise ValueError("sparse sign needs 1 <= zeta <= min(s, 64)")
    j = np.arange(n, dtype=np.uint64)
    rows = np.full((n, zeta), -1, dtype=np.int64)
    count = np.zeros(n, dtype=np.int64)
    first = 32  # candidates examined in the vectorised pass
    for t in range(first):
        h = rng.u(seed, rng.STREAM_SPARSE_ROWS, j * np.uint64(128) + np.uint64(t // 2))
        half = (h & np.uint64(0xFFFFFFFF)) if t % 2 == 0 else (h >> np.uint64(32))
        cand = rng.mulhi32(half, s).astype(np.int64)
        dup = (rows == cand[:, None]).any(axis=1)
        take = (~dup) & (count < zeta)
        idx = np.nonzero(take)[0]
        rows[idx, count[idx]] = cand[idx]
        count[idx] += 1
    for col in np.nonzero(count < zeta)[0]:  # rare: continue the same draw sequence
        have = list(rows[col, : count[col]])
        for t in range(first, 256):
            h = rng.u_int(seed, rng.STREAM_SPARSE_ROWS, 128 * int(col) + t // 2)
            half = (h & 0xFFFFFFFF) if t % 2 == 0 else (h >> 32)
            cand = (half * s) >> 32
            if cand not in have:
                have.append(cand)
                if len(have) == zeta:
                    break
        r = 0
        while len(have) < zeta:
            if r not in have:
                have.append(r)
            r += 1
        rows[col] = have
    words = rng.u(seed, rng.STREAM_SPARSE_SIGNS, j)
    q = np.arange(zeta, dtype=np.uint64)
    bits = (words[:, None] >> q[None, :]) & np.uint64(1)
    signs = 1.0 - 2.0 * bits.astype(np.float64)
    return rows, signs


class SparseSign:
    def __init__(self, n: int, s: int, zeta: int, seed: int):
        self.n, self.s, self.zeta, self.seed = n, s, zeta, seed
        self.rows, self.signs = sparse_sign_rows(n, s, zeta, seed)
        cols = np.repeat(np.arange(n), zeta)
        self.matrix = scipy.sparse.csr_matrix(
            (self.signs.ravel() / math.sqrt(zeta), (self.rows.ravel(), cols)), shape=(s, n))

    def apply(self, V: np.ndarray) -> np.ndarray:
        return self.matrix @ np.asarray(V, dtype=np.float64)

    def dense(self) -> np.ndarray:
        return self.matrix.toarray()


# -------------------------------------------------------------------------- Gaussian
def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest bfloat16 (ties to even), returned as FP64."""
    x = np.asarray(x, dtype=np.float64)
    bits = x.view(np.uint64).copy()
    sign = bits & np.uint64(1 << 63)
    mag = bits & np.uint64((1 << 63) - 1)
    keep = mag >> np.uint64(45)            # exponent(11) | top 7 mantissa bits
    rem = mag & np.uint64((1 << 45) - 1)
    half = np.uint64(1 << 44)
    up = (rem > half) | ((rem == half) & ((keep & np.uint64(1)) == np.uint64(1)))
    keep = keep + up.astype(np.uint64)     # a carry into the exponent is the correct result
    out = (sign | (keep << np.uint64(45))).view(np.float64)
    return np.where(x == 0, x, out)


def split_bf16(x: np.ndarray):
    """x as a sum of two bfloat16 numbers: hi = round_bf16(x), lo = round_bf16(x - hi)
    (x - hi is exact in FP64). hi + lo is x to 2^-16 relative, hi alone to 2^-8."""
    x = np.asarray(x, dtype=np.float64)
    hi = round_bf16(x)
    return hi, round_bf16(x - hi)


def gaussian_entries(s: int, n: int, seed: int, rows=None, bf16: bool = True) -> np.ndarray:
    """Rows `rows` (default all) of the Gaussian sketch, as FP64 values."""
    rows = np.arange(s) if rows is None else np.asarray(rows)
    idx = rows[:, None].astype(np.uint64) * np.uint64(n) + np.arange(n, dtype=np.uint64)[None, :]
    h1 = rng.u(seed, rng.STREAM_GAUSS, np.uint64(2) * idx)
    h2 = rng.u(seed, rng.STREAM_GAUSS, np.uint64(2) * idx + np.uint64(1))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0**-53
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2) / math.sqrt(s)
    return round_bf16(g) if bf16 else g


class Gaussian:
    def __init__(self, n: int, s: int, seed: int, bf16: bool = True):
        self.n, self.s, self.seed = n, s, seed
        self.G = gaussian_entries(s, n, seed, bf16=bf16)

    def apply(self, V):
        return self.G @ np.asarray(V, dtype=np.float64)

    def dense(self):
        return self.G


def make(kind: int, n: int, s: int, seed: int, zeta: int = 8):
    if kind == SPARSE_SIGN:
        return SparseSign(n, s, zeta, seed)
    if kind == SRHT:
        return SRHT_(n, s, seed)
    if kind == GAUSSIAN:
        return Gaussian(n, s, seed)
    raise ValueError("unknown sketch kind")
