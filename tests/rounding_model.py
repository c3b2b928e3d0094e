"""The rounding model the mixed-precision GPU tests derive their bars from (test
infrastructure: numpy only, drives the FP64 oracle).

The FP32 basis and the BF16 copy the Gaussian sketch reads are modelled by
perturbing the oracle's own arithmetic with random rounding errors of the stated
size; the bar of a comparison is TAIL times the RMS change of the oracle's result
over DRAWS draws. To first order the error is a linear function of many
independent rounding errors, close to Gaussian, so a draw beyond TAIL = 4 RMS is rare.
"""
import numpy as np

from oracle import krylov
from oracle import sketch as osk


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


U32 = 2.0**-24   # unit roundoff of FP32
U_BF16 = 2.0**-8  # unit roundoff of BF16 (8 significant bits): round to nearest moves x by <= 2^-8 |x|
DRAWS = 16        # draws of the rounding model
TAIL = 4.0        # bar = TAIL x the model's RMS error


class _Fp32Operator:
    """The rounding model of the FP32 basis (probabilistic rounding analysis, Higham
    and Mary 2019: N independent roundings of relative size <= u move a sum by about
    sqrt(N) u times its terms): A_32 v, with A_32 the FP32 copy of A the device
    multiplies by, and every entry moved by xi_i (|A_32| |v|)_i, xi_i uniform on
    [-g_i, g_i], g_i = sqrt(nnz_i + k + 2) u_32 (the row's FMA chain, the window update's
    k FMAs and the FP32 store of the new vector); fresh draws per product."""

    def __init__(self, As, k, rng):
        self.A = As.copy()
        self.A.data = self.A.data.astype(np.float32).astype(np.float64)
        self.absA, self.rng = abs(self.A), rng
        self.g = np.sqrt(np.diff(As.indptr) + k + 2.0) * U32

    def __matmul__(self, v):
        v = np.asarray(v, dtype=np.float64)
        return self.A @ v + self.rng.uniform(-1.0, 1.0, v.shape[0]) * self.g * (self.absA @ np.abs(v))


class _Bf16Sketch:
    """The rounding model of the tensor-core Gaussian sketch: G applied to the basis
    columns split into two BF16 terms (hi + lo, each rounded to nearest, ties to even)
    at a random scale 2^u_j, u_j uniform on [0, 1) per column (the device splits the
    unnormalized column, whose scale against a power of two is arbitrary); G itself is
    exact in BF16. The FP32 accumulation of the products (about sqrt(K) u_32 for K
    terms per split) is not modelled: it is of the size of the split's 2^-16."""

    def __init__(self, th, rng):
        self.th, self.rng = th, rng

    def apply(self, V):
        V = np.asarray(V, dtype=np.float64)
        one = V.ndim == 1
        V2 = V[:, None] if one else V
        c = 2.0 ** self.rng.uniform(0.0, 1.0, V2.shape[1])
        cols = []
        for j0 in range(0, V2.shape[1], 8):  # a few columns at a time: bounded temporaries
            hi, lo = osk.split_bf16(V2[:, j0:j0 + 8] * c[j0:j0 + 8])
            cols.append(self.th.apply((hi + lo) / c[j0:j0 + 8]))
        out = np.concatenate(cols, axis=1)
        return out[:, 0] if one else out


def model_rms(As, b, m, k, f, th, t, method, ref_x, gauss, seed=11):
    """RMS relative change of the oracle's f_m over DRAWS draws of the rounding model
    (FP32 products and, with the Gaussian sketch, the BF16 copy of the basis)."""
    rng = np.random.default_rng(seed)
    errs = []
    for _ in range(DRAWS):
        op = _Fp32Operator(As, k, rng)
        sk = _Bf16Sketch(th, rng) if gauss else th
        r = krylov.run(method, op, b, m, k, f, sk, t, tol=1e-10)
        errs.append(_rel(r.x, ref_x))
    return float(np.sqrt(np.mean(np.square(errs)))), float(np.max(errs))
