"""Writes c3_gauss.txt: the FP64 oracle's sketched_fast solves of the power-law graph
workload (Chung-Lu Laplacian + 0.1 I, n = 4,000,000, graph seed 2; b from seed 0;
m = 150, k = 2, Gaussian sketch s = 600, sketch seed 1; f = A^{-1/2} and A^{1/2}; the
sketch-and-solve form of the Remark after eq. sFOM), and the RMS relative change of
each solution under DRAWS draws of the rounding model of the FP32 basis and the
two-term BF16 sketch (tests/rounding_model.py, which drives only the oracle). For each
f the file holds the coefficient vector c, ||x||_2, x at 1024 rows drawn with numpy
default_rng(12345), and the model's RMS. G's entries are BF16 values, held exactly in
FP32 so that the 600 x n matrix is generated once. Calls only oracle/, the seeded input
generators and the rounding model. Run: python tests/golden/make_c3_reference.py
(about a quarter of an hour on 8 cores, 30 GB of memory).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import krylov, matfun  # noqa: E402
from oracle import sketch as osk  # noqa: E402
from paper_2212_12758_gb300 import workloads as W  # noqa: E402
import rounding_model as RM  # noqa: E402

N, M, K, S, SEED = 4_000_000, 150, 2, 600, 1
SAMPLE, DRAWS = 1024, 8


class StoredGaussian:
    """The Gaussian sketch of oracle/sketch.py with G generated once, 16 rows at a time,
    and kept in FP32 (exact for its BF16 entries); applied in FP64."""

    def __init__(self, n, s, seed, block=16):
        self.s, self.block = s, block
        self.G = np.empty((s, n), dtype=np.float32)
        for q0 in range(0, s, block):
            rows = np.arange(q0, min(s, q0 + block))
            self.G[rows] = osk.gaussian_entries(s, n, seed, rows=rows, bf16=True).astype(np.float32)

    def apply(self, V):
        V = np.asarray(V, dtype=np.float64)
        out = np.empty((self.s,) + V.shape[1:])
        for q0 in range(0, self.s, self.block):
            out[q0:q0 + self.block] = self.G[q0:q0 + self.block].astype(np.float64) @ V
        return out


def solves(B, SV, fs):
    out = {}
    for name, f in fs:
        _, _, c, _ = krylov.sketch_solve_stage(B.H[: M + 1, :M], SV, f, 1.0)
        out[name] = (c, B.beta * (B.V[:, :M] @ c))
    return out


def main():
    A = W.chung_lu_laplacian(N, seed=2)
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    th = StoredGaussian(A.n, S, SEED)
    fs = (("invsqrt", matfun.INVSQRT), ("sqrt", matfun.SQRT))
    B = krylov.nt_basis(As, b, M, K)
    assert B.m_used == M
    ref = solves(B, th.apply(B.V), fs)
    del B
    rng = np.random.default_rng(11)
    errs = {name: [] for name, _ in fs}
    for _ in range(DRAWS):
        Bd = krylov.nt_basis(RM._Fp32Operator(As, K, rng), b, M, K)
        got = solves(Bd, RM._Bf16Sketch(th, rng).apply(Bd.V), fs)
        del Bd
        for name, _ in fs:
            errs[name].append(float(np.linalg.norm(got[name][1] - ref[name][1]) / np.linalg.norm(ref[name][1])))
    idx = np.sort(np.random.default_rng(12345).choice(A.n, SAMPLE, replace=False))
    with open(os.path.join(HERE, "c3_gauss.txt"), "w") as fh:
        fh.write("# oracle sketched_fast, Chung-Lu Laplacian n=4M (+0.1 I), m=150 k=2 Gaussian s=600 seed 1\n")
        fh.write(f"# written by tests/golden/make_c3_reference.py (oracle + rounding model, {DRAWS} draws)\n")
        fh.write(f"nnz {A.nnz}\n")
        for name, _ in fs:
            c, x = ref[name]
            fh.write(f"{name} model_rms {float(np.sqrt(np.mean(np.square(errs[name])))):.6e}\n")
            fh.write(f"{name} xnorm {np.linalg.norm(x):.17e}\n")
            fh.write(f"{name} coeffs " + " ".join(f"{v:.17e}" for v in c) + "\n")
            for i in idx:
                fh.write(f"{name} x {int(i)} {x[i]:.17e}\n")


if __name__ == "__main__":
    main()
