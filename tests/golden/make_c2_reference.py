"""Writes c2_sketched_fast.txt: the FP64 oracle's sketched_fast solve of the 3D
convection-diffusion workload (200^3 grid, n = 8,000,000; exp(-1e-3 A) b with b from
seed 0; m = 100, k = 4, SRHT s = 400, sketch seed 1; the sketch-and-solve form of the
Remark after eq. sFOM). The file holds the coefficient vector c (x = ||b|| V_m c),
||x||_2, and x at 1024 rows drawn with numpy default_rng(12345). Calls only oracle/
and the seeded input generators. Run: python tests/golden/make_c2_reference.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import krylov, matfun  # noqa: E402
from oracle import sketch as osk  # noqa: E402
from paper_2212_12758_gb300 import workloads as W  # noqa: E402

N, M, K, S, T = 200, 100, 4, 400, -1e-3
SAMPLE = 1024


def main():
    A = W.convdiff(3, N)
    b = W.random_vector(A.n, 0)
    th = osk.SRHT_(A.n, S, 1)
    r = krylov.sketched_fast(W.to_scipy(A), b, M, K, matfun.EXP, th, T, form="sketch_solve")
    idx = np.sort(np.random.default_rng(12345).choice(A.n, SAMPLE, replace=False))
    with open(os.path.join(HERE, "c2_sketched_fast.txt"), "w") as f:
        f.write("# oracle sketched_fast, 3D convection-diffusion 200^3, exp(-1e-3 A) b, m=100 k=4 SRHT s=400 seed 1\n")
        f.write("# written by tests/golden/make_c2_reference.py (oracle only)\n")
        f.write(f"m_used {r.m_used}\n")
        f.write(f"xnorm {np.linalg.norm(r.x):.17e}\n")
        f.write("coeffs " + " ".join(f"{v:.17e}" for v in r.coeffs) + "\n")
        for i in idx:
            f.write(f"x {int(i)} {r.x[i]:.17e}\n")


if __name__ == "__main__":
    main()
