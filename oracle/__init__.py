"""Plain FP64 CPU oracle for randomized Krylov f(A)b (arXiv 2212.12758).

TEST INFRASTRUCTURE ONLY. This package is the independent reference that the
CUDA library is checked against. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its CPU-baseline leg and its ``--impl reference`` arm) may
import it. It shares no code with the CUDA path and never imports it.

Everything is written to be read against the paper: numpy/scipy library
primitives (sparse mat-vec, dense QR, expm, sqrtm, Hadamard matrices) serve as
steps, and no blocking, fusion or reordering is added beyond what each
algorithm states.

Modules
-------
rng      SplitMix64 counter-based generator (Steele, Lea, Flood 2014).
sketch   Sketch operators Theta: SRHT (§2.1.1), sparse sign (§2.1.1, defined in
         Martinsson-Tropp §9), Gaussian (dense N(0, 1/s)).
krylov   Alg. 2 (truncated orthogonalization), Arnoldi (eq. arnoldi), Alg. 4
         (sketched LS with Blendenpik + LSQR), Alg. 5 (no LS solve), sFOM
         (eq. sFOM) and its sketch-and-solve form (Remark in §3.3).
matfun   f(H) e_1 for the small projected matrix, and exact f(A)b for small n.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, brute force on tiny inputs, the paper's theorems); none is
"parity unpinned".
"""
from . import rng, sketch, krylov, matfun  # noqa: F401
