"""Randomized Krylov f(A)b on GB300 (arXiv 2212.12758).

The CUDA library and its ctypes binding live in ``paper_2212_12758_gb300.fab``;
it is imported explicitly (``from paper_2212_12758_gb300 import fab``) so that
the input generators in ``paper_2212_12758_gb300.workloads`` can be used
without the compiled library.
"""
