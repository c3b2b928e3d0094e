"""fab_sketch_apply_noalloc: the sketch entry point for callers that cannot allocate
device memory while they run (a host application that owns and caps the whole device
memory budget, or a latency-sensitive loop where cudaMalloc/cudaFree would synchronize
the device). It must give the same Theta V as fab_sketch_apply, whose scratch is
allocated per call, on consecutive calls that share the library's fixed scratch.

This file is collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def test_noalloc_sketch_matches_allocating_entry_point(fab):
    import torch

    cases = [(fab.SRHT, 70000, 400, 11), (fab.SPARSE_SIGN, 12345, 160, 4), (fab.SRHT, 5000, 64, 11)]
    for kind, n, s, seed in cases:  # consecutive calls share (and reuse) the fixed scratch
        V = torch.randn((3, n), dtype=torch.float64, device="cuda")
        V[1] *= 1e-6
        ref = fab.sketch_apply(V, s, sketch=kind, zeta=8, seed=seed)
        out = torch.full((3, s), float("nan"), dtype=torch.float64, device="cuda")
        rc = fab.lib.fab_sketch_apply_noalloc(kind, n, s, 8, seed, V.data_ptr(), n, 3, out.data_ptr(), None)
        assert rc == fab.FAB_OK
        o, r = out.cpu().numpy(), ref.cpu().numpy()
        for j in range(3):
            tol = 1e-13 * float(torch.linalg.norm(V[j]))
            assert np.max(np.abs(o[j] - r[j])) <= tol


def test_noalloc_rejects_sizes_beyond_its_scratch(fab):
    dummy = ctypes.c_void_p(256)  # never dereferenced: rejected before any device work
    n = 1 << 30  # 262,144 chunks x 400 rows > 1,048,576 partial sums
    assert fab.lib.fab_sketch_apply_noalloc(fab.SRHT, n, 400, 8, 1, dummy, n, 1, dummy, None) == fab.FAB_EINVAL
    assert fab.lib.fab_sketch_apply_noalloc(fab.SRHT, 100, 5000, 8, 1, dummy, 100, 1, dummy, None) == fab.FAB_EINVAL
