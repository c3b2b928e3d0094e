"""fab_sketch_apply_noalloc: the sketch entry point for callers that cannot allocate
device memory while they run (a host application that owns and caps the whole device
memory budget, or a latency-sensitive loop where cudaMalloc/cudaFree would synchronize
the device). It must give the same Theta V as fab_sketch_apply, whose scratch is
allocated per call, on consecutive calls that share the library's fixed scratch, and
it must not change the device's free memory.

This file is collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the fixed scratch holds ceil(n / 4096) * s <= 2^20 chunk partial sums
LIMIT = 1 << 20


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def _noalloc(fab, kind, V, s, seed, out):
    n = V.shape[1]
    return fab.lib.fab_sketch_apply_noalloc(kind, n, s, 8, seed, V.data_ptr(), n, V.shape[0], out.data_ptr(), None)


def _check_equal(V, o, r):
    import torch

    for j in range(V.shape[0]):
        tol = 1e-13 * float(torch.linalg.norm(V[j]))
        assert np.max(np.abs(o[j] - r[j])) <= tol


def test_noalloc_sketch_matches_allocating_entry_point(fab):
    import torch

    cases = [(fab.SRHT, 70000, 400, 11), (fab.SPARSE_SIGN, 12345, 160, 4), (fab.SRHT, 5000, 64, 11)]
    for kind, n, s, seed in cases:  # consecutive calls share (and reuse) the fixed scratch
        V = torch.randn((3, n), dtype=torch.float64, device="cuda")
        V[1] *= 1e-6
        ref = fab.sketch_apply(V, s, sketch=kind, zeta=8, seed=seed)
        out = torch.full((3, s), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(fab, kind, V, s, seed, out) == fab.FAB_OK
        _check_equal(V, out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_largest_accepted_size_allocates_nothing(fab):
    """n = 2^20 rows and s = 4096 fill the fixed scratch exactly (256 chunks x 4096
    partial sums). Repeated calls at that size leave the device's free memory as it
    was, and give fab_sketch_apply's result."""
    import torch

    n, s = 1 << 20, 4096
    assert ((n + 4095) // 4096) * s == LIMIT
    V = torch.randn((2, n), dtype=torch.float64, device="cuda")
    out = torch.full((2, s), float("nan"), dtype=torch.float64, device="cuda")
    ref = fab.sketch_apply(V, s, sketch=fab.SRHT, seed=5).cpu().numpy()
    torch.cuda.synchronize()
    assert _noalloc(fab, fab.SRHT, V, s, 5, out) == fab.FAB_OK  # first call: scratch address set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for seed in (5, 6, 5):
        assert _noalloc(fab, fab.SRHT, V, s, seed, out) == fab.FAB_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    _check_equal(V, out.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(fab):
    dummy = ctypes.c_void_p(256)  # never dereferenced: rejected before any device work
    n = 1 << 30  # 262,144 chunks x 400 rows > 1,048,576 partial sums
    assert fab.lib.fab_sketch_apply_noalloc(fab.SRHT, n, 400, 8, 1, dummy, n, 1, dummy, None) == fab.FAB_EINVAL
    assert fab.lib.fab_sketch_apply_noalloc(fab.SRHT, 100, 5000, 8, 1, dummy, 100, 1, dummy, None) == fab.FAB_EINVAL
    n = (1 << 20) + 1  # 257 chunks x 4096 rows: one chunk past the limit
    assert fab.lib.fab_sketch_apply_noalloc(fab.SRHT, n, 4096, 8, 1, dummy, n, 1, dummy, None) == fab.FAB_EINVAL
    assert fab.lib.fab_sketch_apply_noalloc(fab.SPARSE_SIGN, n, 4096, 8, 1, dummy, n, 1, dummy, None) == fab.FAB_EINVAL
