"""The C-ABI library builds, loads, and exports every entry point include/fab.h declares.

Runs without a GPU (no compute calls): loading libfab.so needs only the CUDA
runtime library, and argument validation happens before any device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def _declared():
    text = open(os.path.join(ROOT, "include", "fab.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fab_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_symbols(fab):
    assert _declared() == sorted(fab.SYMBOLS)


def test_library_exports_every_declared_symbol(fab):
    lib = ctypes.CDLL(fab._LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_and_defaults(fab):
    assert fab.lib.fab_strerror(0) == b"ok"
    assert fab.lib.fab_strerror(fab.FAB_EINVAL) == b"invalid argument"
    p = fab.Params()
    fab.lib.fab_params_default(ctypes.byref(p))
    assert p.precision == fab.FP64 and p.m > 0 and p.stream is None


def test_create_rejects_bad_csr_before_any_device_work(fab):
    h = ctypes.c_void_p()
    rowptr = np.array([0, 2, 1, 3], dtype=np.int64)  # decreasing
    colind = np.array([0, 1, 2], dtype=np.int32)
    vals = np.ones(3)
    rc = fab.lib.fab_create(ctypes.byref(h), 3, 3, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, 0)
    assert rc == fab.FAB_EINVAL and not h.value
    rowptr = np.array([0, 1, 2, 3], dtype=np.int64)
    colind = np.array([0, 5, 2], dtype=np.int32)  # out of range
    rc = fab.lib.fab_create(ctypes.byref(h), 3, 3, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, 0)
    assert rc == fab.FAB_EINVAL
    assert fab.lib.fab_create(None, 3, 3, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, 0) == fab.FAB_EINVAL
    fab.lib.fab_destroy(None)  # NULL-safe


def test_sketch_apply_rejects_bad_sizes(fab):
    out = ctypes.c_void_p(1)
    assert fab.lib.fab_sketch_apply(fab.SRHT, 10, 32, 8, 1, out, 10, 1, out, None) == fab.FAB_EINVAL  # s > n'
    assert fab.lib.fab_sketch_apply(fab.SPARSE_SIGN, 10, 4, 8, 1, out, 10, 1, out, None) == fab.FAB_EINVAL  # zeta > s
    assert fab.lib.fab_sketch_apply(fab.GAUSSIAN, 10, 4, 2, 1, out, 10, 257, out, None) == fab.FAB_EINVAL  # ncols
    assert fab.lib.fab_sketch_apply(7, 10, 4, 2, 1, out, 10, 1, out, None) == fab.FAB_EINVAL  # unknown sketch


def test_profile_class_selection_is_host_side(fab):
    """fab_profile_only takes the kernel class names of fab_profile_query (NULL or ""
    for every class) and rejects others; no device work is involved."""
    for name in fab.PROFILE_KINDS:
        assert fab.lib.fab_profile_only(name.encode()) == fab.FAB_OK
    assert fab.lib.fab_profile_only(None) == fab.FAB_OK
    assert fab.lib.fab_profile_only(b"") == fab.FAB_OK
    assert fab.lib.fab_profile_only(b"spmv") == fab.FAB_EINVAL
    assert fab.lib.fab_profile_query(b"spmv", None, None) == fab.FAB_EINVAL
    ms, cnt = ctypes.c_double(-1.0), ctypes.c_int64(-1)
    assert fab.lib.fab_profile_enable(0) == fab.FAB_OK  # resets the accumulators
    assert fab.lib.fab_profile_query(b"spmv_dots", ctypes.byref(ms), ctypes.byref(cnt)) == fab.FAB_OK
    assert ms.value == 0.0 and cnt.value == 0


def test_create_allocation_fault_returns_enomem(fab):
    """Host-side fault injection: FAB_FAULT=alloc:1 fails the first device allocation,
    which fab_create consults before any CUDA call. It returns FAB_ENOMEM, leaves *out
    NULL and releases its partial handle through the same cleanup as a real failure.
    (Without a GPU the allocation would fail with the same code anyway; there the check
    is that the failing path returns cleanly.) The setting is read once per process,
    so the check runs in a child process."""
    import subprocess
    import sys

    code = (
        "import ctypes, numpy as np\n"
        "from paper_2212_12758_gb300 import fab\n"
        "h = ctypes.c_void_p()\n"
        "rp = np.array([0, 1, 2], dtype=np.int64); ci = np.array([0, 1], dtype=np.int32); va = np.ones(2)\n"
        "rc = fab.lib.fab_create(ctypes.byref(h), 2, 2, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0)\n"
        "assert rc == fab.FAB_ENOMEM and not h.value, (rc, h.value)\n"
        "print('ok')\n")
    env = dict(os.environ, FAB_FAULT="alloc:1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
