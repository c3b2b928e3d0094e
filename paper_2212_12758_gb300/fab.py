"""ctypes binding of libfab (include/fab.h): argument marshalling only.

Every step of a solve runs in the CUDA kernels of libfab.so. Device arrays are
passed as torch CUDA tensors (data_ptr), host arrays as numpy arrays. There is
no fallback: importing this module raises if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libfab.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libfab.so is not built ({_LIB_PATH}); run __graft_entry__.build() first")
lib = ctypes.CDLL(_LIB_PATH)

FAB_OK, FAB_EINVAL, FAB_ENOMEM, FAB_ECUDA, FAB_ENUMERIC, FAB_ETIMEOUT, FAB_ENOTCONV = 0, -1, -2, -3, -4, -5, -6
EXP, SQRT, INVSQRT, SIGN = 0, 1, 2, 3
ARNOLDI, SKETCHED_LS, SKETCHED_FAST, NOPROJ, BG_LS, WHITEN = 0, 1, 2, 3, 4, 5
SPARSE_SIGN, SRHT, GAUSSIAN = 0, 1, 2
FP64, MIXED = 0, 1

# Every symbol the header declares (checked against include/fab.h by the tests).
SYMBOLS = ("fab_params_default", "fab_strerror", "fab_last_error", "fab_create", "fab_apply", "fab_destroy", "fab_last_state",
           "fab_last_basis", "fab_sketch_apply", "fab_sketch_apply_noalloc", "fab_profile_enable",
           "fab_profile_only", "fab_profile_query", "fab_server_create", "fab_server_submit", "fab_server_poll", "fab_server_stats_get",
           "fab_server_destroy", "fab_batch_create", "fab_batch_exec", "fab_batch_input", "fab_batch_output",
           "fab_batch_kernels", "fab_batch_destroy", "fab_batch_run", "fab_set_tiling", "fab_set_fusion", "fab_inject_wait_timeout", "fab_tune", "fab_fma_peak")
PROFILE_KINDS = ("spmv_dots", "update", "sketch_reduce", "gemv_t", "small", "combine", "fused_step")


class Params(ctypes.Structure):
    _fields_ = [("f", ctypes.c_int), ("t", ctypes.c_double), ("m", ctypes.c_int), ("k", ctypes.c_int),
                ("s", ctypes.c_int), ("zeta", ctypes.c_int), ("sketch", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("method", ctypes.c_int), ("precision", ctypes.c_int), ("lsqr_tol", ctypes.c_double),
                ("lsqr_maxit", ctypes.c_int), ("stream", ctypes.c_void_p), ("target_rel_err", ctypes.c_double),
                ("m_step", ctypes.c_int), ("m_max", ctypes.c_int), ("whiten_kappa", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("m_used", ctypes.c_int), ("lsqr_iters", ctypes.c_int), ("fh_iters", ctypes.c_int),
                ("launches", ctypes.c_int), ("h_last", ctypes.c_double), ("beta", ctypes.c_double),
                ("ms_basis", ctypes.c_double), ("ms_small", ctypes.c_double), ("ms_combine", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("err_est", ctypes.c_double), ("whiten_at", ctypes.c_int),
                ("kappa_est", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_vp, _i64, _i32, _u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
lib.fab_params_default.argtypes = [ctypes.POINTER(Params)]
lib.fab_params_default.restype = None
lib.fab_strerror.argtypes = [_i32]
lib.fab_strerror.restype = ctypes.c_char_p
lib.fab_last_error.argtypes = []
lib.fab_last_error.restype = ctypes.c_char_p
lib.fab_create.argtypes = [ctypes.POINTER(_vp), _i64, _i64, _vp, _vp, _vp, _i32]
lib.fab_create.restype = _i32
lib.fab_apply.argtypes = [_vp, ctypes.POINTER(Params), _vp, _vp, _i32, ctypes.POINTER(Stats)]
lib.fab_apply.restype = _i32
lib.fab_destroy.argtypes = [_vp]
lib.fab_destroy.restype = None
lib.fab_last_state.argtypes = [_vp, _vp, _vp, _vp, _vp]
lib.fab_last_state.restype = _i32
lib.fab_last_basis.argtypes = [_vp, _vp, _i32]
lib.fab_last_basis.restype = _i32
lib.fab_sketch_apply.argtypes = [_i32, _i64, _i32, _i32, _u64, _vp, _i64, _i32, _vp, _vp]
lib.fab_sketch_apply.restype = _i32
lib.fab_sketch_apply_noalloc.argtypes = [_i32, _i64, _i32, _i32, _u64, _vp, _i64, _i32, _vp, _vp]
lib.fab_sketch_apply_noalloc.restype = _i32
class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("bytes_in_use", ctypes.c_double), ("bytes_budget", ctypes.c_double)]


lib.fab_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_size_t, _i32]
lib.fab_server_create.restype = _i32
lib.fab_server_submit.argtypes = [_vp, _vp, ctypes.POINTER(Params), _vp, ctypes.POINTER(ctypes.c_uint64)]
lib.fab_server_submit.restype = _i32
lib.fab_server_poll.argtypes = [_vp, ctypes.c_uint64, _vp, ctypes.POINTER(Stats), ctypes.POINTER(ctypes.c_double), _i32]
lib.fab_server_poll.restype = _i32
lib.fab_server_stats_get.argtypes = [_vp, ctypes.POINTER(ServerStats)]
lib.fab_server_stats_get.restype = _i32
lib.fab_server_destroy.argtypes = [_vp]
lib.fab_server_destroy.restype = None
lib.fab_batch_create.argtypes = [ctypes.POINTER(_vp), _vp, _vp, _i32]
lib.fab_batch_create.restype = _i32
lib.fab_batch_exec.argtypes = [_vp, _vp, _vp, _vp, _vp]
lib.fab_batch_exec.restype = _i32
lib.fab_batch_input.argtypes = [_vp, _i32]
lib.fab_batch_input.restype = _vp
lib.fab_batch_output.argtypes = [_vp, _i32]
lib.fab_batch_output.restype = _vp
lib.fab_batch_kernels.argtypes = [_vp]
lib.fab_batch_kernels.restype = _i32
lib.fab_batch_destroy.argtypes = [_vp]
lib.fab_batch_destroy.restype = None
lib.fab_batch_run.argtypes = [_vp, _vp, _vp, _vp, _i32, _vp]
lib.fab_batch_run.restype = _i32
lib.fab_set_tiling.argtypes = [_vp, _i32, _i32, _i32]
lib.fab_set_tiling.restype = _i32
lib.fab_inject_wait_timeout.argtypes = [_vp, _i32, _i32]
lib.fab_inject_wait_timeout.restype = _i32
lib.fab_set_fusion.argtypes = [_vp, _i32]
lib.fab_set_fusion.restype = _i32
lib.fab_tune.argtypes = [_vp, _i32, _i32, _vp, _vp]
lib.fab_tune.restype = _i32
lib.fab_fma_peak.argtypes = [_i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp]
lib.fab_fma_peak.restype = _i32
lib.fab_profile_enable.argtypes = [_i32]
lib.fab_profile_enable.restype = _i32
lib.fab_profile_only.argtypes = [ctypes.c_char_p]
lib.fab_profile_only.restype = _i32
lib.fab_profile_query.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
lib.fab_profile_query.restype = _i32


class FabError(RuntimeError):
    def __init__(self, code: int, where: str):
        detail = lib.fab_last_error().decode() if code == FAB_ECUDA else ""
        super().__init__(f"{where}: {lib.fab_strerror(code).decode()} ({code}){' - ' + detail if detail else ''}")
        self.code = code


def _check(code: int, where: str):
    if code != FAB_OK:
        raise FabError(code, where)


def _addr(a):
    """Pointer of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    return a.data_ptr()


def _on_device(a) -> int:
    return 0 if isinstance(a, np.ndarray) else int(getattr(a, "is_cuda", False))


def params(f=EXP, t=1.0, m=30, k=2, s=None, zeta=8, sketch=SPARSE_SIGN, seed=1, method=SKETCHED_FAST,
           precision=FP64, lsqr_tol=1e-6, lsqr_maxit=0, stream=None, target_rel_err=0.0, m_step=0,
           m_max=0, whiten_kappa=0.0) -> Params:
    p = Params()
    lib.fab_params_default(ctypes.byref(p))
    p.f, p.t, p.m, p.k = int(f), float(t), int(m), int(k)
    p.s = int(s if s is not None else 4 * m)
    p.zeta, p.sketch, p.seed, p.method = int(zeta), int(sketch), int(seed), int(method)
    p.precision, p.lsqr_tol, p.lsqr_maxit = int(precision), float(lsqr_tol), int(lsqr_maxit)
    p.stream = stream
    p.target_rel_err, p.m_step, p.m_max = float(target_rel_err), int(m_step), int(m_max)
    p.whiten_kappa = float(whiten_kappa)
    return p


@dataclass
class LastState:
    H: np.ndarray
    SV: np.ndarray | None
    y: np.ndarray
    coeffs: np.ndarray


class Matrix:
    """A handle owning a device copy of A (fab_create / fab_destroy)."""

    def __init__(self, rowptr, colind, vals, n: int | None = None):
        n = int(n if n is not None else len(rowptr) - 1)
        on_dev = _on_device(rowptr)
        if not on_dev:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            colind = np.ascontiguousarray(colind, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        nnz = int(rowptr[-1])
        h = ctypes.c_void_p()
        _check(lib.fab_create(ctypes.byref(h), n, nnz, _addr(rowptr), _addr(colind), _addr(vals), on_dev),
               "fab_create")
        self._h = h
        self.n = n
        self.nnz = nnz
        self._last = None

    @classmethod
    def from_csr(cls, A):
        return cls(A.rowptr, A.colind, A.vals, A.n)

    def close(self):
        if getattr(self, "_h", None):
            lib.fab_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def apply(self, b, p: Params, x=None, stats: bool = False):
        """x ~ f(A) b. b and x are both numpy (host) or both torch CUDA tensors."""
        on_dev = _on_device(b)
        if x is None:
            if on_dev:
                import torch

                x = torch.empty_like(b)
            else:
                x = np.empty(self.n, dtype=np.float64)
        if not on_dev:
            b = np.ascontiguousarray(b, dtype=np.float64)
        st = Stats()
        _check(lib.fab_apply(self._h, ctypes.byref(p), _addr(b), _addr(x), on_dev, ctypes.byref(st)), "fab_apply")
        # growing m: the final dimension is not known here, so the state is not inspectable
        self._last = None if p.target_rel_err > 0 else (p.m, p.s, p.method in (SKETCHED_FAST, SKETCHED_LS, BG_LS,
                                                                                WHITEN))
        return (x, st) if stats else x

    def set_tiling(self, rows_max: int = 256, nnz_cap: int = 2048, staged: int = 1):
        """staged: 0 direct loads, 1 (or True) staged tiles with a row per lane group,
        2 staged tiles processed by nonzeros when they have many rows."""
        _check(lib.fab_set_tiling(self._h, int(rows_max), int(nnz_cap), int(staged)), "fab_set_tiling")

    def set_fusion(self, on: bool = True):
        """Allow or forbid (the default) the one-pass basis steps of the FP32 basis."""
        _check(lib.fab_set_fusion(self._h, 1 if on else 0), "fab_set_fusion")

    def tune(self, precision: int = FP64, k: int = 2, stream=None):
        """Autotune the SpMV tiling for this matrix; returns (rows_max, nnz_cap, staged)."""
        ch = (ctypes.c_int * 3)()
        _check(lib.fab_tune(self._h, int(precision), int(k), ctypes.cast(ch, _vp), stream), "fab_tune")
        return tuple(ch)

    def _last_sizes(self):
        if self._last is None:
            raise ValueError("no inspectable state: no fixed-m solve has run on this handle")
        return self._last

    def last_state(self) -> LastState:
        m, s, sk = self._last_sizes()
        H = np.zeros((m, m + 1))  # column-major (m+1) x m read as row-major transpose
        SV = np.zeros((m + 1, s)) if sk else None
        y = np.zeros(m)
        c = np.zeros(m)
        _check(lib.fab_last_state(self._h, _addr(H), _addr(SV), _addr(y), _addr(c)), "fab_last_state")
        return LastState(H=H.T.copy(), SV=None if SV is None else SV.T.copy(), y=y, coeffs=c)

    def last_basis(self) -> np.ndarray:
        m = self._last_sizes()[0]
        V = np.zeros((m + 1, self.n))
        _check(lib.fab_last_basis(self._h, _addr(V), 0), "fab_last_basis")
        return V.T.copy()


def sketch_apply(V, s: int, sketch: int = SPARSE_SIGN, zeta: int = 8, seed: int = 1, out=None, stream=None):
    """Theta V for a torch CUDA tensor V of shape (ncols, n) (each row one column
    vector, contiguous); returns a (ncols, s) tensor."""
    import torch

    if not (V.is_cuda and V.dtype == torch.float64 and V.is_contiguous()):
        raise ValueError("V must be a contiguous float64 CUDA tensor")
    ncols, n = V.shape
    if out is None:
        out = torch.empty((ncols, s), dtype=torch.float64, device=V.device)
    _check(lib.fab_sketch_apply(int(sketch), int(n), int(s), int(zeta), int(seed), V.data_ptr(), int(n), int(ncols),
                                out.data_ptr(), stream), "fab_sketch_apply")
    return out


def fma_peak(precision: int = FP64, stream=None):
    """Measured FMA throughput (GFLOP/s, ms of the timed launch) of the current GPU:
    FP64 for FP64, FP32 for MIXED (fab_fma_peak)."""
    g, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.fab_fma_peak(int(precision), ctypes.byref(g), ctypes.byref(ms), stream), "fab_fma_peak")
    return g.value, ms.value


def profile_enable(on: bool = True):
    _check(lib.fab_profile_enable(1 if on else 0), "fab_profile_enable")


def profile_only(name=None):
    """Record only kernel class `name` (None: every class) while profiling is on."""
    _check(lib.fab_profile_only(name.encode() if name else None), "fab_profile_only")


def profile_query():
    """{kernel class: (total device ms, launches)} accumulated since profile_enable."""
    out = {}
    for name in PROFILE_KINDS:
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(lib.fab_profile_query(name.encode(), ctypes.byref(ms), ctypes.byref(cnt)), "fab_profile_query")
        out[name] = (ms.value, cnt.value)
    return out


def sketch_apply_noalloc(V, s: int, sketch: int = SPARSE_SIGN, zeta: int = 8, seed: int = 1, out=None, stream=None):
    """Same result as sketch_apply, computed with the library's fixed scratch
    (fab_sketch_apply_noalloc): no device allocation inside the call. `out` must
    be given by callers that cannot allocate either."""
    import torch

    if not (V.is_cuda and V.dtype == torch.float64 and V.is_contiguous()):
        raise ValueError("V must be a contiguous float64 CUDA tensor")
    ncols, n = V.shape
    if out is None:
        out = torch.empty((ncols, s), dtype=torch.float64, device=V.device)
    _check(lib.fab_sketch_apply_noalloc(int(sketch), int(n), int(s), int(zeta), int(seed), V.data_ptr(), int(n),
                                        int(ncols), out.data_ptr(), stream), "fab_sketch_apply_noalloc")
    return out


class Server:
    """Continuous-batching server (fab_server_*): submit f(A)b requests on any
    Matrix handles; each result is polled by its ticket."""

    def __init__(self, hbm_budget_bytes: int = 0, slots: int = 4):
        h = ctypes.c_void_p()
        _check(lib.fab_server_create(ctypes.byref(h), int(hbm_budget_bytes), int(slots)), "fab_server_create")
        self._s = h
        self._mats = {}

    def submit(self, M: "Matrix", b: np.ndarray, p: Params) -> int:
        b = np.ascontiguousarray(b, dtype=np.float64)
        t = ctypes.c_uint64()
        _check(lib.fab_server_submit(self._s, M._h, ctypes.byref(p), b.ctypes.data, ctypes.byref(t)), "fab_server_submit")
        self._mats[t.value] = M.n
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 60000):
        """(x, stats, latency_ms), or None if not done within timeout_ms."""
        n = self._mats[ticket]
        x = np.empty(n)
        st = Stats()
        lat = ctypes.c_double()
        rc = lib.fab_server_poll(self._s, ctypes.c_uint64(ticket), x.ctypes.data, ctypes.byref(st), ctypes.byref(lat),
                                 int(timeout_ms))
        if rc == FAB_ETIMEOUT:
            return None
        del self._mats[ticket]
        _check(rc, "fab_server_poll")
        return x, st, lat.value

    def stats(self) -> ServerStats:
        out = ServerStats()
        _check(lib.fab_server_stats_get(self._s, ctypes.byref(out)), "fab_server_stats_get")
        return out

    def close(self):
        if getattr(self, "_s", None):
            lib.fab_server_destroy(self._s)
            self._s = None

    def __del__(self):
        self.close()


class Batch:
    """Many solves of uneven size as one CUDA graph (fab_batch_*). The Matrix
    handles must outlive the batch."""

    def __init__(self, mats, ps):
        self._mats = list(mats)
        self.count = len(self._mats)
        hs = (ctypes.c_void_p * self.count)(*[M._h.value for M in self._mats])
        self._ps = (Params * self.count)(*ps)
        h = ctypes.c_void_p()
        _check(lib.fab_batch_create(ctypes.byref(h), ctypes.cast(hs, _vp), ctypes.cast(self._ps, _vp), self.count),
               "fab_batch_create")
        self._b = h
        self.kernels = lib.fab_batch_kernels(self._b)

    def run(self, bs=None, xs=None, stream=None, stats: bool = False):
        """One run. bs: list of numpy (host) or torch CUDA arrays, or None when
        the inputs were written to input(i). Returns the list of results as
        numpy arrays (xs None), or fills xs."""
        keep = []
        bp = None
        if bs is not None:
            bs = [np.ascontiguousarray(b, dtype=np.float64) if isinstance(b, np.ndarray) else b for b in bs]
            keep.append(bs)
            bp = (ctypes.c_void_p * self.count)(*[_addr(b) for b in bs])
        out = xs
        if xs is None and bs is not None:
            out = [np.empty(M.n) for M in self._mats]
        xp = None if out is None else (ctypes.c_void_p * self.count)(*[_addr(x) for x in out])
        sts = (Stats * self.count)()
        _check(lib.fab_batch_exec(self._b, None if bp is None else ctypes.cast(bp, _vp),
                                  None if xp is None else ctypes.cast(xp, _vp), ctypes.cast(sts, _vp), stream),
               "fab_batch_exec")
        return (out, list(sts)) if stats else out

    def input(self, i: int) -> int:
        return lib.fab_batch_input(self._b, int(i))

    def output(self, i: int) -> int:
        return lib.fab_batch_output(self._b, int(i))

    def close(self):
        if getattr(self, "_b", None):
            lib.fab_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        self.close()
