"""Benchmark: randomized Krylov f(A)b solves on one GB300 (or N replicas).

Workload (one "step" = one whole solve of the hot path): 3D convection-diffusion,
7-point upwind finite differences on a 200^3 grid (n = 8,000,000, nnz = 55,760,000,
CSR FP64), x = exp(-1e-3 A) b with b ~ N(0,1) (seed 0, normalized), Krylov dimension
m = 100, truncation window k = 4, SRHT sketch with s = 400 rows, method sketched_fast
(eq. sFOM, sketch-and-solve form), all arithmetic FP64. sketched_ls (Alg. 4) and full
Arnoldi on the same inputs are timed beside it. Inputs are synthetic.

Timed region: K solves on the device with A, b and x resident in HBM (CUDA events on
the solving stream, synchronize + barrier on both sides, max over ranks). The inputs
(A 0.7 GB, basis 6.5 GB per solve) are far larger than L2. e2e repeats the measurement
through the C ABI with pinned host buffers (b copied in, x copied out inside the call).

N > 1 (torchrun): every rank runs its own replica of the workload (no collective);
value = all ranks' solves / the slowest rank's time ("scaling": "weak").

--impl reference times the plain FP64 CPU oracle (oracle/) on this host's cores on a
bounded sample of the same workload and reports the same metric.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "f(A)b solves/s + HBM GB/s at rel err ≤1e-6, sketched vs Arnoldi; p99 latency"
N_GRID, M, K_WIN, S_ROWS, T_EXP, SEED_B, SEED_SK = 200, 100, 4, 400, -1e-3, 0, 1
WORKLOAD = ("3D convection-diffusion 200^3 upwind FD (n=8,000,000, nnz=55,760,000), x=exp(-1e-3 A) b, "
            "m=100, k=4, SRHT s=400, sketched_fast, FP64")


def workload_name(N: int, n: int, nnz: int) -> str:
    return (f"3D convection-diffusion {N}^3 upwind FD (n={n:,}, nnz={nnz:,}), x=exp(-1e-3 A) b, "
            f"m={M}, k={K_WIN}, SRHT s={S_ROWS}, sketched_fast, FP64")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# FP64 FMA rate used only when the live measurement (fab_fma_peak) fails: the
# nominal GB300 FP64 rate.
FP64_PEAK_GFLOPS_NOMINAL = 1250.0
# Basis steps in each sample of the CPU oracle (the GPU line's cpu_baseline and every
# step of --impl reference use the same sample).
CPU_SAMPLE_STEPS = 16
# DRAM bytes (read + write) of one k_spmv_dots launch measured by ncu on the
# 128^3 case of this workload (262.4 MB for n = 2,097,152, window k = 4); traffic
# grows with n and nnz, so it is scaled by n to the bench size. Only valid for the
# kernel version it was taken on, and only for the 3D convection-diffusion operator.
SPMV_DRAM_BYTES_PER_ROW = 262_368_512 / 2_097_152


def oracle_golden_error(x_dev, coeffs):
    """The solve against the FP64 oracle's solve of the same workload, stored by
    tests/golden/make_c2_reference.py: relative 2-norm error on the 1024 stored rows of
    x and on the coefficient vector c (x = ||b|| V_m c)."""
    path = os.path.join(ROOT, "tests", "golden", "c2_sketched_fast.txt")
    if not os.path.exists(path):
        return None
    rows, vals, gc = [], [], None
    for line in open(path):
        if line.startswith("x "):
            _, i, v = line.split()
            rows.append(int(i))
            vals.append(float(v))
        elif line.startswith("coeffs "):
            gc = np.array([float(v) for v in line.split()[1:]])
    import torch

    xs = x_dev[torch.tensor(rows, device=x_dev.device)].cpu().numpy()
    vals = np.array(vals)
    return {"x_sampled_rows": float(np.linalg.norm(xs - vals) / np.linalg.norm(vals)),
            "coeffs": float(np.linalg.norm(coeffs - gc) / np.linalg.norm(gc)) if gc is not None else None,
            "reference": "FP64 oracle sketched_fast on the same inputs (tests/golden/c2_sketched_fast.txt: "
                         f"{len(rows)} sampled rows of x and the m coefficients)"}


def oracle_golden_c3(fname: str, x_dev, coeffs):
    """The graph solve against the FP64 oracle's f_m at the same m and sketch, stored by
    tests/golden/make_c3_reference.py (1024 sampled rows of x, the coefficients, and the
    rounding model's RMS at this size)."""
    path = os.path.join(ROOT, "tests", "golden", "c3_gauss.txt")
    if not os.path.exists(path):
        return None
    rows, vals, gc, rms = [], [], None, None
    for line in open(path):
        p = line.split()
        if not p or p[0] != fname:
            continue
        if p[1] == "x":
            rows.append(int(p[2]))
            vals.append(float(p[3]))
        elif p[1] == "coeffs":
            gc = np.array([float(v) for v in p[2:]])
        elif p[1] == "model_rms":
            rms = float(p[2])
    import torch

    xs = x_dev[torch.tensor(rows, device=x_dev.device)].cpu().numpy()
    vals = np.array(vals)
    return {"x_sampled_rows": float(np.linalg.norm(xs - vals) / np.linalg.norm(vals)),
            "coeffs": float(np.linalg.norm(coeffs - gc) / np.linalg.norm(gc)) if gc is not None else None,
            "rounding_model_rms": rms,
            "reference": "FP64 oracle sketched_fast, same m, k and Gaussian sketch (tests/golden/c3_gauss.txt)"}


def bench_config(grid: int, n: int, nnz: int, world: int) -> dict:
    """The workload description both arms print (the same dict in both lines)."""
    return {"workload": workload_name(grid, n, nnz), "n": n, "nnz": nnz, "m": M, "k": K_WIN, "s": S_ROWS,
            "sketch": "srht", "method": "sketched_fast", "f": "exp(tA), t=-1e-3",
            "l2": "inputs larger than L2 (A 0.7 GB, basis 6.5 GB per solve)",
            "parallelism": f"replicas x{world}"}


def algorithmic_cost(n: int, nnz: int, m: int, k: int, s: int):
    """Algorithmic bytes and FP64 flops per launch of the basis kernels (FP64 path).

    spmv_dots (step c, window kw <= k): A values + column indices (12 nnz), row
      pointers (4 (n+1)), the gathered column v_{c-1} (8 n, counted once), the other
      kw-1 window columns (8 n each), the write of w (8 n). Flops: 2 nnz (SpMV)
      + 2 n kw (window dots); ||A v|| for the breakdown test comes from the
      coefficients, not the rows.
    update (step c): read w and kw window columns, write the new column: 8 n (kw + 2);
      flops 2 n kw + 2 n; the sketch partials add 8 s per 4096-row chunk.
    """
    kw = k
    sp_bytes = 12 * nnz + 4 * (n + 1) + 8 * n * kw + 8 * n
    sp_flops = 2 * nnz + 2 * n * kw
    nch = (n + 4095) // 4096
    up_bytes = 8 * n * (kw + 2) + 8 * s * nch
    up_flops = 2 * n * kw + 2 * n
    return {"spmv_dots": (sp_bytes, sp_flops), "update": (up_bytes, up_flops)}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"fab_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def fp32_step_bytes(n: int, nnz: int, kw: int, s: int) -> int:
    """Algorithmic bytes of one basis step of the FP32 path (SpMV + dots, update +
    sketch partials): 8 nnz + 4 (n+1) + 4 n kw + 4 n, then 4 n (kw + 2) + 8 s per chunk."""
    return 8 * nnz + 4 * (n + 1) + 4 * n * kw + 4 * n + 4 * n * (kw + 2) + 8 * s * ((n + 4095) // 4096)


def bench_mixed_same(fab, torch, Mx, bd, ref_x, stream, n: int, nnz: int, P, reps: int = 5):
    """The bench workload with FP32 A and basis (FP64 small stage): solves/s, the
    basis kernels against the HBM roofline (FP32 algorithmic bytes), error against
    the FP64 Arnoldi reference solution."""
    p = P(fab.SKETCHED_FAST)
    p.precision = fab.MIXED
    x = torch.empty_like(bd)
    Mx.apply(bd, p, x=x)
    torch.cuda.synchronize()
    fab.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        Mx.apply(bd, p, x=x)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = fab.profile_query()
    fab.profile_enable(False)
    ms = e0.elapsed_time(e1) / reps
    peak = float(_peaks().get("hbm_gbs", 6800.0))
    kw = K_WIN
    nch = (n + 4095) // 4096
    sp_bytes = 8 * nnz + 4 * (n + 1) + 4 * n * kw + 4 * n
    up_bytes = 4 * n * (kw + 2) + 8 * S_ROWS * nch
    # one-pass step (steady state): A, row pointers, the previous SpMV output and the k
    # update-window columns read once, the updated column and the new SpMV output
    # written, the sketch partials (at most one s-vector per block, counted per chunk)
    fu_bytes = 8 * nnz + 4 * (n + 1) + 4 * n * (kw + 1) + 8 * n + 8 * S_ROWS * nch
    out = {"solves_per_s": 1000.0 / ms, "ms_per_solve": ms,
           "rel_err_vs_fp64_arnoldi_m150": float(torch.linalg.norm(x - ref_x) / torch.linalg.norm(ref_x))
           if ref_x is not None else None}
    for name, byts in (("spmv_dots", sp_bytes), ("update", up_bytes), ("fused_step", fu_bytes)):
        t_ms, cnt = prof[name]
        if cnt == 0:
            continue
        sec = t_ms / cnt / 1000.0
        out[name] = {"ms_per_launch": sec * 1000.0, "launches_per_solve": cnt / reps,
                     "algorithmic_bytes_per_launch": byts,
                     "hbm_gbs": byts / sec / 1e9, "hbm_frac_of_measured": byts / sec / 1e9 / peak}
    basis_s = sum(prof[k_][0] for k_ in ("spmv_dots", "update", "sketch_reduce", "fused_step")) / 1000.0 / reps
    out["basis_pass_hbm_frac_of_measured"] = M * (sp_bytes + up_bytes) / basis_s / 1e9 / peak
    # the same pass against the single-pass floor of one basis step with its fused sign
    # sketch, 8 nnz + 4 (n+1) + 4 n (k+1) bytes (A, row pointers, the k window columns,
    # the new column written once)
    b8d = sum(8 * nnz + 4 * (n + 1) + 4 * n * (min(c, kw) + 1) for c in range(1, M + 1))
    out["basis_pass_frac_vs_8d"] = b8d / basis_s / 1e9 / peak
    out["basis_pass_bytes_8d"] = b8d
    out["basis_pass_ms"] = basis_s * 1000.0
    return out


def bench_bg_laplacian(fab, torch, W, N: int = 80, ms=(40, 80, 160), reps: int = 3):
    """Alg. 3 (Alg. 1 basis + LSQR) against Arnoldi on the paper's §5.1.4 setting: 3D
    Laplacian N = 80 (n = 512,000), f = A^{-1/2}, SRHT with s = floor(1.05 m), FP64.
    Error of both against Arnoldi with m = 320 (FP64, this library)."""
    A = W.laplacian3d(N)
    Mx = fab.Matrix.from_csr(A)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    b = torch.from_numpy(W.random_vector(A.n, 0)).cuda()
    xr = torch.empty_like(b)
    Mx.apply(b, fab.params(f=fab.INVSQRT, m=320, method=fab.ARNOLDI, stream=sp), x=xr)
    out = {"workload": f"3D Laplacian {N}^3 (n={A.n:,}), x = A^(-1/2) b, SRHT s = floor(1.05 m), FP64; reference "
                       "Arnoldi m=320"}

    def timed(p):
        x = torch.empty_like(b)
        _, st = Mx.apply(b, p, x=x, stats=True)  # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            Mx.apply(b, p, x=x)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr)), st

    for m in ms:
        s = int(1.05 * m)
        t_bg, e_bg, st = timed(fab.params(f=fab.INVSQRT, m=m, s=s, sketch=fab.SRHT, seed=1, method=fab.BG_LS,
                                          lsqr_tol=1e-6, stream=sp))
        t_ar, e_ar, _ = timed(fab.params(f=fab.INVSQRT, m=m, method=fab.ARNOLDI, stream=sp))
        out[f"m={m}"] = {"bg_ls_ms": t_bg, "arnoldi_ms": t_ar, "bg_ls_rel_err": e_bg, "arnoldi_rel_err": e_ar,
                         "lsqr_iters": st.lsqr_iters, "speedup_vs_arnoldi": t_ar / t_bg}
    return out


def bench_skew_convdiff(fab, torch, W, N: int = 352, t: float = -1e-6, ms=(30, 60, 90), reps: int = 3):
    """The paper's first experiment re-created (§5.1.1): skew-form convection-diffusion
    with discontinuous diffusion, Pe = 200, N x N grid, b = sin(pi x) sin(pi y)
    normalised, x = exp(t A) b (t ||A|| ~ 370; t is not given in the paper). Every method
    at each m (SRHT s = 4m, k = 2, LSQR tol 1e-6), FP64; error against Arnoldi m = 200."""
    A = W.convdiff_skew(N)
    Mx = fab.Matrix.from_csr(A)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    b = torch.from_numpy(W.sine_vector(N)).cuda()
    xr = torch.empty_like(b)
    Mx.apply(b, fab.params(f=fab.EXP, t=t, m=200, method=fab.ARNOLDI, stream=sp), x=xr)
    out = {"workload": f"skew-form convection-diffusion {N}x{N} (n={A.n:,}), Pe=200, D=1000 on [0.25,0.75]^2, "
                       f"exp({t:g} A) b, b = sin(pi x) sin(pi y); reference Arnoldi m=200"}
    names = (("noproj", fab.NOPROJ), ("sketched_fast", fab.SKETCHED_FAST), ("sketched_ls", fab.SKETCHED_LS),
             ("bg_ls", fab.BG_LS), ("arnoldi", fab.ARNOLDI))
    for m in ms:
        row = {}
        for name, meth in names:
            p = fab.params(f=fab.EXP, t=t, m=m, k=2, s=4 * m, sketch=fab.SRHT, seed=1, method=meth, lsqr_tol=1e-6,
                           stream=sp)
            x = torch.empty_like(b)
            Mx.apply(b, p, x=x)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                Mx.apply(b, p, x=x)
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = {"ms": e0.elapsed_time(e1) / reps,
                         "rel_err": float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr))}
        row["fastest"] = min(row, key=lambda k_: row[k_]["ms"])
        out[f"m={m}"] = row
    return out


def bench_whiten_graph(fab, torch, W, ns=(6301, 1_000_000), ms=(60, 100, 140, 180), reps: int = 3):
    """The paper's whitening experiment re-created (§5.1.3): x = A^{1/2} b for the
    Laplacian of a directed Chung-Lu graph (nonsymmetric, eigenvalues with positive
    real part; n = 6301 as the paper's graph, and n = 1M), b random unit, k = 2,
    SRHT s = 4m, LSQR tol 1e-6, FP64. Alg. 2's sketch passes kappa_1 = 1000 near
    column 60 here: every method at each m, error against Arnoldi m = 240."""
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    out = {"workload": "directed Chung-Lu graph Laplacian (seed 2), x = A^(1/2) b, k=2, SRHT s=4m, FP64; "
                       "reference Arnoldi m=240"}
    names = (("whiten", fab.WHITEN), ("noproj", fab.NOPROJ), ("sketched_fast", fab.SKETCHED_FAST),
             ("bg_ls", fab.BG_LS), ("arnoldi", fab.ARNOLDI))
    for n in ns:
        A = W.chung_lu_laplacian(n, seed=2)
        Mx = fab.Matrix.from_csr(A)
        b = torch.from_numpy(W.random_vector(n, 7)).cuda()
        xr = torch.empty_like(b)
        Mx.apply(b, fab.params(f=fab.SQRT, m=240, method=fab.ARNOLDI, stream=sp), x=xr)
        res = {"nnz": int(A.nnz)}
        for m in ms:
            row = {}
            for name, meth in names:
                p = fab.params(f=fab.SQRT, m=m, k=2, s=4 * m, sketch=fab.SRHT, seed=1, method=meth, lsqr_tol=1e-6,
                               stream=sp)
                x = torch.empty_like(b)
                st = fab.Stats()
                rc = fab.lib.fab_apply(Mx._h, ctypes.byref(p), b.data_ptr(), x.data_ptr(), 1, ctypes.byref(st))
                if rc != fab.FAB_OK:  # e.g. no real principal square root of a garbled projection
                    row[name] = {"error": rc, "m_used": st.m_used, "kappa_est": st.kappa_est,
                                 "fh_iters": st.fh_iters}
                    continue
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    Mx.apply(b, p, x=x)
                e1.record(stream)
                torch.cuda.synchronize()
                row[name] = {"ms": e0.elapsed_time(e1) / reps,
                             "rel_err": float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr))}
                if meth in (fab.SKETCHED_FAST, fab.SKETCHED_LS):
                    row[name]["kappa_est"] = st.kappa_est
                if meth == fab.WHITEN:
                    row[name]["whiten_at"] = st.whiten_at
                    row[name]["lsqr_iters"] = st.lsqr_iters
            res[f"m={m}"] = row
        out[f"n={n}"] = res
    return out


def bench_batch(fab, torch, W, steps: int = 3, count: int = 256):
    """256 uneven 2D convection-diffusion solves (n log-uniform on [1e4, 1e6], t on
    [1e-4, 1e-2], m on {20..80}, k = 2, sparse sign s = 4m, zeta = 8, batch seed 3)
    as one CUDA graph, FP32 basis / FP64 small stage; inputs resident on the device."""
    specs = W.batch_specs(count, seed=3)
    A = [W.convdiff(2, it.N) for it in specs]
    mats = [fab.Matrix.from_csr(a) for a in A]
    k = 2

    def ps(prec):
        return [fab.params(f=fab.EXP, t=-it.t, m=it.m, k=k, s=4 * it.m, zeta=8, sketch=fab.SPARSE_SIGN, seed=1 + i,
                           method=fab.SKETCHED_FAST, precision=prec) for i, it in enumerate(specs)]

    bs = [torch.from_numpy(W.random_vector(a.n, 100 + i)).cuda() for i, a in enumerate(A)]
    t0 = time.perf_counter()
    choices = {}
    for Mx in mats:  # the autotuner picks each matrix's SpMV tiling for the FP32 kernel, window k
        ch = Mx.tune(fab.MIXED, k=k)
        choices[str(ch)] = choices.get(str(ch), 0) + 1
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    bt = fab.Batch(mats, ps(fab.MIXED))
    create_s = time.perf_counter() - t0
    xs = [torch.empty_like(b) for b in bs]
    bt.run(bs, xs)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        bt.run(None, None, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        bt.run(None, None, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    byts = 0
    for a, it in zip(A, specs):
        byts += sum(fp32_step_bytes(a.n, a.nnz, min(c, k), 4 * it.m) for c in range(1, it.m + 1))
        byts += 4 * a.n * it.m + 8 * a.n  # combine
    bt.run(None, xs)
    bt64 = fab.Batch(mats, ps(fab.FP64))
    x64 = [torch.empty_like(b) for b in bs]
    bt64.run(bs, x64)
    err = max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(xs, x64))
    kernels = bt.kernels
    bt.close()
    bt64.close()
    vs_exact = batch_vs_exact(fab, torch, mats, specs, bs, xs, x64)
    peak = float(_peaks().get("hbm_gbs", 6800.0))
    return {"workload": f"{count} uneven 2D convection-diffusion solves (n 1e4..1e6 log-uniform, m 20..80, t 1e-4..1e-2), "
                        "k=2, sparse sign s=4m, sketched_fast, FP32 basis / FP64 small stage, one CUDA graph",
            "solves_per_s": count / (ms / 1000.0), "ms_per_batch": ms, "graph_kernels": kernels, "count": count,
            "sum_n": int(sum(a.n for a in A)), "algorithmic_gb": byts / 1e9,
            "hbm_gbs_algorithmic": byts / (ms / 1000.0) / 1e9,
            "hbm_frac_of_measured": byts / (ms / 1000.0) / 1e9 / peak,
            "note": "solves with n below ~3e5 keep their basis in L2, so algorithmic GB/s is not all HBM traffic",
            "max_rel_err_vs_fp64_same_m": err, "vs_exact": vs_exact, "create_s": create_s, "autotune_s": tune_s,
            "tilings_chosen": choices}


def batch_vs_exact(fab, torch, mats, specs, bs, x32, x64, bar: float = 1e-6):
    """Each batched solve against f(A)b. The FP64 Arnoldi approximation at 2m stands in
    for f(A)b where it has converged (its change from m' = 3m/2 to 2m at most 1e-10);
    the 1e-6 bar applies to the solves whose FP64 f_m reaches it (the Krylov error
    allows it), and the FP32-basis solve is checked on exactly those."""
    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    trusted = reach = ok = 0
    reach7 = ok7 = 0
    worst32 = worst64 = 0.0
    e64_all = []
    for i, (Mx, it) in enumerate(zip(mats, specs)):
        def arnoldi(mm):
            return Mx.apply(bs[i], fab.params(f=fab.EXP, t=-it.t, m=mm, method=fab.ARNOLDI))

        r2 = arnoldi(2 * it.m)
        if rel(arnoldi(3 * it.m // 2), r2) > 1e-10:
            continue
        trusted += 1
        e64, e32 = rel(x64[i], r2), rel(x32[i], r2)
        e64_all.append(e64)
        if e64 <= bar:
            reach += 1
            ok += e32 <= bar
            worst32 = max(worst32, e32)
            worst64 = max(worst64, e64)
        if e64 <= 0.1 * bar:  # the Krylov error leaves room for the FP32 rounding
            reach7 += 1
            ok7 += e32 <= bar
    return {"reference": "FP64 Arnoldi at 2m (this library), used where its change from 3m/2 to 2m is <= 1e-10",
            "solves_with_converged_reference": trusted, "fp64_f_m_within_1e-6": reach,
            "fp32_basis_within_1e-6_of_those": ok, "max_fp32_err_of_those": worst32,
            "max_fp64_err_of_those": worst64, "fp64_f_m_within_1e-7": reach7,
            "fp32_basis_within_1e-6_of_those_1e-7": ok7,
            "median_fp64_err_all": float(np.median(e64_all)) if e64_all else None}


def bench_mixed_graph(fab, torch, W, reps: int = 2, n: int = 4_000_000, references: bool = True):
    """Shifted Chung-Lu Laplacian (n = 4M, exponent 2.5, mean degree 10, L + 0.1 I), f = A^{-1/2}
    and A^{1/2}, m = 150, k = 2, Gaussian sketch s = 600 (BF16 on the tensor cores, FP32
    accumulation), FP32 basis, FP64 QR and f(H). Error against the library's FP64 Arnoldi
    f_m at the same m and at m = 300."""
    A = W.chung_lu_laplacian(n, seed=2)
    Mx = fab.Matrix.from_csr(A)
    b = torch.from_numpy(W.random_vector(A.n, 0)).cuda()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    m, s = 150, 600
    out = {"workload": f"Chung-Lu Laplacian n={A.n:,} nnz={A.nnz:,} (+0.1 I), m=150, k=2, Gaussian s=600 BF16 "
                       "tensor cores, FP32 basis, FP64 small stage, sketched_fast"}
    peaks = _peaks()
    for name, f in (("invsqrt", fab.INVSQRT), ("sqrt", fab.SQRT)):
        p = fab.params(f=f, m=m, k=2, s=s, sketch=fab.GAUSSIAN, seed=1, method=fab.SKETCHED_FAST,
                       precision=fab.MIXED, stream=sp)
        x = torch.empty_like(b)
        Mx.apply(b, p, x=x)  # warm (draws G once per handle)
        torch.cuda.synchronize()
        fab.profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            Mx.apply(b, p, x=x)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = fab.profile_query()
        fab.profile_enable(False)
        ms = e0.elapsed_time(e1) / reps
        g_ms = prof["sketch_reduce"][0] / max(prof["sketch_reduce"][1], 1)
        coeffs = Mx.last_state().coeffs  # before the reference solves replace the state
        flops = 2.0 * s * A.n * (m + 1)
        gbytes = 2.0 * s * A.n + 4.0 * A.n * (m + 1)  # G once, both BF16 terms of the basis once
        ref = {150: None, 300: None}
        for mr in ((150, 300) if references else ()):
            xr = torch.empty_like(b)
            Mx.apply(b, fab.params(f=f, m=mr, k=2, method=fab.ARNOLDI, stream=sp), x=xr)
            ref[mr] = float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr))
        fm = oracle_golden_c3(name, x, coeffs) if n == 4_000_000 else None
        out[name] = {"solves_per_s": 1000.0 / ms, "ms_per_solve": ms, "rel_err_vs_oracle_fm": fm,
                     "rel_err_vs_fp64_arnoldi_m150": ref[150], "rel_err_vs_fp64_arnoldi_m300": ref[300],
                     "gauss_sketch_ms": g_ms, "gauss_tflops": flops / (g_ms / 1000.0) / 1e12,
                     "gauss_tensor_frac_of_measured_bf16": flops / (g_ms / 1000.0) / 1e12
                     / float(peaks.get("bf16_tflops", 1900.0)),
                     "gauss_hbm_gbs_algorithmic": gbytes / (g_ms / 1000.0) / 1e9,
                     "gauss_hbm_frac_of_measured": gbytes / (g_ms / 1000.0) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
                     "kernels_ms": {k_: v[0] / reps for k_, v in prof.items()}}
    return out


def _serving_run(fab, W, reqs, arr, slots):
    """Submit reqs at the arrival times arr (seconds), then poll all; returns latencies etc."""
    srv = fab.Server(slots=slots)
    for Mx, b, p, _ in reqs[:slots]:  # warm: workspaces and FP32 matrix copies
        try:
            srv.poll(srv.submit(Mx, b, p), timeout_ms=600000)
        except fab.FabError as e:
            if e.code != fab.FAB_ENOTCONV:  # a target miss still returns its best solution
                raise
    t0 = time.perf_counter()
    tickets = []
    for (Mx, b, p, cls), ta in zip(reqs, arr):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((srv.submit(Mx, b, p), cls))
    lat, miss, ms_used = [], [0, 0, 0], []
    for tk, cls in tickets:
        n_ = srv._mats.pop(tk)
        x = np.empty(n_)
        st = fab.Stats()
        lt = ctypes.c_double()
        rc = fab.lib.fab_server_poll(srv._s, ctypes.c_uint64(tk), x.ctypes.data, ctypes.byref(st), ctypes.byref(lt),
                                     600000)
        if rc == fab.FAB_ENOTCONV:
            miss[cls] += 1
        elif rc != fab.FAB_OK:
            raise RuntimeError(f"request failed: {rc}")
        lat.append(lt.value)
        ms_used.append(st.m_used)
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array(lat)
    return {"requests": len(reqs), "solves_per_s": len(reqs) / wall, "wall_s": wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "target_misses_by_class": {"convdiff2d": miss[0], "convdiff3d": miss[1], "graph": miss[2]},
            "mean_m_used": float(np.mean(ms_used))}


def bench_serving(fab, torch, W, count: int = 600, rate: float = 2000.0, slots: int = 16, pool: int = 12,
                  m_step: int = 20):
    """Continuous batching: Poisson arrivals (mean `rate` per s, seed 4) of f(A)b requests
    over a pool of pre-created handles, a third each 2D and 3D convection-diffusion and
    power-law graph Laplacians (n log-uniform on [1e4, 4e6], pool seed 5); exp(tA) for
    convection-diffusion with t ||A|| log-uniform on [50, 400], sqrt / inverse sqrt for
    the graphs; sketched_fast, SRHT s = 400, FP32 basis, m grown from 30 by m_step up to
    150 until the sketched relative change is below 1e-6. Two runs: the offered rate
    (saturating: its throughput is the sustainable rate) and half the sustainable rate
    (queueing-free latency). Latency = submission to completion."""
    import math as _m

    rng = np.random.default_rng(5)
    mats = []
    for i in range(pool):
        cls = i % 3
        n = float(np.exp(rng.uniform(_m.log(1e4), _m.log(4e6))))
        if cls == 0:
            N = max(10, int(round(_m.sqrt(n))))
            A = W.convdiff(2, N)
            lam = 8.0 * (N + 1) ** 2 + 20.0 * (N + 1)
        elif cls == 1:
            N = max(5, int(round(n ** (1.0 / 3.0))))
            A = W.convdiff(3, N)
            lam = 12.0 * (N + 1) ** 2 + 30.0 * (N + 1)
        else:
            A = W.chung_lu_laplacian(int(n), seed=2 + i)
            lam = None
        mats.append((fab.Matrix.from_csr(A), A.n, lam, cls))

    def requests(cnt, seed):
        r = np.random.default_rng(seed)
        pick = r.integers(0, pool, cnt)
        out = []
        for i in range(cnt):
            Mx, n, lam, cls = mats[pick[i]]
            if lam is not None:
                f, t = fab.EXP, -float(np.exp(r.uniform(_m.log(50.0), _m.log(400.0)))) / lam
            else:
                f, t = (fab.SQRT if r.random() < 0.5 else fab.INVSQRT), 1.0
            p = fab.params(f=f, t=t, m=30, k=2, s=400, sketch=fab.SRHT, seed=1 + i % 7, method=fab.SKETCHED_FAST,
                           precision=fab.MIXED, target_rel_err=1e-6, m_step=m_step, m_max=150)
            out.append((Mx, W.random_vector(n, 1000 + i), p, cls))
        return out

    sat = _serving_run(fab, W, requests(count, 6), W.poisson_arrivals(rate, count, seed=4), slots)
    low_rate = 0.5 * sat["solves_per_s"]
    low_cnt = max(50, int(round(low_rate * 8.0)))
    low = _serving_run(fab, W, requests(low_cnt, 7), W.poisson_arrivals(low_rate, low_cnt, seed=4), slots)
    return {"workload": f"Poisson arrivals over a pool of {pool} handles (2D/3D convection-diffusion, power-law "
                        "graphs; n 1e4..4e6), exp / sqrt / inverse sqrt, sketched_fast SRHT s=400, FP32 basis, "
                        f"m 30..150 (step {m_step}) grown to a 1e-6 sketched relative change",
            "slots": slots, "offered": {"rate_per_s": rate, **sat}, "half_sustainable": {"rate_per_s": low_rate, **low},
            "sustainable_solves_per_s": sat["solves_per_s"]}


def _dist():
    """(torch.distributed or None, rank, world size) from the torchrun environment;
    NCCL on GPUs, gloo otherwise (replicas exchange only their timings)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def max_over_ranks(dist, x: float) -> float:
    """The largest x over all ranks (the slowest replica's time)."""
    if dist is None:
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units processed by all replicas per second of the slowest replica."""
    return units_per_rank * world / max_seconds


def _oracle_small_stage_s(m: int, s: int, reps: int = 3) -> float:
    """Seconds the oracle's small stage of one solve takes at the workload's sizes
    (s x m QR of the sketched basis, the triangular solve of the sketch-and-solve
    form, exp of the m x m projected matrix): timed on a synthetic problem of those
    shapes, since the sampled solve has only a few columns."""
    import scipy.linalg

    import oracle

    rng = np.random.default_rng(0)
    SV = rng.standard_normal((s, m + 1))
    H = np.triu(rng.standard_normal((m, m)), -1) * 0.1
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        Q, R = np.linalg.qr(SV[:, :m])
        y = scipy.linalg.solve_triangular(R, Q.T @ SV[:, m], lower=False)
        Hh = H.copy()
        Hh[:, m - 1] += 0.01 * y
        _ = oracle.matfun.f_e1(Hh, oracle.matfun.EXP, T_EXP)
        best = min(best, time.perf_counter() - t0)
    return best


def cpu_oracle_sample(A, b, steps: int = CPU_SAMPLE_STEPS, small_s: float | None = None):
    """Time the FP64 CPU oracle on a bounded sample of one solve of the workload: the
    first `steps` steps of Alg. 2 (SpMV + window orthogonalization) on the full
    matrix, the SRHT sketch of those columns and their combine, measured; the per-step
    time is extrapolated linearly to the m = 100 steps of one solve, and the small
    stage (QR, triangular solve, f(H) at m = 100, s = 400) is added as measured on
    a problem of those shapes."""
    import oracle
    from paper_2212_12758_gb300 import workloads as W

    As = W.to_scipy(A)
    th = oracle.sketch.SRHT_(A.n, S_ROWS, SEED_SK)
    if small_s is None:
        small_s = _oracle_small_stage_s(M, S_ROWS)
    t0 = time.perf_counter()
    B = oracle.krylov.nt_basis(As, b, steps, K_WIN)
    _ = th.apply(B.V)
    _ = B.V[:, :steps] @ np.ones(steps)
    dt = time.perf_counter() - t0
    per_step = dt / (steps + 1)
    solve_s = per_step * (M + 1) + small_s
    cores = len(os.sched_getaffinity(0))
    return {"value": 1.0 / solve_s, "unit": "solves/s", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": f"first {steps} of {M} basis steps (Alg. 2 window k={K_WIN}, SRHT sketch, combine) of one "
                      f"solve on the full n={A.n} matrix, measured {dt:.2f} s and extrapolated to {M} steps; plus "
                      f"the m={M} small stage (QR, triangular solve, exp) measured on its own, {small_s * 1e3:.1f} ms"}


def run_reference(args):
    dist, rank, ws = _dist()
    if rank != 0:
        return 0
    from paper_2212_12758_gb300 import workloads as W

    A = W.convdiff(3, args.grid)
    b = W.random_vector(A.n, SEED_B)
    small_s = _oracle_small_stage_s(M, S_ROWS)
    for _ in range(args.warmup):
        cpu_oracle_sample(A, b, small_s=small_s)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(A, b, small_s=small_s))
    wall = time.perf_counter() - t0
    v = float(np.median([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.grid, A.n, A.nnz, ws),
            "extrapolated": True,
            "step": f"each of the {args.steps} timed steps is one bounded sample of a solve ({CPU_SAMPLE_STEPS} of "
                    f"{M} basis steps measured, extrapolated to a whole solve; value = median over the steps)",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)
    return 0


def run_only(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab
    from paper_2212_12758_gb300 import workloads as W

    if args.only == "mixed":
        A = W.convdiff(3, args.grid)
        Mx = fab.Matrix.from_csr(A)
        Mx.set_fusion(args.fusion)
        stream = torch.cuda.current_stream()
        bd = torch.from_numpy(W.random_vector(A.n, SEED_B)).cuda()

        def P(method, m=M):
            return fab.params(f=fab.EXP, t=T_EXP, m=m, k=K_WIN, s=S_ROWS, sketch=fab.SRHT, seed=SEED_SK,
                              method=method, lsqr_tol=1e-6, stream=stream.cuda_stream)

        out = {"workload": workload_name(args.grid, A.n, A.nnz).replace("FP64", "FP32 basis"),
               **bench_mixed_same(fab, torch, Mx, bd, None, stream, A.n, A.nnz, P, reps=args.steps)}
    elif args.only == "batch":
        out = bench_batch(fab, torch, W, steps=args.steps, count=args.batch_count)
    elif args.only == "bg":
        out = bench_bg_laplacian(fab, torch, W)
    elif args.only == "skew":
        out = bench_skew_convdiff(fab, torch, W)
    elif args.only == "whiten":
        out = bench_whiten_graph(fab, torch, W)
    elif args.only == "graph":
        out = bench_mixed_graph(fab, torch, W, reps=args.steps, n=args.graph_n, references=not args.no_extras)
    else:
        out = bench_serving(fab, torch, W, slots=args.serving_slots)
    print(json.dumps({"only": args.only, **out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fab", choices=["fab", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the sketched_ls / Arnoldi side measurements")
    ap.add_argument("--extras", default="mixed,batch,graph,bg,skew,whiten,serving",
                    help="side workloads measured after the main one: mixed (the same workload with an FP32 "
                         "basis), batch (256 uneven solves, one graph), "
                         "graph (4M-node power-law Laplacian, mixed precision, Gaussian sketch), serving "
                         "(Poisson arrivals, continuous batching, p50/p99 latency), bg (Alg. 3 vs Arnoldi on the "
                         "3D Laplacian), skew (every method on the skew-form convection-diffusion problem)")
    ap.add_argument("--only", choices=["mixed", "batch", "graph", "bg", "skew", "whiten", "serving"], default=None,
                    help="measure one side workload alone and print its JSON (for profiler runs)")
    ap.add_argument("--serving-slots", type=int, default=16, help="server slots of the --only serving workload")
    ap.add_argument("--fusion", action="store_true",
                    help="--only mixed: the one-pass basis steps (fab_set_fusion) in place of the two-pass loop "
                         "(SpMV + dots, then update + sketch)")
    ap.add_argument("--graph-n", type=int, default=4_000_000,
                    help="nodes of the --only graph workload (smaller only for profiler captures)")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="solves in the --only batch workload (same generator, batch seed 3)")
    ap.add_argument("--grid", type=int, default=N_GRID,
                    help="grid side N of the 3D operator (default 200, the benchmark workload; smaller N only "
                         "for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)

    import torch

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__

    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2212_12758_gb300 import fab
    from paper_2212_12758_gb300 import workloads as W

    A = W.convdiff(3, args.grid)
    b = W.random_vector(A.n, SEED_B)
    n, nnz = A.n, A.nnz
    Mx = fab.Matrix.from_csr(A)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def P(method, m=M):
        return fab.params(f=fab.EXP, t=T_EXP, m=m, k=K_WIN, s=S_ROWS, sketch=fab.SRHT, seed=SEED_SK, method=method,
                          lsqr_tol=1e-6, stream=sp)

    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    p_fast = P(fab.SKETCHED_FAST)
    # The last warm-up solve records every kernel class (the per-class shares). Each
    # recorded launch adds an event pair, so the timed region brackets only the
    # dominant kernel, whose average launch time the roofline needs.
    for i in range(args.warmup):
        if i == args.warmup - 1:
            fab.profile_enable(True)
        _, st = Mx.apply(bd, p_fast, x=xd, stats=True)
    torch.cuda.synchronize()
    prof_warm = fab.profile_query()
    fab.profile_enable(False)
    launches_per_solve = st.launches
    dom = max(("spmv_dots", "update", "fused_step"), key=lambda k_: prof_warm[k_][0])

    # FP64 FMA rate of this GPU at its current clocks (the arithmetic roof of the FP64
    # basis kernels), measured live with its own clock samples
    fma_clk = ClockSampler(local)
    fma_clk.start()
    try:
        fp64_peak, fp64_peak_ms = fab.fma_peak(fab.FP64, stream=sp)
        fp32_peak, _ = fab.fma_peak(fab.MIXED, stream=sp)
        fp64_src = ("measured (fab_fma_peak: independent FP64 FMA chains on every SM in three operand "
                    "patterns, the fastest kept; CUDA events)")
    except Exception:
        fp64_peak, fp64_peak_ms, fp32_peak = FP64_PEAK_GFLOPS_NOMINAL, 0.0, None
        fp64_src = "nominal (measurement failed)"
    fma_clocks = fma_clk.stop()

    # ---------------------------------------------------------------- timed
    clocks = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fab.profile_enable(True)
    fab.profile_only(dom)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for i in range(args.steps):
        evs[i][0].record(stream)
        Mx.apply(bd, p_fast, x=xd)
        evs[i][1].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    prof = fab.profile_query()
    fab.profile_enable(False)
    fab.profile_only(None)
    total_ms = max_over_ranks(dist, t_all0.elapsed_time(t_all1))
    lat = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
    solves_per_s = whole_job_rate(args.steps, ws, total_ms / 1000.0)
    ms_per_step = total_ms / args.steps

    # ------------------------------------------------------------ roofline
    cost = algorithmic_cost(n, nnz, M, K_WIN, S_ROWS)
    tot_ms, cnt = prof[dom]
    avg_s = tot_ms / max(cnt, 1) / 1000.0
    bytes_l, flops_l = cost[dom]
    peaks = _peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_frac = bytes_l / avg_s / 1e9 / hbm_peak
    alu_frac = flops_l / avg_s / 1e9 / fp64_peak
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": flops_l / avg_s / 1e9, "peak": fp64_peak,
                "unit": "GFLOP/s (FP64)", "frac": alu_frac}
    else:
        roof = {"bound": "hbm", "achieved": bytes_l / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_frac}
    traffic = SPMV_DRAM_BYTES_PER_ROW * n if dom == "spmv_dots" else None
    roof.update({"kernel": dom, "traffic": traffic, "traffic_source": "ncu dram__bytes on the 128^3 case, scaled by n"
                 if traffic else None, "ms_per_launch": avg_s * 1000.0,
                 "algorithmic_bytes_per_launch": bytes_l, "algorithmic_flops_per_launch": flops_l,
                 "hbm_gbs_algorithmic": bytes_l / avg_s / 1e9, "hbm_frac_of_measured": hbm_frac,
                 "fp64_gflops": flops_l / avg_s / 1e9, "fp64_frac_of_measured": alu_frac,
                 "fp64_peak": {"gflops": fp64_peak, "source": fp64_src, "ms": fp64_peak_ms, "clocks": fma_clocks,
                               "fp32_gflops": fp32_peak}})
    kernel_share = {k_: {"ms": v[0], "launches": v[1],
                         "share": v[0] / max(sum(x[0] for x in prof_warm.values()), 1e-9)}
                    for k_, v in prof_warm.items()}
    kernel_share["source"] = "CUDA events around every launch of the last warm-up solve"
    # the whole basis pass (SpMV + dots, update + norm + sketch, sketch reduce) of the
    # last warm-up solve against its floor: the larger of the single-pass bytes of
    # each step, 12 nnz + 4 (n+1) + 8 n (k+1), at the measured HBM rate and its FP64
    # operations, 2 nnz + 4 n k + 3 n, at the measured FP64 FMA rate
    basis_s = sum(prof_warm[k_][0] for k_ in ("spmv_dots", "update", "sketch_reduce")) / 1000.0
    b64 = sum(12 * nnz + 4 * (n + 1) + 8 * n * (min(c, K_WIN) + 1) for c in range(1, M + 1))
    f64 = sum(2 * nnz + 4 * n * min(c, K_WIN) + 3 * n for c in range(1, M + 1))
    floor_s = max(b64 / (hbm_peak * 1e9), f64 / (fp64_peak * 1e9))
    basis_pass = {"ms": basis_s * 1000.0, "bytes_8d": b64, "fp64_flops_8d": f64,
                  "floor_ms": floor_s * 1000.0, "floor_bound": "hbm" if b64 / hbm_peak >= f64 / fp64_peak else "fp64",
                  "frac_of_floor": floor_s / basis_s, "hbm_frac_vs_8d": b64 / basis_s / 1e9 / hbm_peak}
    # whole-solve algorithmic traffic (basis steps + combine)
    solve_bytes = M * (cost["spmv_dots"][0] + cost["update"][0]) + 8 * n * M
    hbm_gbs_solve = solve_bytes / (ms_per_step / 1000.0) / 1e9

    # ------------------------------------------------------- accuracy (untimed)
    x_fast = xd.clone()
    vs_oracle = oracle_golden_error(x_fast, Mx.last_state().coeffs) if args.grid == N_GRID else None
    extras = {}
    ref_x = None
    if not args.no_extras:
        xr = torch.empty_like(bd)
        Mx.apply(bd, P(fab.ARNOLDI, m=150), x=xr)
        xr2 = torch.empty_like(bd)
        Mx.apply(bd, P(fab.ARNOLDI, m=140), x=xr2)
        ref_x = xr
        ref_conv = float(torch.linalg.norm(xr - xr2) / torch.linalg.norm(xr))
        extras["reference_solution"] = {"method": "arnoldi m=150 (FP64, this library)",
                                        "rel_change_vs_m140": ref_conv}
        for name, meth in (("arnoldi", fab.ARNOLDI), ("sketched_ls", fab.SKETCHED_LS), ("noproj", fab.NOPROJ)):
            reps = 2 if meth == fab.ARNOLDI else 3
            xo = torch.empty_like(bd)
            Mx.apply(bd, P(meth), x=xo)  # warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                _, sto = Mx.apply(bd, P(meth), x=xo, stats=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            extras[name] = {"solves_per_s": 1000.0 / ms, "ms_per_solve": ms,
                            "rel_err": float(torch.linalg.norm(xo - ref_x) / torch.linalg.norm(ref_x)),
                            "lsqr_iters": sto.lsqr_iters}
    rel_err = float(torch.linalg.norm(x_fast - ref_x) / torch.linalg.norm(ref_x)) if ref_x is not None else None
    if not args.no_extras and "mixed" in args.extras.split(","):
        extras["mixed_same_workload"] = bench_mixed_same(fab, torch, Mx, bd, ref_x, stream, n, nnz, P)

    # ----------------------------------------------------------------- e2e
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    for _ in range(2):
        fab.lib.fab_apply(Mx._h, p_fast, bh.data_ptr(), xh.data_ptr(), 0, None)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = fab.lib.fab_apply(Mx._h, p_fast, bh.data_ptr(), xh.data_ptr(), 0, None)
        assert rc == 0, rc
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, (time.perf_counter() - t0) / e2e_steps)
    e2e = {"value": whole_job_rate(1, ws, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    if not args.no_extras and "batch" in args.extras.split(","):
        extras["batch_256"] = bench_batch(fab, torch, W)
    if not args.no_extras and "graph" in args.extras.split(","):
        extras["mixed_graph_4M"] = bench_mixed_graph(fab, torch, W)
    if not args.no_extras and "skew" in args.extras.split(","):
        extras["skew_convdiff_352"] = bench_skew_convdiff(fab, torch, W)
    if not args.no_extras and "whiten" in args.extras.split(","):
        extras["whiten_graph"] = bench_whiten_graph(fab, torch, W)
    if not args.no_extras and "bg" in args.extras.split(","):
        extras["bg_ls_laplacian3d"] = bench_bg_laplacian(fab, torch, W)
    if not args.no_extras and "serving" in args.extras.split(","):
        extras["serving"] = bench_serving(fab, torch, W)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(A, b)

    if rank == 0:
        line = {"metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": bench_config(args.grid, n, nnz, ws),
                "hbm_gbs": hbm_gbs_solve, "rel_err": rel_err, "rel_err_vs_oracle": vs_oracle,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "roofline": roof, "basis_pass": basis_pass, "kernels": kernel_share, "gpu_launches": launches_per_solve * args.steps,
                "e2e": e2e, "clocks": clk, "cpu_baseline": cpu, **extras}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
