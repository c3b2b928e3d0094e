"""GPU: the Gaussian sketch on the tensor cores and the mixed-precision path.

Gaussian entries are defined in FP64 (Box-Muller of SplitMix64 stream 5) and
rounded to BF16; sketching one-hot columns reveals G column by column, which
must equal the oracle's entries exactly. For general columns the device splits V
into two BF16 terms (hi + lo, exactly as the oracle's split_bf16) and accumulates
the exact BF16 products of both terms in FP32 within a split of the reduction,
then in FP64 across splits; the bound used is the classical accumulation bound
gamma_K sum |g| (|hi| + |lo|) with K = 2n (no assumption on the order), u = 2^-24.

Mixed precision (FP32 matrix and basis, FP64 small stage) is compared with the
FP64 oracle's f_m at the same m and sketch; the tolerance per case is stated
with the test.
"""
import numpy as np
import pytest

from oracle import krylov, matfun
from oracle import sketch as osk
from paper_2212_12758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fab():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2212_12758_gb300 import fab as f

    return f


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,s", [(5000, 300), (777, 128), (70000, 64)])
def test_gaussian_entries_bit_exact(fab, n, s):
    import torch

    rng = np.random.default_rng(n)
    cols = np.unique(np.r_[np.arange(min(60, n)), np.arange(n - 60, n), rng.integers(0, n, 100)])[:256]
    V = torch.zeros((len(cols), n), dtype=torch.float64, device="cuda")
    V[torch.arange(len(cols)), torch.from_numpy(cols).cuda()] = 1.0
    out = fab.sketch_apply(V, s, sketch=fab.GAUSSIAN, seed=9).cpu().numpy().T  # s x ncols
    G = osk.gaussian_entries(s, n, 9, bf16=True)
    mism = int(np.count_nonzero(out != G[:, cols]))
    assert mism == 0, f"{mism} Gaussian entries differ"


@pytest.mark.parametrize("n,s", [(70000, 300), (4096 * 3 + 5, 128)])
def test_gaussian_sketch_random_columns(fab, n, s):
    import torch

    rng = np.random.default_rng(1)
    Vh = rng.standard_normal((5, n)) * np.array([[1.0], [1e-5], [3e3], [1.0], [1.0]])
    out = fab.sketch_apply(torch.from_numpy(Vh).cuda(), s, sketch=fab.GAUSSIAN, seed=4).cpu().numpy()
    G = osk.gaussian_entries(s, n, 4, bf16=True)
    hi, lo = osk.split_bf16(Vh)
    ref = (hi + lo) @ G.T  # exact products of BF16 values, FP64 sums
    bound = 2 * n * 2.0**-24 * ((np.abs(hi) + np.abs(lo)) @ np.abs(G).T)
    assert np.all(np.abs(out - ref) <= bound)
    # the two terms carry v to 2^-16: far closer than one BF16 rounding (2^-8)
    assert np.all(np.abs(out - Vh @ G.T) <= (2.0**-16 + 2 * n * 2.0**-24) * (np.abs(Vh) @ np.abs(G).T))


CASES = [
    # name, matrix builder, f, t, m, k, sketch, s
    ("convdiff2d_exp_srht", lambda: W.convdiff(2, 100), matfun.EXP, -0.002, 30, 2, osk.SRHT, 120),
    ("graph_invsqrt_gauss", lambda: W.chung_lu_laplacian(20000, seed=2), matfun.INVSQRT, 1.0, 30, 2, osk.GAUSSIAN, 120),
    ("graph_sqrt_gauss", lambda: W.chung_lu_laplacian(20000, seed=2), matfun.SQRT, 1.0, 30, 2, osk.GAUSSIAN, 120),
]

from rounding_model import DRAWS, TAIL, U32, U_BF16, model_rms as _model_rms  # noqa: E402


@pytest.mark.parametrize("name,build,f,t,m,k,sk,s", CASES)
@pytest.mark.parametrize("method", [krylov.NOPROJ, krylov.SKETCHED_FAST, krylov.SKETCHED_LS, krylov.ARNOLDI])
def test_mixed_precision_vs_fp64_oracle(fab, name, build, f, t, m, k, sk, s, method):
    """FP32 matrix and basis (and the BF16 Gaussian sketch) against the FP64 oracle's f_m
    at the same m and sketch. The bar is TAIL x the RMS of the oracle's own change under
    DRAWS draws of the stated rounding model (_Fp32Operator, _Bf16Sketch): to first
    order the error is a linear function of many independent rounding errors, close to
    Gaussian, and a draw beyond 4 RMS is rare."""
    import torch

    A = build()
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    th = osk.make(sk, A.n, s, 3, 8)
    ref = krylov.run(method, As, b, m, k, f, th, t, tol=1e-10)
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=f, t=t, m=m, k=k, s=s, sketch=sk, seed=3, method=method, precision=fab.MIXED, lsqr_tol=1e-10)
    x = M.apply(torch.from_numpy(b).cuda(), p).cpu().numpy()
    err = _rel(x, ref.x)
    rms, mx = _model_rms(As, b, m, k, f, th, t, method, ref.x, sk == osk.GAUSSIAN and method != krylov.ARNOLDI)
    tol = TAIL * rms
    print(f"\nMIXED {name} method={method}: rel err vs FP64 oracle f_m = {err:.3e}; model RMS {rms:.3e} "
          f"(max of {DRAWS} {mx:.3e}); bar {tol:.3e}")
    assert err <= tol


@pytest.mark.parametrize("staged", [1, 2])
@pytest.mark.parametrize("name,build,f,t,m,k,sk,s", [c for c in CASES if c[6] == osk.GAUSSIAN])
def test_mixed_gaussian_stages(fab, name, build, f, t, m, k, sk, s, staged):
    """Stage by stage on the GPU's own quantities, sketched_fast with the BF16 Gaussian
    sketch: (1) the FP32 basis satisfies the Arnoldi-like relation (eq. arnoldilike)
    within the componentwise rounding bound gamma (|A||V_m| + |V_{m+1}||H|) with
    gamma = (max nnz per row + k + 2) u_32; (2) its sketch is G times the basis within
    (u_bf16^2 + 2 n u_32) |G| |V| entry by entry (the two-term BF16 split of each basis
    entry, FP32 accumulation of exact products over at most 2n terms); (3) the FP64 small stage
    (Remark after eq. sFOM: QR, y, f(Hhat) e_1) on the GPU's H and Theta V equals the
    oracle's to 1e-12. Both SpMV tile forms (a row per lane group; by nonzeros) are held
    to the same componentwise bound."""
    import torch

    A = build()
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    M = fab.Matrix.from_csr(A)
    M.set_tiling(256, 2048, staged)
    p = fab.params(f=f, t=t, m=m, k=k, s=s, sketch=sk, seed=3, method=krylov.SKETCHED_FAST, precision=fab.MIXED)
    M.apply(torch.from_numpy(b).cuda(), p)
    ls, V = M.last_state(), M.last_basis()
    # (1) Arnoldi-like relation of the FP32 basis
    gam = (int(np.diff(As.indptr).max()) + k + 2) * U32
    F = np.abs(As @ V[:, :m] - V @ ls.H)
    Bnd = gam * (abs(As) @ np.abs(V[:, :m]) + np.abs(V) @ np.abs(ls.H))
    assert np.all(F <= Bnd + 1e-300), float((F / (Bnd + 1e-300)).max())
    # (2) the sketch
    G = osk.gaussian_entries(s, A.n, 3, bf16=True)
    D = np.abs(ls.SV - G @ V)
    assert np.all(D <= (U_BF16**2 + 2 * A.n * U32) * (np.abs(G) @ np.abs(V))), "sketch outside its rounding bound"
    # (3) the FP64 small stage
    y, _, c, _ = krylov.sketch_solve_stage(ls.H, ls.SV, f, t)
    assert _rel(ls.y, y) <= 1e-12
    assert _rel(ls.coeffs, c) <= 1e-12


def _golden_c3():
    """The oracle's C3 solves and the rounding model's RMS at full size, as stored by
    tests/golden/make_c3_reference.py."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3_gauss.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        if parts[0] == "nnz":
            out["nnz"] = int(parts[1])
            continue
        d = out.setdefault(parts[0], {"x": {}})
        if parts[1] == "x":
            d["x"][int(parts[2])] = float(parts[3])
        elif parts[1] == "coeffs":
            d["coeffs"] = np.array([float(v) for v in parts[2:]])
        else:
            d[parts[1]] = float(parts[2])
    return out


@pytest.fixture(scope="module")
def c3_matrix():
    return W.chung_lu_laplacian(4_000_000, seed=2)


@pytest.mark.slow
@pytest.mark.parametrize("fname", ["invsqrt", "sqrt"])
def test_c3_full_size_against_the_oracle(fab, c3_matrix, fname):
    """The power-law graph workload at full size (n = 4M, nnz = 44M): m = 150, k = 2,
    Gaussian sketch s = 600 on the tensor cores (two BF16 terms), FP32 basis, FP64 small
    stage, sketched_fast. Against the FP64 oracle's f_m at the same m and sketch (stored:
    1024 sampled rows of x and the coefficients), at 4 x the rounding model's RMS at this
    size (stored with it); and stage by stage on the GPU's own quantities: the
    Arnoldi-like relation on sampled rows, the sketch on sampled sketch rows, the FP64
    small stage. The coefficient vector c (x = ||b|| V_m c) is printed, not held to the
    bar: the basis is far from orthogonal (the condition estimate of its sketch is
    printed), so rounding moves c by up to kappa times what it moves x, and the model's
    RMS is of x."""
    import torch

    A = c3_matrix
    gold = _golden_c3()
    assert gold["nnz"] == A.nnz
    g = gold[fname]
    f = matfun.INVSQRT if fname == "invsqrt" else matfun.SQRT
    m, k, s = 150, 2, 600
    b = W.random_vector(A.n, 0)
    M = fab.Matrix.from_csr(A)
    p = fab.params(f=f, t=1.0, m=m, k=k, s=s, sketch=fab.GAUSSIAN, seed=1, method=krylov.SKETCHED_FAST,
                   precision=fab.MIXED)
    x, st = M.apply(torch.from_numpy(b).cuda(), p, stats=True)
    x = x.cpu().numpy()
    ls = M.last_state()
    idx = np.array(sorted(g["x"]))
    xs = np.array([g["x"][i] for i in idx])
    e_x, e_c = _rel(x[idx], xs), _rel(ls.coeffs, g["coeffs"])
    bar = TAIL * g["model_rms"]
    print(f"\nC3 {fname}: rel err vs FP64 oracle f_m {e_x:.3e} (sampled rows), {e_c:.3e} (coefficients); bar {bar:.3e}; "
          f"kappa estimate of the sketched basis {st.kappa_est:.3e}")
    assert e_x <= bar
    # stage by stage: the FP64 small stage on the GPU's H and sketch
    y, _, c, _ = krylov.sketch_solve_stage(ls.H, ls.SV, f, 1.0)
    assert _rel(ls.coeffs, c) <= 1e-10
    # the relation A V_m = V_{m+1} H on sampled rows, within the FP32 componentwise bound
    V = torch.empty((m + 1, A.n), dtype=torch.float64, device="cuda")
    assert fab.lib.fab_last_basis(M._h, V.data_ptr(), 1) == 0
    As = W.to_scipy(A)
    rows = np.random.default_rng(1).choice(A.n, 64, replace=False)
    gam_rows = (np.diff(As.indptr)[rows] + k + 2) * U32
    A32 = As[rows].astype(np.float32).astype(np.float64)
    cols = np.unique(A32.indices)
    Vc = V[:, torch.from_numpy(cols).cuda()].cpu().numpy().T  # referenced rows of V
    Vr = V[:, torch.from_numpy(rows).cuda()].cpu().numpy().T
    A32c = A32[:, cols]
    F = np.abs(A32c @ Vc[:, :m] - Vr @ ls.H)
    B = gam_rows[:, None] * (abs(A32c) @ np.abs(Vc[:, :m]) + np.abs(Vr) @ np.abs(ls.H))
    assert np.all(F <= B + 1e-300)
    # the sketch on sampled sketch rows: within the two-term split and FP32 accumulation
    qs = np.array([0, 1, 257, 599])
    Gq = osk.gaussian_entries(s, A.n, 1, rows=qs, bf16=True)
    Vh = V.cpu().numpy().T  # n x (m+1)
    D = np.abs(ls.SV[qs] - Gq @ Vh)
    assert np.all(D <= (U_BF16**2 + 2 * A.n * U32) * (np.abs(Gq) @ np.abs(Vh)))
