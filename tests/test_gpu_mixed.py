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


@pytest.mark.parametrize("name,build,f,t,m,k,sk,s", [c for c in CASES if c[6] == osk.GAUSSIAN])
def test_mixed_gaussian_stages(fab, name, build, f, t, m, k, sk, s):
    """Stage by stage on the GPU's own quantities, sketched_fast with the BF16 Gaussian
    sketch: (1) the FP32 basis satisfies the Arnoldi-like relation (eq. arnoldilike)
    within the componentwise rounding bound gamma (|A||V_m| + |V_{m+1}||H|) with
    gamma = (max nnz per row + k + 2) u_32; (2) its sketch is G times the basis within
    (u_bf16^2 + 2 n u_32) |G| |V| entry by entry (the two-term BF16 split of each basis
    entry, FP32 accumulation of exact products over at most 2n terms); (3) the FP64 small stage
    (Remark after eq. sFOM: QR, y, f(Hhat) e_1) on the GPU's H and Theta V equals the
    oracle's to 1e-12."""
    import torch

    A = build()
    As = W.to_scipy(A)
    b = W.random_vector(A.n, 0)
    M = fab.Matrix.from_csr(A)
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
