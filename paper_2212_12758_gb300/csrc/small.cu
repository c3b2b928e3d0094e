// Small dense FP64 kernels of libfab: the m x m / s x m work after the basis
// loop. Householder QR of the sketch Theta V_m (the R factor of Blendenpik and
// of eq. sFOM), triangular solves, the projected matrix H_m + h y e_m^T
// (eq. relationxx), dense products and LU for f(H) (Pade scaling and squaring
// for exp, product-form Denman-Beavers for the square root), and the scalar
// recurrence of LSQR. Matrix sizes are read from the device (m_used), so a
// breakdown of the basis needs no host round trip.
#include <float.h>
#include <math.h>

#include <cooperative_groups.h>

#include "fab_internal.cuh"
#include "small.cuh"

namespace fab {

// ------------------------------------------------------------ Householder QR
// In place on A (rows x (mu + extra), column-major): R in the upper triangle,
// reflector vectors below it (implicit leading 1), tau[j]. The reflectors are
// also applied to the `extra` trailing columns (right-hand sides), which then
// hold Q^T rhs. Reflector j: beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta,
// v = x / (alpha - beta).
__device__ __forceinline__ void householder_qr_body(double* __restrict__ A, int lda, int rows, int mu, int extra,
                                                    double* __restrict__ tau) {
  __shared__ double red[32];
  __shared__ double s_beta, s_tau, s_vinv;
  const int ncols = mu + extra;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < mu && j < rows; ++j) {
    double* aj = A + (size_t)j * lda;
    double ss = 0.0;
    for (int i = j + 1 + tid; i < rows; i += blockDim.x) ss = fma(aj[i], aj[i], ss);
    ss = warp_sum(ss);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    if (tid == 0) {
      double sig = 0.0;
      for (int w = 0; w < nw; ++w) sig += red[w];
      const double alpha = aj[j];
      if (sig == 0.0) {
        s_tau = 0.0;
        s_beta = alpha;
        s_vinv = 0.0;
      } else {
        const double nrm = sqrt(fma(alpha, alpha, sig));
        const double beta = (alpha <= 0.0) ? nrm : -nrm;
        s_tau = (beta - alpha) / beta;
        s_vinv = 1.0 / (alpha - beta);
        s_beta = beta;
      }
    }
    __syncthreads();
    const double tj = s_tau, vinv = s_vinv;
    for (int i = j + 1 + tid; i < rows; i += blockDim.x) aj[i] *= vinv;
    __syncthreads();
    for (int col = j + 1 + warp; col < ncols; col += nw) {
      double* ac = A + (size_t)col * lda;
      double d = (lane == 0) ? ac[j] : 0.0;
      for (int i = j + 1 + lane; i < rows; i += 32) d = fma(aj[i], ac[i], d);
      d = warp_sum(d) * tj;
      if (lane == 0) ac[j] -= d;
      for (int i = j + 1 + lane; i < rows; i += 32) ac[i] = fma(-d, aj[i], ac[i]);
    }
    if (tid == 0) {
      tau[j] = tj;
      aj[j] = s_beta;
    }
    __syncthreads();
  }
}

__global__ __launch_bounds__(1024) void k_householder_qr(double* __restrict__ A, int lda, int rows,
                                                          const int* __restrict__ mdev, int extra,
                                                          double* __restrict__ tau) {
  householder_qr_body(A, lda, rows, *mdev, extra, tau);
}

cudaError_t launch_householder_qr(double* A, int lda, int rows, const int* mdev, int extra, double* tau,
                                  cudaStream_t s) {
  k_householder_qr<<<1, 1024, 0, s>>>(A, lda, rows, mdev, extra, tau);
  return cudaGetLastError();
}

// ------------------------------------------------------- triangular solves
// Block-wide solve with the upper triangle R of the leading mu x mu block (ld ldr):
// x = R^{-1} (p xin) (trans = 0) or R^{-T} (p xin) (trans = 1), published in the
// shared array xpub (xin may be xpub: the solve is then in place). Row i lives in a
// register of thread i % blockDim (mu <= kR blockDim); step j (mu sequential steps)
// solves x_j in its owner, publishes it behind one block barrier, and every row still
// to be solved takes its FMA. The entries of R a step needs are loaded two steps
// ahead, so their latency hides behind the barriers in between.
// sR (optional, mu * mu doubles of shared memory): R's upper triangle is staged there
// first, so that a step waits on shared memory instead of L2.
template <int kR>
__device__ __forceinline__ void trsv_core(const double* __restrict__ Rg, int ldg, int mu, const double* xin,
                                          double* xpub, int trans, double p, double* sR = nullptr) {
  const int tid = threadIdx.x, bd = blockDim.x;
  if (sR) {
    for (int idx = tid; idx < mu * mu; idx += bd) {
      const int i = idx % mu, j = idx / mu;
      if (i <= j) sR[idx] = Rg[i + (size_t)j * ldg];
    }
    __syncthreads();
  }
  const double* R = sR ? sR : Rg;
  const int ldr = sR ? mu : ldg;
  double xv[kR], dv[kR], r0[kR], r1[kR];
  // entry of row i that step j uses: R(i, j) (trans = 0, rows i < j) or R(j, i) (trans = 1, rows i > j)
  auto entry = [&](int i, int j) -> double {
    if (j < 0 || j >= mu) return 0.0;
    if (!trans) return i < j ? R[i + (size_t)j * ldr] : 0.0;
    return (i > j && i < mu) ? R[j + (size_t)i * ldr] : 0.0;
  };
  const int jfirst = trans ? 0 : mu - 1, dj = trans ? 1 : -1;
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const int i = tid + r * bd;
    xv[r] = i < mu ? p * xin[i] : 0.0;
    dv[r] = i < mu ? 1.0 / R[i + (size_t)i * ldr] : 1.0;  // reciprocal, off the sequential path
    r0[r] = entry(i, jfirst);
    r1[r] = entry(i, jfirst + dj);
  }
  __syncthreads();  // xin is read everywhere before xpub (maybe the same array) is written
  for (int step = 0; step < mu; ++step) {
    const int j = jfirst + step * dj;
    if (tid == j % bd) {
      const int rj = j / bd;
#pragma unroll
      for (int r = 0; r < kR; ++r)
        if (r == rj) xpub[j] = xv[r] * dv[r];
    }
    __syncthreads();
    const double xj = xpub[j];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      xv[r] = fma(-r0[r], xj, xv[r]);  // zero entry for rows the step does not touch
      r0[r] = r1[r];
      r1[r] = entry(tid + r * bd, j + 2 * dj);
    }
  }
  __syncthreads();
}

// x <- R^{-1} x (trans = 0) or R^{-T} x (trans = 1), with an optional pre-scale *pre.
__device__ __forceinline__ void trsv_body(const double* __restrict__ R, int ldr, int mu, const double* __restrict__ xin,
                                          double* __restrict__ xout, int trans, const double* __restrict__ pre,
                                          double* sR = nullptr) {
  __shared__ double xs[kMaxM];
  trsv_core<kMaxM / 256>(R, ldr, mu, xin, xs, trans, pre ? *pre : 1.0, sR);  // 256-thread blocks
  for (int i = threadIdx.x; i < mu; i += blockDim.x) xout[i] = xs[i];
}
// Largest triangle staged in shared memory by the one-block solves (180 KB).
constexpr int kTriSmemMax = 150;
inline size_t tri_smem_bytes(int mmax) { return mmax <= kTriSmemMax ? (size_t)mmax * mmax * sizeof(double) : 0; }

__global__ __launch_bounds__(1024) void k_trsv(const double* __restrict__ R, int ldr, const int* __restrict__ mdev,
                                                const double* __restrict__ xin, double* __restrict__ xout, int trans,
                                                const double* __restrict__ pre, int staged) {
  extern __shared__ double s_tri[];
  trsv_body(R, ldr, *mdev, xin, xout, trans, pre, staged ? s_tri : nullptr);
}

cudaError_t launch_trsv(const double* R, int ldr, const int* mdev, const double* xin, double* xout, int trans,
                        const double* pre, cudaStream_t s, int mmax) {
  const size_t smem = tri_smem_bytes(mmax);
  if (smem > 0) {
    const cudaError_t e = ensure_smem_limit((const void*)k_trsv, smem);
    if (e != cudaSuccess) return e;
  }
  k_trsv<<<1, 256, smem, s>>>(R, ldr, mdev, xin, xout, trans, pre, smem > 0 ? 1 : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------ projected matrix
// M = scale * (H_mu + h_{mu+1,mu} y e_mu^T), H column-major with ld ldh. y may be NULL.
__global__ void k_build_hhat(const double* __restrict__ H, int ldh, const int* __restrict__ mdev,
                             const double* __restrict__ y, double scale, double* __restrict__ M, int ldm) {
  const int mu = *mdev;
  const double hl = (y && mu > 0) ? H[mu + (size_t)ldh * (mu - 1)] : 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mu * mu; idx += gridDim.x * blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    double v = H[i + (size_t)ldh * j];
    if (y && j == mu - 1) v = fma(hl, y[i], v);
    M[i + (size_t)ldm * j] = scale * v;
  }
}

cudaError_t launch_build_hhat(const double* H, int ldh, const int* mdev, const double* y, double scale, double* M,
                              int ldm, int mmax, cudaStream_t s) {
  const int grid = (mmax * mmax + 255) / 256;
  k_build_hhat<<<grid < 1 ? 1 : (grid > 1024 ? 1024 : grid), 256, 0, s>>>(H, ldh, mdev, y, scale, M, ldm);
  return cudaGetLastError();
}

// ||M||_1 (maximum absolute column sum) into *out.
__device__ __forceinline__ double norm1_body(const double* __restrict__ M, int ldm, int mu, double* out) {
  __shared__ double red[32];
  __shared__ double s_out;
  double best = 0.0;
  for (int j = threadIdx.x; j < mu; j += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < mu; ++i) a += fabs(M[i + (size_t)ldm * j]);
    best = fmax(best, a);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, red[w]);
    if (out) *out = b;
    s_out = b;
  }
  __syncthreads();
  return s_out;
}

__global__ void k_norm1(const double* __restrict__ M, int ldm, const int* __restrict__ mdev, double* out) {
  norm1_body(M, ldm, *mdev, out);
}

cudaError_t launch_norm1(const double* M, int ldm, const int* mdev, double* out, cudaStream_t s) {
  k_norm1<<<1, 1024, 0, s>>>(M, ldm, mdev, out);
  return cudaGetLastError();
}

// --------------------------------------------------------- dense products
// C = alpha A B + beta C (mu x mu, common ld); C must not alias A or B.
// C = alpha A B + beta C for the leading mu x mu blocks (ld ld). FP64 runs at about two
// FMAs per clock per SM on GB300, so the product is spread over many SMs: one 8 x 8
// output tile per 64-thread block (169 blocks at mu = 100), with A's 8 rows and B's 8
// columns staged in shared memory 128 inner indices at a time.
constexpr int kGemmT = 8, kGemmK = 128;
__global__ __launch_bounds__(kGemmT * kGemmT) void k_gemm(double* __restrict__ C, const double* __restrict__ A,
                                                          const double* __restrict__ B, int ld,
                                                          const int* __restrict__ mdev, double alpha, double beta) {
  __shared__ double sA[kGemmK][kGemmT + 1];  // sA[l][i] = A(i0 + i, k0 + l)
  __shared__ double sB[kGemmK][kGemmT + 1];  // sB[l][j] = B(k0 + l, j0 + j)
  const int mu = *mdev;
  const int i0 = blockIdx.x * kGemmT, j0 = blockIdx.y * kGemmT;
  if (i0 >= mu || j0 >= mu) return;
  const int tid = threadIdx.x, ti = tid % kGemmT, tj = tid / kGemmT;
  double a0 = 0.0, a1 = 0.0;
  for (int k0 = 0; k0 < mu; k0 += kGemmK) {
    const int kn = mu - k0 < kGemmK ? mu - k0 : kGemmK;
    __syncthreads();  // the previous chunk is consumed
    for (int idx = tid; idx < kn * kGemmT; idx += kGemmT * kGemmT) {
      const int r = idx % kGemmT, l = idx / kGemmT;
      sA[l][r] = (i0 + r < mu) ? A[(i0 + r) + (size_t)ld * (k0 + l)] : 0.0;
      sB[l][r] = (j0 + r < mu) ? B[(k0 + l) + (size_t)ld * (j0 + r)] : 0.0;
    }
    __syncthreads();
    int l = 0;
    for (; l + 1 < kn; l += 2) {
      a0 = fma(sA[l][ti], sB[l][tj], a0);
      a1 = fma(sA[l + 1][ti], sB[l + 1][tj], a1);
    }
    if (l < kn) a0 = fma(sA[l][ti], sB[l][tj], a0);
  }
  const int i = i0 + ti, j = j0 + tj;
  if (i >= mu || j >= mu) return;
  const double acc = a0 + a1;
  C[i + (size_t)ld * j] = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * C[i + (size_t)ld * j]);
}

cudaError_t launch_gemm(double* C, const double* A, const double* B, int ld, const int* mdev, int mmax, double alpha,
                        double beta, cudaStream_t s) {
  dim3 grid((mmax + kGemmT - 1) / kGemmT, (mmax + kGemmT - 1) / kGemmT);
  k_gemm<<<grid, kGemmT * kGemmT, 0, s>>>(C, A, B, ld, mdev, alpha, beta);
  return cudaGetLastError();
}

// out = a0 X0 + a1 X1 + a2 X2 + a3 X3 + d I (any X may be NULL; out may alias one X)
__global__ void k_lincomb(double* out, const double* X0, const double* X1, const double* X2, const double* X3,
                          double a0, double a1, double a2, double a3, double d, int ld, const int* __restrict__ mdev) {
  const int mu = *mdev;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mu * mu; idx += gridDim.x * blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    const size_t o = i + (size_t)ld * j;
    double v = (i == j) ? d : 0.0;
    if (X0) v = fma(a0, X0[o], v);
    if (X1) v = fma(a1, X1[o], v);
    if (X2) v = fma(a2, X2[o], v);
    if (X3) v = fma(a3, X3[o], v);
    out[o] = v;
  }
}

cudaError_t launch_lincomb(double* out, const double* X0, const double* X1, const double* X2, const double* X3,
                           double a0, double a1, double a2, double a3, double d, int ld, const int* mdev, int mmax,
                           cudaStream_t s) {
  int grid = (mmax * mmax + 255) / 256;
  grid = grid < 1 ? 1 : (grid > 1024 ? 1024 : grid);
  k_lincomb<<<grid, 256, 0, s>>>(out, X0, X1, X2, X3, a0, a1, a2, a3, d, ld, mdev);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- LU
// In-place LU with partial pivoting (rows swapped across the whole matrix,
// ties to the smallest row index). piv[k] = row swapped with k. Writes
// log|det| to *logdet and flags a zero pivot in st->status (FAB_ENUMERIC).
__device__ __forceinline__ void lu_body(double* __restrict__ M, int ld, int mu, int* __restrict__ piv,
                                        double* __restrict__ logdet, DevState* st) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int s_p;
  __shared__ double s_logdet;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) s_logdet = 0.0;
  for (int k = 0; k < mu; ++k) {
    double best = -1.0;
    int bi = mu;
    for (int i = k + tid; i < mu; i += blockDim.x) {
      const double a = fabs(M[i + (size_t)ld * k]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      rv[warp] = best;
      ri[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = mu;
      for (int w = 0; w < nw; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < p)) {
          b = rv[w];
          p = ri[w];
        }
      if (p < k || p >= mu) {  // only with non-finite entries: keep the row, flag the matrix
        p = k;
        st->status = FAB_ENUMERIC;
      }
      s_p = p;
      piv[k] = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != k) {
      for (int j = tid; j < mu; j += blockDim.x) {
        const double t = M[k + (size_t)ld * j];
        M[k + (size_t)ld * j] = M[p + (size_t)ld * j];
        M[p + (size_t)ld * j] = t;
      }
    }
    __syncthreads();
    const double pivot = M[k + (size_t)ld * k];
    if (tid == 0) {
      if (pivot == 0.0 || !isfinite(pivot)) {
        st->status = FAB_ENUMERIC;
      } else {
        s_logdet += log(fabs(pivot));
      }
    }
    const double pinv = (pivot != 0.0) ? 1.0 / pivot : 0.0;
    for (int i = k + 1 + tid; i < mu; i += blockDim.x) M[i + (size_t)ld * k] *= pinv;
    __syncthreads();
    const int r = mu - k - 1;
    for (int idx = tid; idx < r * r; idx += blockDim.x) {
      const int i = k + 1 + idx % r, j = k + 1 + idx / r;
      M[i + (size_t)ld * j] = fma(-M[i + (size_t)ld * k], M[k + (size_t)ld * j], M[i + (size_t)ld * j]);
    }
    __syncthreads();
  }
  if (tid == 0 && logdet) *logdet = s_logdet;
  __syncthreads();
}

__global__ __launch_bounds__(1024) void k_lu(double* __restrict__ M, int ld, const int* __restrict__ mdev,
                                              int* __restrict__ piv, double* __restrict__ logdet, DevState* st) {
  lu_body(M, ld, *mdev, piv, logdet, st);
}

cudaError_t launch_lu(double* M, int ld, const int* mdev, int* piv, double* logdet, DevState* st, cudaStream_t s) {
  k_lu<<<1, 1024, 0, s>>>(M, ld, mdev, piv, logdet, st);
  return cudaGetLastError();
}

// Solve LU X = P B in place for the mu columns of B (one warp per column at a time,
// column-oriented substitution). identity_rhs: B is set to I first. staged: every
// block first copies the mu x mu factors into shared memory, so that the 2 mu
// dependent substitution steps of a column read shared memory instead of L2.
__global__ void k_lu_solve(const double* __restrict__ LUg, int ldg, const int* __restrict__ piv,
                           const int* __restrict__ mdev, double* __restrict__ B, int ldb, int identity_rhs,
                           int staged, int wpb) {
  extern __shared__ double sm[];
  const int mu = *mdev;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (staged) {  // every warp of the block stages; only the first wpb_solve warps solve
#pragma unroll 4
    for (int idx = threadIdx.x; idx < mu * mu; idx += blockDim.x) sm[idx] = LUg[idx % mu + (size_t)ldg * (idx / mu)];
    __syncthreads();
  }
  const double* LU = staged ? sm : LUg;
  const int ld = staged ? mu : ldg;
  // staged: reciprocals of U's diagonal after the factors (one division per row, in
  // parallel, instead of one per step on the sequential path)
  double* dinv = staged ? sm + (size_t)mu * mu : nullptr;
  if (staged) {
    for (int k = threadIdx.x; k < mu; k += blockDim.x) dinv[k] = 1.0 / sm[k + (size_t)mu * k];
    __syncthreads();
  }
  double* b = sm + (staged ? (size_t)mu * mu + mu : 0) + (size_t)warp * mu;
  for (int col = blockIdx.x * wpb + warp; warp < wpb && col < mu; col += gridDim.x * wpb) {
    double* bg = B + (size_t)ldb * col;
    int kstart = 0;
    if (identity_rhs) {
      // P e_col is the unit vector at the row the swaps carry col to; every lane follows
      // it through the swap sequence, and the forward pass starts there (zeros above)
      int pos = col;
      for (int k = 0; k < mu; ++k) {
        const int p = piv[k];
        if (p != k && p > k && p < mu) pos = (pos == k) ? p : (pos == p ? k : pos);
      }
      for (int i = lane; i < mu; i += 32) b[i] = (i == pos) ? 1.0 : 0.0;
      kstart = pos;
    } else {
      for (int i = lane; i < mu; i += 32) b[i] = bg[i];
      __syncwarp();
      if (lane == 0) {
        for (int k = 0; k < mu; ++k) {
          const int p = piv[k];
          if (p != k && p > k && p < mu) {
            const double t = b[k];
            b[k] = b[p];
            b[p] = t;
          }
        }
      }
    }
    __syncwarp();
    for (int k = kstart; k < mu; ++k) {  // unit lower
      const double bk = b[k];
      for (int i = k + 1 + lane; i < mu; i += 32) b[i] = fma(-LU[i + (size_t)ld * k], bk, b[i]);
      __syncwarp();
    }
    for (int k = mu - 1; k >= 0; --k) {  // upper
      if (lane == 0) b[k] = dinv ? b[k] * dinv[k] : b[k] / LU[k + (size_t)ld * k];
      __syncwarp();
      const double bk = b[k];
      for (int i = lane; i < k; i += 32) b[i] = fma(-LU[i + (size_t)ld * k], bk, b[i]);
      __syncwarp();
    }
    for (int i = lane; i < mu; i += 32) bg[i] = b[i];
    __syncwarp();
  }
}

cudaError_t launch_lu_solve(const double* LU, int ld, const int* piv, const int* mdev, int mmax, double* B, int ldb,
                            int identity_rhs, cudaStream_t s) {
  const size_t stage = (size_t)mmax * mmax * sizeof(double);
  if (mmax <= 160) {  // factors staged by 8 warps; 2 of them solve: the FP64 work spreads over mmax / 2 SMs
    const int wpb = 2;
    const size_t smem = stage + (size_t)(wpb + 1) * mmax * sizeof(double);
    const cudaError_t e = ensure_smem_limit((const void*)k_lu_solve, smem);
    if (e != cudaSuccess) return e;
    const int grid = (mmax + wpb - 1) / wpb;
    k_lu_solve<<<grid, 256, smem, s>>>(LU, ld, piv, mdev, B, ldb, identity_rhs, 1, wpb);
    return cudaGetLastError();
  }
  const int wpb = 4;
  const int grid = (mmax + wpb - 1) / wpb;
  k_lu_solve<<<grid, wpb * 32, (size_t)wpb * mmax * sizeof(double), s>>>(LU, ld, piv, mdev, B, ldb, identity_rhs, 0,
                                                                         wpb);
  return cudaGetLastError();
}

// --------------------------------------------------- Denman-Beavers step
// Product form with determinant scaling (mu_k = |det M_k|^{-1/(2 m)}):
//   M <- (I + (mu^2 M + mu^-2 Minv) / 2) / 2,   y <- mu (y + mu^-2 Minv y) / 2,
// with M_0 = Y_0 = H (y_0 = H e_1 for the square root, e_1 for the inverse
// square root with Z_0 = I). Writes ||M - I||_F to st->scal[1].
__device__ __forceinline__ void db_update_body(double* __restrict__ M, const double* __restrict__ Minv, int ld, int mu,
                                               double* __restrict__ y, const double* __restrict__ logdet,
                                               int scale_on, DevState* st) {
  __shared__ double ys[kMaxM];
  __shared__ double red[32];
  const double g = scale_on ? exp(-(*logdet) / (2.0 * mu)) : 1.0;
  const double g2 = g * g, gi2 = 1.0 / g2;
  for (int i = threadIdx.x; i < mu; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int i = threadIdx.x; i < mu; i += blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;  // four chains: FP64 latency, not throughput, bounds this
    int j = 0;
    for (; j + 3 < mu; j += 4) {
      a0 = fma(Minv[i + (size_t)ld * j], ys[j], a0);
      a1 = fma(Minv[i + (size_t)ld * (j + 1)], ys[j + 1], a1);
      a2 = fma(Minv[i + (size_t)ld * (j + 2)], ys[j + 2], a2);
      a3 = fma(Minv[i + (size_t)ld * (j + 3)], ys[j + 3], a3);
    }
    for (; j < mu; ++j) a0 = fma(Minv[i + (size_t)ld * j], ys[j], a0);
    y[i] = 0.5 * g * fma(gi2, (a0 + a1) + (a2 + a3), ys[i]);
  }
  double err = 0.0;
  for (int idx = threadIdx.x; idx < mu * mu; idx += blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    const size_t o = i + (size_t)ld * j;
    const double v = 0.5 * ((i == j ? 1.0 : 0.0) + 0.5 * fma(g2, M[o], gi2 * Minv[o]));
    M[o] = v;
    const double dv = v - (i == j ? 1.0 : 0.0);
    err = fma(dv, dv, err);
  }
  err = warp_sum(err);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = err;
  __syncthreads();
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) e += red[w];
    st->scal[1] = sqrt(e);
    if (!isfinite(e)) st->status = FAB_ENUMERIC;
  }
  __syncthreads();
}

// The same step over many blocks (a single SM's FP64 rate made the m^2 elementwise
// update the bottleneck): block 0 alone forms y from Minv and the old y (no other
// block touches y); every block updates its slice of M and adds its share of
// ||M - I||_F^2 to part[]; the last block sums the shares in block order.
__global__ __launch_bounds__(256) void k_db_update(double* __restrict__ M, const double* __restrict__ Minv, int ld,
                                                     const int* __restrict__ mdev, double* __restrict__ y,
                                                     const double* __restrict__ logdet, int scale_on,
                                                     double* __restrict__ part, unsigned* __restrict__ counter,
                                                     DevState* st) {
  __shared__ double ys[kMaxM];
  __shared__ double red[32];
  __shared__ double tot[1];
  const int mu = *mdev;
  const double g = scale_on ? exp(-(*logdet) / (2.0 * mu)) : 1.0;
  const double g2 = g * g, gi2 = 1.0 / g2;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < mu; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (int i = threadIdx.x; i < mu; i += blockDim.x) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = 0;
      for (; j + 3 < mu; j += 4) {
        a0 = fma(Minv[i + (size_t)ld * j], ys[j], a0);
        a1 = fma(Minv[i + (size_t)ld * (j + 1)], ys[j + 1], a1);
        a2 = fma(Minv[i + (size_t)ld * (j + 2)], ys[j + 2], a2);
        a3 = fma(Minv[i + (size_t)ld * (j + 3)], ys[j + 3], a3);
      }
      for (; j < mu; ++j) a0 = fma(Minv[i + (size_t)ld * j], ys[j], a0);
      y[i] = 0.5 * g * fma(gi2, (a0 + a1) + (a2 + a3), ys[i]);
    }
  }
  double err = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < mu * mu; idx += gridDim.x * blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    const size_t o = i + (size_t)ld * j;
    const double v = 0.5 * ((i == j ? 1.0 : 0.0) + 0.5 * fma(g2, M[o], gi2 * Minv[o]));
    M[o] = v;
    const double dv = v - (i == j ? 1.0 : 0.0);
    err = fma(dv, dv, err);
  }
  double ev[1] = {err};
  block_sum<1>(ev, red);
  if (threadIdx.x == 0) part[blockIdx.x] = ev[0];
  if (!last_block(counter)) return;
  sum_partials(part, gridDim.x, 1, tot, red);
  if (threadIdx.x == 0) {
    st->scal[1] = sqrt(tot[0]);
    if (!isfinite(tot[0])) st->status = FAB_ENUMERIC;
    *counter = 0;
  }
}

cudaError_t launch_db_update(double* M, const double* Minv, int ld, const int* mdev, double* y, const double* logdet,
                             int scale_on, DevState* st, cudaStream_t s, int mmax, double* part, unsigned* counter) {
  const int nb = (mmax * mmax + 1023) / 1024;  // about four entries per thread
  const int grid = nb < 1 ? 1 : (nb > 64 ? 64 : nb);
  k_db_update<<<grid, 256, 0, s>>>(M, Minv, ld, mdev, y, logdet, scale_on, part, counter, st);
  return cudaGetLastError();
}

// Copy column 0 of M (or e_1 when M is NULL) into y.
__global__ void k_first_column(const double* __restrict__ M, const int* __restrict__ mdev, double* __restrict__ y) {
  const int mu = *mdev;
  for (int i = threadIdx.x; i < mu; i += blockDim.x) y[i] = M ? M[i] : (i == 0 ? 1.0 : 0.0);
}

cudaError_t launch_first_column(const double* M, const int* mdev, double* y, cudaStream_t s) {
  k_first_column<<<1, 1024, 0, s>>>(M, mdev, y);
  return cudaGetLastError();
}

// coef_j = ||b|| c_j sigma_j for the combine x = sum_j coef_j W_j.
__global__ void k_prep_coef(const double* __restrict__ c, const double* __restrict__ sigma,
                            const int* __restrict__ mdev, const DevState* st, double* __restrict__ coef) {
  const int mu = *mdev;
  for (int j = threadIdx.x; j < mu; j += blockDim.x) coef[j] = st->beta * c[j] * sigma[j];
}

cudaError_t launch_prep_coef(const double* c, const double* sigma, const int* mdev, const DevState* st, double* coef,
                             cudaStream_t s) {
  k_prep_coef<<<1, 1024, 0, s>>>(c, sigma, mdev, st, coef);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ LSQR
// State in st->scal: 0 alpha, 1 beta, 2 phibar, 3 rhobar, 4 anorm2, 5 tau
// (u = tau * ustore), 6 keep (= -alpha * tau, the factor of ustore in the next
// u update), 7 tol. m-vectors in lv: v, w, x, z (= R^{-1} v), coef (= sigma z).
// Paige-Saunders recurrences, in the order of their published algorithm.

__device__ void lsqr_block_norm(const double* a, int mu, double* red, double* out) {
  double ss = 0.0;
  for (int i = threadIdx.x; i < mu; i += blockDim.x) ss = fma(a[i], a[i], ss);
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = sqrt(t);
  }
  __syncthreads();
}

// Back substitution z = R^{-1} v in shared memory, in place (block-wide).
// (the LSQR kernels run kMaxM threads: one row each)
__device__ void lsqr_trsv(const double* R, int ldr, int mu, double* zs, double* sR) {
  trsv_core<1>(R, ldr, mu, zs, zs, 0, 1.0, sR);
}

// Start: beta_1 from ||ustore|| (u_1 = v_{m+1} = sigma_mu ustore), then
// v = R^{-T} V_m^T u_1, alpha, w = v, phibar = beta_1, rhobar = alpha, x = 0.
__global__ __launch_bounds__(1024) void k_lsqr_start(const double* __restrict__ R, int ldr,
                                                      const int* __restrict__ mdev, const double* __restrict__ sigma,
                                                      const double* __restrict__ unorm2, LsqrVecs lv, double tol,
                                                      DevState* st, int staged) {
  extern __shared__ double s_tri[];  // R's triangle (staged) or unused
  double* sR = staged ? s_tri : nullptr;
  __shared__ double vs[kMaxM];
  __shared__ double red[32];
  __shared__ double s_nrm;
  const int mu = *mdev;
  const double beta1 = sigma[mu] * sqrt(*unorm2);
  const double tau = (beta1 > 0.0) ? sigma[mu] / beta1 : 0.0;
  // v = R^{-T} (tau q)
  trsv_core<1>(R, ldr, mu, lv.q, vs, 1, tau, sR);
  lsqr_block_norm(vs, mu, red, &s_nrm);
  const double alpha = s_nrm;
  const double ainv = alpha > 0.0 ? 1.0 / alpha : 0.0;
  for (int i = threadIdx.x; i < mu; i += blockDim.x) {
    const double vi = vs[i] * ainv;
    vs[i] = vi;
    lv.v[i] = vi;
    lv.w[i] = vi;
    lv.x[i] = 0.0;
  }
  __syncthreads();
  lsqr_trsv(sR ? sR : R, sR ? mu : ldr, mu, vs, nullptr);  // z = R^{-1} v (triangle already staged)
  for (int i = threadIdx.x; i < mu; i += blockDim.x) {
    lv.z[i] = vs[i];
    lv.coef[i] = sigma[i] * vs[i];
  }
  if (threadIdx.x == 0) {
    st->scal[0] = alpha;
    st->scal[1] = beta1;
    st->scal[2] = beta1;
    st->scal[3] = alpha;
    st->scal[4] = 0.0;
    st->scal[5] = tau;
    st->scal[6] = -alpha * tau;
    st->scal[7] = tol;
    st->iters = 0;
    st->flag = (beta1 == 0.0 || alpha == 0.0) ? 1 : 0;
  }
}

cudaError_t launch_lsqr_start(const double* R, int ldr, const int* mdev, const double* sigma, const double* unorm2,
                              const LsqrVecs& lv, double tol, DevState* st, cudaStream_t s, int mmax) {
  const size_t smem = tri_smem_bytes(mmax);
  if (smem > 0) {
    const cudaError_t e = ensure_smem_limit((const void*)k_lsqr_start, smem);
    if (e != cudaSuccess) return e;
  }
  k_lsqr_start<<<1, 1024, smem, s>>>(R, ldr, mdev, sigma, unorm2, lv, tol, st, smem > 0 ? 1 : 0);
  return cudaGetLastError();
}

// After ustore <- V_m z - alpha u (unnormalized) with ||ustore||^2 in *unorm2 and
// q_j = sigma_j <W_j, ustore>:
//   beta = ||ustore||, anorm2 += alpha^2 + beta^2, u = ustore / beta,
//   v <- R^{-T} (q / beta) - beta v, alpha = ||v||, v /= alpha,
//   rotation, x += (phi/rho) w, w = v - (theta/rho) w, stopping test,
//   z = R^{-1} v, coef = sigma z, keep = -alpha / beta.
__global__ __launch_bounds__(1024) void k_lsqr_step(const double* __restrict__ Rg, int ldg,
                                                     const int* __restrict__ mdev, const double* __restrict__ sigma,
                                                     const double* __restrict__ unorm2, LsqrVecs lv, DevState* st,
                                                     int staged) {
  extern __shared__ double s_tri[];  // R's triangle (staged) or unused
  __shared__ double vs[kMaxM];
  __shared__ double red[32];
  __shared__ double s_nrm;
  if (st->flag) return;
  const int mu = *mdev;
  if (staged) {  // both solves below read the triangle from shared memory
    for (int idx = threadIdx.x; idx < mu * mu; idx += blockDim.x) {
      const int i = idx % mu, j = idx / mu;
      if (i <= j) s_tri[idx] = Rg[i + (size_t)j * ldg];
    }
    __syncthreads();
  }
  const double* R = staged ? s_tri : Rg;
  const int ldr = staged ? mu : ldg;
  double alpha = st->scal[0];
  const double beta = sqrt(*unorm2);
  const double anorm2 = st->scal[4] + alpha * alpha + beta * beta;
  double alpha_new = alpha;
  if (beta > 0.0) {
    const double binv = 1.0 / beta;
    trsv_core<1>(R, ldr, mu, lv.q, vs, 1, binv);
    for (int i = threadIdx.x; i < mu; i += blockDim.x) vs[i] = fma(-beta, lv.v[i], vs[i]);
    __syncthreads();
    lsqr_block_norm(vs, mu, red, &s_nrm);
    alpha_new = s_nrm;
    if (alpha_new > 0.0) {
      const double ainv = 1.0 / alpha_new;
      for (int i = threadIdx.x; i < mu; i += blockDim.x) vs[i] *= ainv;
    }
    __syncthreads();
  } else {
    for (int i = threadIdx.x; i < mu; i += blockDim.x) vs[i] = lv.v[i];
    __syncthreads();
  }
  const double rhobar = st->scal[3], phibar = st->scal[2];
  const double rho = hypot(rhobar, beta);
  const double c = rhobar / rho, sn = beta / rho;
  const double theta = sn * alpha_new;
  const double rhobar_new = -c * alpha_new;
  const double phi = c * phibar;
  const double phibar_new = sn * phibar;
  const double f1 = phi / rho, f2 = theta / rho;
  for (int i = threadIdx.x; i < mu; i += blockDim.x) {
    const double wi = lv.w[i];
    lv.x[i] = fma(f1, wi, lv.x[i]);
    lv.w[i] = fma(-f2, wi, vs[i]);
    lv.v[i] = vs[i];
  }
  __syncthreads();
  lsqr_trsv(R, ldr, mu, vs, nullptr);
  for (int i = threadIdx.x; i < mu; i += blockDim.x) {
    lv.z[i] = vs[i];
    lv.coef[i] = sigma[i] * vs[i];
  }
  if (threadIdx.x == 0) {
    const double tol = st->scal[7];
    st->scal[0] = alpha_new;
    st->scal[1] = beta;
    st->scal[2] = phibar_new;
    st->scal[3] = rhobar_new;
    st->scal[4] = anorm2;
    st->scal[5] = beta > 0.0 ? 1.0 / beta : 0.0;
    st->scal[6] = beta > 0.0 ? -alpha_new / beta : 0.0;
    st->iters += 1;
    const bool done = (phibar_new * alpha_new * fabs(c) <= tol * sqrt(anorm2) * phibar_new) || beta == 0.0 ||
                      alpha_new == 0.0;
    if (done) st->flag = 1;
    if (!isfinite(anorm2) || !isfinite(phibar_new)) {
      st->status = FAB_ENUMERIC;
      st->flag = 1;
    }
  }
}

cudaError_t launch_lsqr_step(const double* R, int ldr, const int* mdev, const double* sigma, const double* unorm2,
                             const LsqrVecs& lv, DevState* st, cudaStream_t s, int mmax) {
  const size_t smem = tri_smem_bytes(mmax);
  if (smem > 0) {
    const cudaError_t e = ensure_smem_limit((const void*)k_lsqr_step, smem);
    if (e != cudaSuccess) return e;
  }
  k_lsqr_step<<<1, 1024, smem, s>>>(R, ldr, mdev, sigma, unorm2, lv, st, smem > 0 ? 1 : 0);
  return cudaGetLastError();
}

// ustore[r] <- sum_q coef_q W_q[r] + keep * ustore[r] with keep = st->scal[6]
// (keep_zero: ustore is overwritten); ||ustore||^2 reduced over the grid into *unorm2.
template <typename TV>
__global__ __launch_bounds__(kThreads) void k_lsqr_u(int n, const TV* __restrict__ W, int64_t ld, int nc,
                                                      const double* __restrict__ coef, double* __restrict__ u,
                                                      int keep_zero, double* __restrict__ part,
                                                      unsigned* __restrict__ counter, double* __restrict__ unorm2,
                                                      const DevState* st) {
  extern __shared__ double s_cf[];
  __shared__ double sh[32];
  __shared__ double tot[1];
  if (st->flag) return;
  const double keep = keep_zero ? 0.0 : st->scal[6];
  combine_coef_load<TV>(s_cf, coef, nc);
  __syncthreads();
  double nrm = 0.0;
  for (int r = blockIdx.x * kThreads + threadIdx.x; r < n; r += gridDim.x * kThreads) {
    double a = combine_row<TV>(W, ld, nc, s_cf, r);
    if (!keep_zero) a = fma(keep, u[r], a);
    u[r] = a;
    nrm = fma(a, a, nrm);
  }
  double nv[1] = {nrm};
  block_sum<1>(nv, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = nv[0];
  if (!last_block(counter)) return;
  sum_partials(part, gridDim.x, 1, tot, sh);
  if (threadIdx.x == 0) {
    *unorm2 = tot[0];
    *counter = 0;
  }
}

template <typename TV>
cudaError_t launch_lsqr_u(int n, const TV* W, int64_t ld, int nc, const double* coef, double* u, int keep_zero,
                          double* part, unsigned* counter, double* unorm2, const DevState* st, cudaStream_t s) {
  k_lsqr_u<TV><<<grid_rows(n), kThreads, (size_t)(nc > 0 ? nc : 1) * 8, s>>>(n, W, ld, nc, coef, u, keep_zero, part,
                                                                          counter, unorm2, st);
  return cudaGetLastError();
}
template cudaError_t launch_lsqr_u<double>(int, const double*, int64_t, int, const double*, double*, int, double*,
                                           unsigned*, double*, const DevState*, cudaStream_t);
template cudaError_t launch_lsqr_u<float>(int, const float*, int64_t, int, const double*, double*, int, double*,
                                          unsigned*, double*, const DevState*, cudaStream_t);


// ------------------------------------------------ cluster QR / LU (DSMEM)
// The s x (mu+extra) matrix of the QR (or the mu x mu matrix of the LU) is
// distributed by columns over the CTAs of one thread-block cluster: global
// column g lives in shared memory of CTA g % CL. At step j the owner of column j
// forms the reflector (QR) or the pivot and multipliers (LU); after one cluster
// barrier every CTA reads that vector from the owner's shared memory and updates
// its own columns. One cluster barrier per step; the FP64 work of a step is
// spread over CL SMs instead of one.
namespace cg = cooperative_groups;

template <int CL>
__global__ void __launch_bounds__(256) k_qr_cluster(double* __restrict__ A, int lda, int rows,
                                                    const int* __restrict__ mdev, int extra,
                                                    double* __restrict__ tau_out, int start, int fresh,
                                                    DevState* st) {
  extern __shared__ __align__(16) double smem_d[];
  __shared__ double red[32];
  __shared__ double s_tau[kMaxM];
  __shared__ int s_flag[kMaxM];  // s_flag[j] = 1 once reflector j is published
  __shared__ int s_fail;
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int mu = *mdev;
  const int ncols = mu + extra;
  const int nloc = (ncols - r + CL - 1) / CL;  // my columns: g = r, r + CL, ...
  double* loc = smem_d;                             // nloc x rows
  double* vbuf = smem_d + (size_t)((ncols + CL - 1) / CL) * rows;  // rows
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int lc = 0; lc < nloc; ++lc) {
    const double* src = A + (size_t)(lc * CL + r) * lda;
    for (int i = tid; i < rows; i += blockDim.x) loc[(size_t)lc * rows + i] = src[i];
  }
  __syncthreads();
  const int steps = mu < rows ? mu : rows;
  // reflector j from the owner's column j (block-wide): v below the diagonal, beta on it
  auto reflector = [&](int j) {
    double* cj = loc + (size_t)(j / CL) * rows;
    double ss = 0.0;
    for (int i = j + 1 + tid; i < rows; i += blockDim.x) ss = fma(cj[i], cj[i], ss);
    ss = warp_sum(ss);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    double sig = lane < nw ? red[lane] : 0.0;  // the nw = 8 warp partials, by shuffles
    for (int o = 4; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
    sig = __shfl_sync(0xffffffffu, sig, 0);
    const double alpha = cj[j];
    double t = 0.0, beta = alpha, vinv = 0.0;
    if (sig != 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, sig));
      beta = (alpha <= 0.0) ? nrm : -nrm;
      t = (beta - alpha) / beta;
      vinv = 1.0 / (alpha - beta);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < rows; i += blockDim.x) cj[i] *= vinv;
    if (tid == 0) {
      cj[j] = beta;
      s_tau[j] = t;
    }
    __syncthreads();
  };
  // H_j = I - tau v v^T (v_j = 1, v in vbuf) applied to one local column by one warp;
  // the dot product runs as four independent chains (FP64 latency bounds it)
  auto apply_col = [&](double* col, int j, double tj) {
    double d0 = (lane == 0) ? col[j] : 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    int i = j + 1 + lane;
    for (; i + 96 < rows; i += 128) {
      d0 = fma(vbuf[i], col[i], d0);
      d1 = fma(vbuf[i + 32], col[i + 32], d1);
      d2 = fma(vbuf[i + 64], col[i + 64], d2);
      d3 = fma(vbuf[i + 96], col[i + 96], d3);
    }
    for (; i < rows; i += 32) d0 = fma(vbuf[i], col[i], d0);
    const double d = warp_sum((d0 + d1) + (d2 + d3)) * tj;
    if (lane == 0) col[j] -= d;
    for (int q = j + 1 + lane; q < rows; q += 32) col[q] = fma(-d, vbuf[q], col[q]);
  };
  // Columns below `start` were factored by an earlier call (v_j below the diagonal
  // of column j, tau_j in tau_out); columns start .. fresh-1 carry that call's
  // transformation already (its extra column). The old reflectors are applied, in
  // order, to my columns g >= fresh, each column on its own, with no cluster barrier
  // (the reflectors are fixed); the factorization then continues at column start.
  if (start > 0) {
    for (int j = tid; j < start; j += blockDim.x) s_tau[j] = tau_out[j];
    for (int j = 0; j < start && j < steps; ++j) {
      __syncthreads();  // vbuf is free
      const double* vj = A + (size_t)j * lda;
      for (int i = j + 1 + tid; i < rows; i += blockDim.x) vbuf[i] = vj[i];
      __syncthreads();
      const double tj = s_tau[j];
      int first = (fresh - r + CL - 1) / CL;  // first local column with g >= fresh
      if (first < 0) first = 0;
      for (int lc = first + warp; lc < nloc; lc += nw) apply_col(loc + (size_t)lc * rows, j, tj);
    }
    __syncthreads();
  }
  // Point-to-point publication instead of an all-CTA barrier per column: the owner
  // of reflector j sets s_flag[j] in every CTA (release at cluster scope) once column
  // j and tau_j are final (they are never written again), and each CTA waits for its
  // own flag (acquire; bounded, FAB_ETIMEOUT on expiry). The owner of column j+1
  // applies H_j to that column first and publishes reflector j+1 before updating its
  // other columns, so the next reflector's critical path is one column's update.
  auto publish = [&](int q) {
    __syncthreads();  // column q and tau_q are written
    if (tid == 0) {
      asm volatile("fence.acq_rel.cluster;" ::: "memory");
      for (int rk = 0; rk < CL; ++rk) {
        int* f = cluster.map_shared_rank(s_flag + q, rk);
        asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(f), "r"(1) : "memory");
      }
    }
  };
  for (int j = tid; j < kMaxM; j += blockDim.x) s_flag[j] = 0;
  if (tid == 0) s_fail = 0;
  cluster.sync();  // every CTA's flags are cleared before any publication
  if (start < steps && r == start % CL) {
    reflector(start);
    publish(start);
  }
  for (int j = start; j < steps; ++j) {
    const int owner = j % CL;
    if (tid == 0) {
      int ok = 0;
      for (int it = 0; it < (1 << 22) && !ok; ++it) {
        asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(ok) : "l"(s_flag + j) : "memory");
        if (!ok) __nanosleep(32);
      }
      if (!ok) {
        s_fail = 1;
        st->status = FAB_ETIMEOUT;
      }
    }
    __syncthreads();
    if (s_fail) break;
    {  // every thread's own acquire of the (set) flag orders its reads after the owner's release
      int f;
      asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(f) : "l"(s_flag + j) : "memory");
      (void)f;
    }
    const double* rcol = cluster.map_shared_rank(loc + (size_t)(j / CL) * rows, owner);
    const double* rtau = cluster.map_shared_rank(s_tau, owner);
    for (int i = j + 1 + tid; i < rows; i += blockDim.x) vbuf[i] = rcol[i];
    const double tj = rtau[j];
    if (r != owner && tid == 0) s_tau[j] = tj;
    __syncthreads();
    const int nxt = j + 1 < steps ? (j + 1) % CL : -1;
    if (r == nxt) {  // H_j on column j+1 by the whole CTA (all four FP64 pipes), then reflector j+1
      double* col = loc + (size_t)((j + 1) / CL) * rows;
      double d = (tid == 0) ? col[j] : 0.0;
      for (int i = j + 1 + tid; i < rows; i += blockDim.x) d = fma(vbuf[i], col[i], d);
      d = warp_sum(d);
      if (lane == 0) red[warp] = d;
      __syncthreads();
      double dd = lane < nw ? red[lane] : 0.0;
      for (int o = 4; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);  // nw = 8 partials
      dd = __shfl_sync(0xffffffffu, dd, 0) * tj;
      if (tid == 0) col[j] -= dd;
      for (int i = j + 1 + tid; i < rows; i += blockDim.x) col[i] = fma(-dd, vbuf[i], col[i]);
      __syncthreads();
      reflector(j + 1);
      publish(j + 1);
    }
    // apply H_j to my other columns g > j, one warp per column
    int first = (j + 1 - r + CL - 1) / CL;  // first local column with g > j
    if (first < 0) first = 0;
    for (int lc = first + warp; lc < nloc; lc += nw) {
      if (r == nxt && lc == (j + 1) / CL) continue;  // done above
      apply_col(loc + (size_t)lc * rows, j, tj);
    }
    __syncthreads();  // vbuf is reused
  }
  cluster.sync();  // no CTA exits while others may still read its shared memory
  for (int lc = 0; lc < nloc; ++lc) {
    double* dst = A + (size_t)(lc * CL + r) * lda;
    for (int i = tid; i < rows; i += blockDim.x) dst[i] = loc[(size_t)lc * rows + i];
  }
  if (r == 0)
    for (int j = tid; j < steps; j += blockDim.x) tau_out[j] = s_tau[j];
}

// LU with partial pivoting (ties to the smallest row), rows swapped across the
// whole matrix; piv[k] = row swapped with k; log|det| to *logdet.
template <int CL>
__global__ void __launch_bounds__(256) k_lu_cluster(double* __restrict__ M, int ld, const int* __restrict__ mdev,
                                                    int* __restrict__ piv, double* __restrict__ logdet,
                                                    DevState* st) {
  extern __shared__ __align__(16) double smem_d[];
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int s_piv[kMaxM];
  __shared__ double s_logdet;
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int mu = *mdev;
  const int nloc = (mu - r + CL - 1) / CL;
  double* loc = smem_d;
  double* lbuf = smem_d + (size_t)((mu + CL - 1) / CL) * mu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int lc = 0; lc < nloc; ++lc) {
    const double* src = M + (size_t)(lc * CL + r) * ld;
    for (int i = tid; i < mu; i += blockDim.x) loc[(size_t)lc * mu + i] = src[i];
  }
  if (tid == 0) s_logdet = 0.0;
  __syncthreads();
  for (int k = 0; k < mu; ++k) {
    const int owner = k % CL;
    if (r == owner) {
      double* ck = loc + (size_t)(k / CL) * mu;
      double best = -1.0;
      int bi = mu;
      for (int i = k + tid; i < mu; i += blockDim.x) {
        const double a = fabs(ck[i]);
        if (a > best) {
          best = a;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        rv[warp] = best;
        ri[warp] = bi;
      }
      __syncthreads();
      double b = -1.0;
      int p = mu;
      for (int w = 0; w < nw; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < p)) {
          b = rv[w];
          p = ri[w];
        }
      if (p < k || p >= mu) {  // only with non-finite entries
        p = k;
        if (tid == 0) st->status = FAB_ENUMERIC;
      }
      if (tid == 0) {
        const double t = ck[k];
        ck[k] = ck[p];
        ck[p] = t;
        s_piv[k] = p;
        const double pv = ck[k];
        if (pv == 0.0 || !isfinite(pv)) st->status = FAB_ENUMERIC;
      }
      __syncthreads();
      const double pv = ck[k];
      const double pinv = pv != 0.0 ? 1.0 / pv : 0.0;
      for (int i = k + 1 + tid; i < mu; i += blockDim.x) ck[i] *= pinv;
    }
    cluster.sync();  // pivot and multipliers of column k are published
    int p = *cluster.map_shared_rank(s_piv + k, owner);
    if (p < k || p >= mu) p = k;
    const double* rcol = cluster.map_shared_rank(loc + (size_t)(k / CL) * mu, owner);
    for (int i = k + 1 + tid; i < mu; i += blockDim.x) lbuf[i] = rcol[i];
    if (tid == 0) {
      if (r != owner) s_piv[k] = p;
      const double pv = rcol[k];  // U_kk (after the owner's swap)
      if (pv != 0.0 && isfinite(pv)) s_logdet += log(fabs(pv));
    }
    __syncthreads();
    for (int lc = warp; lc < nloc; lc += nw) {
      const int g = lc * CL + r;
      if (g == k) continue;
      double* col = loc + (size_t)lc * mu;
      if (lane == 0 && p != k) {
        const double t = col[k];
        col[k] = col[p];
        col[p] = t;
      }
      __syncwarp();
      if (g > k) {
        const double ukj = col[k];
        for (int i = k + 1 + lane; i < mu; i += 32) col[i] = fma(-lbuf[i], ukj, col[i]);
      }
      __syncwarp();
    }
    __syncthreads();
  }
  cluster.sync();
  for (int lc = 0; lc < nloc; ++lc) {
    double* dst = M + (size_t)(lc * CL + r) * ld;
    for (int i = tid; i < mu; i += blockDim.x) dst[i] = loc[(size_t)lc * mu + i];
  }
  if (r == 0) {
    for (int k = tid; k < mu; k += blockDim.x) piv[k] = s_piv[k];
    if (tid == 0 && logdet) *logdet = s_logdet;
  }
}

// ------------------------------------------------ Alg. 1: sketched Gram-Schmidt
// Step c of Alg. 1 on the sketches (one block). SV holds S_0..S_{c-1} (orthonormal
// columns) and, in column c, p = Theta w_c. Computes r = S^T p, s = p - S r,
// r_cc = ||s|| (one classical Gram-Schmidt pass), stores s / r_cc as S_c, the
// column c-1 of H (h_{j,c-1} = r_j, h_{c,c-1} = r_cc), and for the raw basis
// (v_j = sigma_j W_j, A v_{c-1} = scl[c] W_c) the update coefficients
// coef_j = r_j sigma_j / scl[c] of W_c <- W_c - sum_j coef_j W_j and
// sigma_c = scl[c] / r_cc. c = 0 (the start vector, p = Theta b): r_00 = ||p||,
// sigma_0 = 1 / r_00 and gamma_b = r_00 into st->beta. Breakdown: r_cc <= 1e-12 ||p||
// (the sketch is exact to 2^-49 of a chunk's largest entry) ends the basis with m_used = c.
__global__ __launch_bounds__(256) void k_bg_orth(double* __restrict__ SV, int lds, int c, double* __restrict__ H,
                                                 int ldh, double* __restrict__ coef, ColScale cs, DevState* st,
                                                 const double* __restrict__ Ri, int ldr, int gate) {
  __shared__ double s_r[kMaxM + 1];
  __shared__ double red[2][32];
  if (st->stop || gate_closed(st, c, gate)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double* p = SV + (size_t)lds * c;
  for (int j = warp; j < c; j += nw) {  // r_j = <S_j, p>
    const double* sj = SV + (size_t)lds * j;
    double a = 0.0;
    for (int q = lane; q < lds; q += 32) a = fma(sj[q], p[q], a);
    a = warp_sum(a);
    if (lane == 0) s_r[j] = a;
  }
  __syncthreads();
  double ss = 0.0, pp = 0.0;
  for (int q = tid; q < lds; q += blockDim.x) {
    const double pq = p[q];
    double v = pq;
    for (int j = 0; j < c; ++j) v = fma(-SV[q + (size_t)lds * j], s_r[j], v);
    p[q] = v;  // s (normalised below)
    ss = fma(v, v, ss);
    pp = fma(pq, pq, pp);
  }
  ss = warp_sum(ss);
  pp = warp_sum(pp);
  if (lane == 0) {
    red[0][warp] = ss;
    red[1][warp] = pp;
  }
  __syncthreads();
  __shared__ double s_rcc, s_ok;
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    const double rcc = sqrt(a), pn = sqrt(b);
    s_rcc = rcc;
    s_ok = 1.0;
    if (!isfinite(rcc)) {
      st->status = FAB_ENUMERIC;
      st->stop = 1;
      s_ok = 0.0;
    } else if (c == 0) {
      st->beta = rcc;  // gamma_b = r_11
      if (rcc == 0.0) {
        st->m_used = 0;
        st->stop = 1;
        cs.sigma[0] = 0.0;
        cs.shf[0] = 0;
        s_ok = 0.0;
      } else {
        cs.sigma[0] = 1.0 / rcc;
        cs.shf[0] = exponent_of(cs.sigma[0]);
      }
    } else {
      H[c + (size_t)ldh * (c - 1)] = rcc;
      if (!(rcc > 1e-12 * pn)) {  // far above the int64 sketch's rounding, far below a new direction
        st->m_used = c;  // the basis spans an invariant subspace
        st->stop = 1;
        cs.sigma[c] = 0.0;
        cs.shf[c] = 0;
        s_ok = 0.0;
      } else {
        cs.sigma[c] = cs.scl[c] / rcc;
        cs.shf[c] = exponent_of(cs.sigma[c]);
      }
    }
  }
  __syncthreads();
  // column c-1 of H holds A v_{c-1} = sum_j r_j v_j + r_cc v_c, also at a breakdown
  // (then A V_c = V_c H_c spans an invariant subspace)
  for (int j = tid; j < c; j += blockDim.x) H[j + (size_t)ldh * (c - 1)] = s_r[j];
  if (s_ok == 0.0) return;
  const double inv = 1.0 / s_rcc;
  for (int q = tid; q < lds; q += blockDim.x) p[q] *= inv;
  if (c > 0) {
    // After whitening at wh columns (FAB_WHITEN) the whitened vectors 0..wh-2 are
    // V R_{wh-1}^{-1} of the stored Alg. 2 columns: the coefficient of stored
    // column j < wh-1 is (R_{wh-1}^{-1} r)_j.
    const int wh = Ri ? st->wh : 0;
    const int nt = wh > 1 ? (wh - 1 < c ? wh - 1 : c) : 0;
    const double tau = cs.scl[c];
    for (int j = tid; j < c; j += blockDim.x) {
      double r = s_r[j];
      if (j < nt) {
        r = 0.0;
        for (int l = j; l < nt; ++l) r = fma(Ri[j + (size_t)ldr * l], s_r[l], r);
      }
      coef[j] = r * cs.sigma[j] / tau;
    }
  }
}

cudaError_t launch_bg_orth(double* SV, int lds, int c, double* H, int ldh, double* coef, ColScale cs, DevState* st,
                           cudaStream_t s, const double* Ri, int ldr, int gate) {
  if (c > kMaxM) return cudaErrorInvalidValue;
  k_bg_orth<<<1, 256, 0, s>>>(SV, lds, c, H, ldh, coef, cs, st, Ri, ldr, gate);
  return cudaGetLastError();
}

// ------------------------------------------------ whitening (FAB_WHITEN)
// Step c of Alg. 2 with whitening (§2.1.2), on one CTA, after column c and its
// sketch y = Theta v_c (SV column c) exist. The thin QR Theta V_{c+1} = Q R grows
// by one column (classical Gram-Schmidt applied twice against Q's columns; R
// column c = the summed projections and rho = ||y - Q r||), R^{-1} by one column
// (-R_c^{-1} r / rho and 1 / rho), and ||R||_1, ||R^{-1}||_1 (max column sums;
// appending a column leaves the others unchanged) are kept in nrm[0..1], so
// kappa_1(R_{c+1}) is exact. rho <= 1e-12 ||y|| stops the basis at c columns.
// At the first kappa_1 > kmax the basis is whitened at wh = c+1 columns:
//   H_{c} (rows 0..c, columns 0..c-1) <- R_{c+1} H_c R_c^{-1},
//   SV columns 0..c <- Q,  gamma_b <- ||b|| r_00,
//   wcoef[q] = (R^{-1})_{q,c} sigma_q (the explicit whitened column c, written by
//   launch_whiten_column), sigma_c <- 1 and shf_c <- 0 (it is stored at unit scale),
// while columns 0..c-1 stay stored as Alg. 2 vectors with R_c^{-1} applied
// implicitly (k_bg_orth, k_wh_coef). Scratch T holds (c+1) x c values.
__global__ __launch_bounds__(256) void k_wh_check(double* __restrict__ SV, int lds, int c, double* __restrict__ Q,
                                                  double* __restrict__ R, double* __restrict__ Ri,
                                                  double* __restrict__ T, int ldr, double* __restrict__ H, int ldh,
                                                  double kmax, double* __restrict__ wcoef, double* __restrict__ nrm,
                                                  ColScale cs, DevState* st) {
  __shared__ double s_r[kMaxM + 1];
  __shared__ double s_t[kMaxM + 1];
  __shared__ double red[2][32];
  __shared__ double s_rho;
  __shared__ int s_go;
  if (st->stop || *(volatile int*)&st->wh != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, bd = blockDim.x;
  const double* y = SV + (size_t)lds * c;
  double* q = Q + (size_t)lds * c;
  double yy = 0.0;
  for (int i = tid; i < lds; i += bd) {
    q[i] = y[i];
    yy = fma(y[i], y[i], yy);
  }
  for (int j = tid; j < c; j += bd) s_r[j] = 0.0;
  __syncthreads();
  for (int pass = 0; pass < 2 && c > 0; ++pass) {
    for (int j = warp; j < c; j += nw) {
      const double* qj = Q + (size_t)lds * j;
      double a = 0.0;
      for (int i = lane; i < lds; i += 32) a = fma(qj[i], q[i], a);
      a = warp_sum(a);
      if (lane == 0) s_t[j] = a;
    }
    __syncthreads();
    for (int i = tid; i < lds; i += bd) {
      double v = q[i];
      for (int j = 0; j < c; ++j) v = fma(-Q[i + (size_t)lds * j], s_t[j], v);
      q[i] = v;
    }
    for (int j = tid; j < c; j += bd) s_r[j] += s_t[j];
    __syncthreads();
  }
  double qq = 0.0;
  for (int i = tid; i < lds; i += bd) qq = fma(q[i], q[i], qq);
  qq = warp_sum(qq);
  yy = warp_sum(yy);
  if (lane == 0) {
    red[0][warp] = qq;
    red[1][warp] = yy;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    const double rho = sqrt(a), yn = sqrt(b);
    s_rho = rho;
    s_go = 1;
    if (!isfinite(rho) || (c == 0 && !(rho > 0.0))) {
      st->status = FAB_ENUMERIC;
      st->stop = 1;
      s_go = 0;
    } else if (!(rho > 1e-12 * yn)) {  // the sketch of v_c lies in the span of the others
      st->m_used = c;
      st->stop = 1;
      s_go = 0;
    }
  }
  __syncthreads();
  if (!s_go) return;
  const double rho = s_rho, inv = 1.0 / rho;
  for (int i = tid; i < lds; i += bd) q[i] *= inv;
  double cr = 0.0, cz = 0.0;
  for (int j = tid; j < c; j += bd) {
    double a = 0.0;
    for (int l = j; l < c; ++l) a = fma(Ri[j + (size_t)ldr * l], s_r[l], a);
    const double z = -a * inv;
    Ri[j + (size_t)ldr * c] = z;
    R[j + (size_t)ldr * c] = s_r[j];
    cz += fabs(z);
    cr += fabs(s_r[j]);
  }
  cr = warp_sum(cr);
  cz = warp_sum(cz);
  __syncthreads();  // red[] is reused
  if (lane == 0) {
    red[0][warp] = cr;
    red[1][warp] = cz;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    R[c + (size_t)ldr * c] = rho;
    Ri[c + (size_t)ldr * c] = inv;
    const double n1 = c == 0 ? rho : fmax(nrm[0], a + rho);
    const double n2 = c == 0 ? inv : fmax(nrm[1], b + inv);
    nrm[0] = n1;
    nrm[1] = n2;
    nrm[2] = n1 * n2;
    s_go = (c > 0 && n1 * n2 > kmax) ? 1 : 0;
  }
  __syncthreads();
  if (!s_go) return;
  // whiten at c+1 columns: T = H_c R_c^{-1}, then H_c <- R_{c+1} T (H upper Hessenberg)
  const int rows = c + 1;
  for (int idx = tid; idx < rows * c; idx += bd) {
    const int j = idx % rows, l = idx / rows;
    double a = 0.0;
    for (int k = (j > 0 ? j - 1 : 0); k <= l; ++k) a = fma(H[j + (size_t)ldh * k], Ri[k + (size_t)ldr * l], a);
    T[j + (size_t)ldr * l] = a;
  }
  __syncthreads();
  for (int idx = tid; idx < rows * c; idx += bd) {
    const int j = idx % rows, l = idx / rows;
    double a = 0.0;
    for (int k = j; k <= c; ++k) a = fma(R[j + (size_t)ldr * k], T[k + (size_t)ldr * l], a);
    H[j + (size_t)ldh * l] = a;
  }
  for (int idx = tid; idx < lds * rows; idx += bd) SV[idx] = Q[idx];
  for (int k = tid; k <= c; k += bd) wcoef[k] = Ri[k + (size_t)ldr * c] * cs.sigma[k];
  __syncthreads();
  if (tid == 0) {
    st->beta *= R[0];
    cs.sigma[c] = 1.0;
    cs.shf[c] = 0;
    st->wh = c + 1;
  }
}

cudaError_t launch_wh_check(double* SV, int lds, int c, double* Q, double* R, double* Ri, double* T, int ldr,
                            double* H, int ldh, double kmax, double* wcoef, double* nrm, ColScale cs, DevState* st,
                            cudaStream_t s) {
  if (c < 0 || c > kMaxM) return cudaErrorInvalidValue;
  k_wh_check<<<1, 256, 0, s>>>(SV, lds, c, Q, R, Ri, T, ldr, H, ldh, kmax, wcoef, nrm, cs, st);
  return cudaGetLastError();
}

// Preconditioner of Alg. 3's LSQR on a basis whitened at wh columns: the stored
// columns are V' with V_whitened = V' blockdiag(R_{wh-1}^{-1}, I), so LSQR on
// V' P^{-1} with P = blockdiag(R_{wh-1}, I) (rows x mu, ld rows) works on the
// whitened basis and returns y in its coordinates.
__global__ void k_wh_precond(const double* __restrict__ R, int ldr, int wh, double* __restrict__ P, int rows,
                             const int* __restrict__ mdev) {
  const int mu = *mdev;
  const int nt = wh - 1 < mu ? wh - 1 : mu;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * mu; idx += gridDim.x * blockDim.x) {
    const int i = idx % rows, j = idx / rows;
    double v = (i == j) ? 1.0 : 0.0;
    if (j < nt && i <= j) v = R[i + (size_t)ldr * j];
    P[idx] = v;
  }
}

cudaError_t launch_wh_precond(const double* R, int ldr, int wh, double* P, int rows, const int* mdev, int mmax,
                              cudaStream_t s) {
  int grid = (rows * mmax + 255) / 256;
  grid = grid < 1 ? 1 : (grid > 1024 ? 1024 : grid);
  k_wh_precond<<<grid, 256, 0, s>>>(R, ldr, wh, P, rows, mdev);
  return cudaGetLastError();
}

// c <- blockdiag(R_{wh-1}^{-1}, I) c (whitened coordinates to stored columns).
__global__ __launch_bounds__(256) void k_wh_coef(const double* __restrict__ Ri, int ldr, int wh,
                                                 const int* __restrict__ mdev, double* __restrict__ cv) {
  __shared__ double s_c[kMaxM + 1];
  const int mu = *mdev;
  const int nt = wh - 1 < mu ? wh - 1 : mu;
  for (int j = threadIdx.x; j < mu; j += blockDim.x) s_c[j] = cv[j];
  __syncthreads();
  for (int j = threadIdx.x; j < nt; j += blockDim.x) {
    double a = 0.0;
    for (int l = j; l < nt; ++l) a = fma(Ri[j + (size_t)ldr * l], s_c[l], a);
    cv[j] = a;
  }
}

cudaError_t launch_wh_coef(const double* Ri, int ldr, int wh, const int* mdev, double* cv, cudaStream_t s) {
  k_wh_coef<<<1, 256, 0, s>>>(Ri, ldr, wh, mdev, cv);
  return cudaGetLastError();
}

// R = I in the leading mu x mu block of a rows x mu column-major matrix (ld rows):
// LSQR on V_m itself for Alg. 3 (the Alg. 1 basis needs no preconditioner).
__global__ void k_set_identity(double* __restrict__ R, int rows, const int* __restrict__ mdev) {
  const int mu = *mdev;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * mu; idx += gridDim.x * blockDim.x) {
    const int i = idx % rows, j = idx / rows;
    R[idx] = (i == j) ? 1.0 : 0.0;
  }
}

cudaError_t launch_set_identity(double* R, int rows, const int* mdev, int mmax, cudaStream_t s) {
  int grid = (rows * mmax + 255) / 256;
  grid = grid < 1 ? 1 : (grid > 1024 ? 1024 : grid);
  k_set_identity<<<grid, 256, 0, s>>>(R, rows, mdev);
  return cudaGetLastError();
}

// ------------------------------------------------ sketched solution change
// With Theta v_j in the columns of SV (s x (m+1), ld lds): out[0] = || SV c_new -
// SV c_old || (c_old zero past m_old) and out[1] = || SV c_new ||, c_new of length
// *mdev. The sketch embeds x_new - x_old and x_new (§2.1.1), so out[0] / out[1]
// estimates their relative distance.
__global__ void k_sketch_change(const double* __restrict__ SV, int lds, const int* __restrict__ mdev,
                                const double* __restrict__ c_new, int m_old, const double* __restrict__ c_old,
                                double* __restrict__ out) {
  __shared__ double red[2][32];
  const int mu = *mdev;
  double dd = 0.0, aa = 0.0;
  for (int q = threadIdx.x; q < lds; q += blockDim.x) {
    double a = 0.0, o = 0.0;
    for (int j = 0; j < mu; ++j) a = fma(SV[q + (size_t)lds * j], c_new[j], a);
    for (int j = 0; j < m_old && j < mu; ++j) o = fma(SV[q + (size_t)lds * j], c_old[j], o);
    const double d = a - o;
    dd = fma(d, d, dd);
    aa = fma(a, a, aa);
  }
  dd = warp_sum(dd);
  aa = warp_sum(aa);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = dd;
    red[1][threadIdx.x >> 5] = aa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      x += red[0][w];
      y += red[1][w];
    }
    out[0] = sqrt(x);
    out[1] = sqrt(y);
  }
}

cudaError_t launch_sketch_change(const double* SV, int lds, const int* mdev, const double* c_new, int m_old,
                                 const double* c_old, double* out, cudaStream_t s) {
  k_sketch_change<<<1, 256, 0, s>>>(SV, lds, mdev, c_new, m_old, c_old, out);
  return cudaGetLastError();
}

// ------------------------------------------------- fused small stage (batch)
// The steps of the small stage, each done by the whole CTA, with the same
// per-element arithmetic as the multi-kernel path: products and linear
// combinations of m x m matrices, LU solves one warp per right-hand side.
__device__ void blk_gemm(double* __restrict__ C, const double* __restrict__ A, const double* __restrict__ B, int ld,
                         int mu) {
  for (int idx = threadIdx.x; idx < mu * mu; idx += blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    double a0 = 0.0, a1 = 0.0;
    int l = 0;
    for (; l + 1 < mu; l += 2) {
      a0 = fma(A[i + (size_t)ld * l], B[l + (size_t)ld * j], a0);
      a1 = fma(A[i + (size_t)ld * (l + 1)], B[l + 1 + (size_t)ld * j], a1);
    }
    if (l < mu) a0 = fma(A[i + (size_t)ld * l], B[l + (size_t)ld * j], a0);
    C[i + (size_t)ld * j] = a0 + a1;
  }
  __syncthreads();
}

__device__ void blk_lincomb(double* out, const double* X0, const double* X1, const double* X2, const double* X3,
                            double a0, double a1, double a2, double a3, double d, int ld, int mu) {
  for (int idx = threadIdx.x; idx < mu * mu; idx += blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    const size_t o = i + (size_t)ld * j;
    double v = (i == j) ? d : 0.0;
    if (X0) v = fma(a0, X0[o], v);
    if (X1) v = fma(a1, X1[o], v);
    if (X2) v = fma(a2, X2[o], v);
    if (X3) v = fma(a3, X3[o], v);
    out[o] = v;
  }
  __syncthreads();
}

// LU X = P B for all mu columns of B (identity_rhs: B = I); sb holds one mu-vector per warp.
__device__ void blk_lu_solve(const double* __restrict__ LU, int ld, const int* __restrict__ piv, int mu,
                             double* __restrict__ B, int ldb, int identity_rhs, double* sb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* b = sb + (size_t)warp * mu;
  for (int col = warp; col < mu; col += nw) {
    double* bg = B + (size_t)ldb * col;
    for (int i = lane; i < mu; i += 32) b[i] = identity_rhs ? (i == col ? 1.0 : 0.0) : bg[i];
    __syncwarp();
    if (lane == 0) {
      for (int k = 0; k < mu; ++k) {
        const int p = piv[k];
        if (p != k && p > k && p < mu) {
          const double t = b[k];
          b[k] = b[p];
          b[p] = t;
        }
      }
    }
    __syncwarp();
    for (int k = 0; k < mu; ++k) {
      const double bk = b[k];
      for (int i = k + 1 + lane; i < mu; i += 32) b[i] = fma(-LU[i + (size_t)ld * k], bk, b[i]);
      __syncwarp();
    }
    for (int k = mu - 1; k >= 0; --k) {
      if (lane == 0) b[k] /= LU[k + (size_t)ld * k];
      __syncwarp();
      const double bk = b[k];
      for (int i = lane; i < k; i += 32) b[i] = fma(-LU[i + (size_t)ld * k], bk, b[i]);
      __syncwarp();
    }
    for (int i = lane; i < mu; i += 32) bg[i] = b[i];
    __syncwarp();
  }
  __syncthreads();
}

// exp(M) e_1 by Pade [13/13] scaling and squaring (Higham 2005); M (ld m) is overwritten.
__device__ void blk_expm_e1(double* mats, int m, int mu, const PadeCoef& pd, double* c, int* piv, double* logdet,
                            double* sb, DevState* st) {
  const size_t mm = (size_t)m * m;
  double *M = mats, *A2 = mats + mm, *A4 = mats + 2 * mm, *A6 = mats + 3 * mm, *T = mats + 4 * mm,
         *U = mats + 5 * mm, *V = mats + 6 * mm, *X = mats + 7 * mm, *X2 = mats + 8 * mm;
  const double* b = pd.b;
  const double nrm = norm1_body(M, m, mu, nullptr);
  if (!isfinite(nrm)) {
    if (threadIdx.x == 0) st->status = FAB_ENUMERIC;
    return;
  }
  int sq = 0;
  if (nrm > pd.theta) sq = (int)ceil(log2(nrm / pd.theta));
  if (sq > 0) blk_lincomb(M, M, nullptr, nullptr, nullptr, ldexp(1.0, -sq), 0, 0, 0, 0.0, m, mu);
  blk_gemm(A2, M, M, m, mu);
  blk_gemm(A4, A2, A2, m, mu);
  blk_gemm(A6, A4, A2, m, mu);
  blk_lincomb(T, A6, A4, A2, nullptr, b[13], b[11], b[9], 0, 0.0, m, mu);
  blk_gemm(X, A6, T, m, mu);
  blk_lincomb(X, X, A6, A4, A2, 1.0, b[7], b[5], b[3], b[1], m, mu);
  blk_gemm(U, M, X, m, mu);
  blk_lincomb(T, A6, A4, A2, nullptr, b[12], b[10], b[8], 0, 0.0, m, mu);
  blk_gemm(V, A6, T, m, mu);
  blk_lincomb(V, V, A6, A4, A2, 1.0, b[6], b[4], b[2], b[0], m, mu);
  blk_lincomb(T, V, U, nullptr, nullptr, 1.0, -1.0, 0, 0, 0.0, m, mu);
  blk_lincomb(X, V, U, nullptr, nullptr, 1.0, 1.0, 0, 0, 0.0, m, mu);
  lu_body(T, m, mu, piv, logdet, st);
  blk_lu_solve(T, m, piv, mu, X, m, 0, sb);
  for (int i = 0; i < sq; ++i) {
    blk_gemm(X2, X, X, m, mu);
    double* t = X;
    X = X2;
    X2 = t;
  }
  for (int i = threadIdx.x; i < mu; i += blockDim.x) c[i] = X[i];
  if (threadIdx.x == 0) st->iters = sq;
  __syncthreads();
}

// f(M) e_1 for f = sqrt or inverse sqrt by the scaled product-form Denman-Beavers
// iteration with the stopping rule of the multi-kernel path.
__device__ void blk_sqrtm_e1(double* mats, int m, int mu, int want_sqrt, double* c, int* piv, double* logdet,
                             double* sb, DevState* st) {
  const size_t mm = (size_t)m * m;
  double *M = mats, *T = mats + mm, *Minv = mats + 2 * mm;
  for (int i = threadIdx.x; i < mu; i += blockDim.x) c[i] = want_sqrt ? M[i] : (i == 0 ? 1.0 : 0.0);
  __syncthreads();
  double err = INFINITY;
  int extra = -1;
  for (int it = 0; it < 100; ++it) {
    for (int idx = threadIdx.x; idx < (int)mm; idx += blockDim.x) T[idx] = M[idx];
    __syncthreads();
    lu_body(T, m, mu, piv, logdet, st);
    blk_lu_solve(T, m, piv, mu, Minv, m, 1, sb);
    db_update_body(M, Minv, m, mu, c, logdet, err > 1e-2 ? 1 : 0, st);
    if (st->status != FAB_OK) return;
    err = st->scal[1];
    if (threadIdx.x == 0) st->iters = it + 1;
    if (extra >= 0) return;
    if (err <= 1e-13 * sqrt((double)m)) extra = 0;
    __syncthreads();
  }
  if (threadIdx.x == 0) st->status = FAB_ENOTCONV;
}

__global__ __launch_bounds__(256) void k_small_fused(const SmallJob* __restrict__ jobs, const int* __restrict__ ids,
                                                     PadeCoef pd) {
  extern __shared__ double s_lu[];  // one mu-vector per warp
  const SmallJob J = jobs[ids ? ids[blockIdx.x] : blockIdx.x];
  DevState* st = J.st;
  if (st->status != FAB_OK) return;
  const int mu = st->m_used, m = J.m;
  if (threadIdx.x == 0) st->scal[15] = (mu == m) ? J.H[m + (size_t)J.ldh * (m - 1)] : 0.0;  // h_{m+1,m}
  if (mu == 0) {  // b = 0
    for (int j = threadIdx.x; j <= m; j += blockDim.x) J.coef[j] = 0.0;
    return;
  }
  const double* yptr = nullptr;
  if (mu == m && J.method == FAB_SKETCHED_FAST) {
    // y = argmin || Theta V_m z - Theta v_{m+1} || (sketch-and-solve form of eq. sFOM)
    const size_t cnt = (size_t)J.s * (mu + 1);
    for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) J.qr[i] = J.SV[i];
    __syncthreads();
    householder_qr_body(J.qr, J.s, J.s, mu, 1, J.tau);
    __syncthreads();
    trsv_body(J.qr, J.s, mu, J.qr + (size_t)mu * J.s, J.y, 0, nullptr);
    __syncthreads();
    yptr = J.y;
  }
  // M = scale (H_mu + h_{mu+1,mu} y e_mu^T)
  const double scale = (J.f == FAB_F_EXP) ? J.t : 1.0;
  const double hl = yptr ? J.H[mu + (size_t)J.ldh * (mu - 1)] : 0.0;
  for (int idx = threadIdx.x; idx < mu * mu; idx += blockDim.x) {
    const int i = idx % mu, j = idx / mu;
    double v = J.H[i + (size_t)J.ldh * j];
    if (yptr && j == mu - 1) v = fma(hl, yptr[i], v);
    J.mats[i + (size_t)m * j] = scale * v;
  }
  __syncthreads();
  if (J.f == FAB_F_EXP)
    blk_expm_e1(J.mats, m, mu, pd, J.cvec, J.piv, J.scal + 11, s_lu, st);
  else
    blk_sqrtm_e1(J.mats, m, mu, J.f == FAB_F_SQRT, J.cvec, J.piv, J.scal + 11, s_lu, st);
  __syncthreads();
  if (st->status != FAB_OK) return;
  const double beta = st->beta;
  for (int j = threadIdx.x; j < mu; j += blockDim.x) J.coef[j] = beta * J.cvec[j] * J.sigma[j];
}

cudaError_t small_fused_prepare(int mmax) {
  return ensure_smem_limit((const void*)k_small_fused, (size_t)(256 / 32) * (mmax > 0 ? mmax : 1) * sizeof(double));
}

cudaError_t launch_small_fused(const SmallJob* jobs, const int* ids, int count, int mmax, const PadeCoef& pd,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = (size_t)(256 / 32) * (mmax > 0 ? mmax : 1) * sizeof(double);
  cudaError_t e = ensure_smem_limit((const void*)k_small_fused, smem);
  if (e != cudaSuccess) return e;
  k_small_fused<<<count, 256, smem, s>>>(jobs, ids, pd);
  return cudaGetLastError();
}

namespace {
template <typename K>
cudaError_t launch_cluster(K kernel, int cl, size_t smem, cudaStream_t s, void** args) {
  cudaError_t e = ensure_smem_limit((const void*)kernel, smem);
  if (e != cudaSuccess) return e;
  if (cl > 8) cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
}
}  // namespace

// Cluster QR when the matrix fits the cluster's shared memory, else the one-block kernel.
bool qr_cluster_fits(int rows, int ncols) {
  for (int cl : {16, 8})
    if (((size_t)((ncols + cl - 1) / cl) + 1) * rows * sizeof(double) <= 200 * 1024) return true;
  return false;
}

cudaError_t launch_qr(double* A, int lda, int rows, const int* mdev, int max_cols, int extra, double* tau,
                      DevState* st, cudaStream_t s, int start, int fresh) {
  const int ncols = max_cols + extra;
  for (int cl : {16, 8}) {
    const size_t smem = ((size_t)((ncols + cl - 1) / cl) + 1) * rows * sizeof(double);
    if (smem > 200 * 1024) continue;
    void* args[] = {&A, &lda, &rows, (void*)&mdev, &extra, &tau, &start, &fresh, &st};
    cudaError_t e = cl == 16 ? launch_cluster(k_qr_cluster<16>, 16, smem, s, args)
                             : launch_cluster(k_qr_cluster<8>, 8, smem, s, args);
    if (e == cudaSuccess) return e;
    cudaGetLastError();
  }
  if (start > 0) return cudaErrorNotSupported;  // the one-CTA fallback starts at column 0
  return launch_householder_qr(A, lda, rows, mdev, extra, tau, s);
}

// Condition estimate of the sketched basis (paper §2.1.2: kappa(Theta V_m) tracks
// kappa(V_m) within the embedding's distortion): max_i |r_ii| / min_i |r_ii| over the
// first min(m_used, ncols) columns of R in the upper triangle of the QR buffer. It is
// a lower bound on kappa_2(R) = kappa_2(Theta V_m) (each |r_ii| lies between the
// smallest and the largest singular value of R). Infinite if some r_ii is zero.
__global__ void k_kappa_diag(const double* __restrict__ R, int lda, const int* __restrict__ mdev, int ncols,
                             DevState* st) {
  __shared__ double s_mx[32], s_mn[32];
  const int nc = min(*mdev, ncols);
  double mx = 0.0, mn = INFINITY;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const double d = fabs(R[i + (size_t)i * lda]);
    mx = fmax(mx, d);
    mn = fmin(mn, d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_mx[threadIdx.x >> 5] = mx;
    s_mn[threadIdx.x >> 5] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mx = fmax(mx, s_mx[w]);
      mn = fmin(mn, s_mn[w]);
    }
    st->kappa = nc < 1 ? 0.0 : (mn > 0.0 ? mx / mn : INFINITY);
  }
}

cudaError_t launch_kappa_diag(const double* R, int lda, const int* mdev, int ncols, DevState* st, cudaStream_t s) {
  k_kappa_diag<<<1, 256, 0, s>>>(R, lda, mdev, ncols, st);
  return cudaGetLastError();
}

// Blocked LU with partial pivoting over a cluster of CL CTAs (ties to the smallest
// row; rows swapped across the whole matrix, as k_lu_cluster; piv[k] = row swapped
// with k; log|det| to *logdet). Panels of kLuB columns are owned cyclically (panel P
// by CTA P % CL, its columns in that CTA's shared memory). Panel P is factored by its
// owner alone (CTA barriers only) and copied to the owner's publish buffer; after one
// cluster barrier every CTA copies it and, on each of its columns, applies the
// panel's row swaps, then (right of the panel) the unit-lower triangular solve for
// the U block and the rank-kLuB update of the rows below. A publish buffer is written
// again only for the owner's next panel, CL panels later, after every CTA has passed
// the barriers of the panels in between (and so has copied it): one cluster barrier
// per panel, and the factorization of panel P+1 overlaps the other CTAs' updates.
constexpr int kLuB = 8;
template <int CL>
__global__ void __launch_bounds__(256) k_lu_blocked(double* __restrict__ M, int ld, const int* __restrict__ mdev,
                                                    int* __restrict__ piv, double* __restrict__ logdet,
                                                    DevState* st) {
  extern __shared__ __align__(16) double smem_d[];
  __shared__ double rv[32];
  __shared__ unsigned long long rk[32];
  __shared__ int ri[32];
  __shared__ int s_pp[kLuB];
  __shared__ int s_piv[kMaxM];
  __shared__ double s_ld;  // this CTA's sum of log|U_jj| over its panels (panel order)
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int mu = *mdev;
  const int np = (mu + kLuB - 1) / kLuB;
  const int maxp = (np + CL - 1) / CL;
  const int myp = r < np ? (np - 1 - r) / CL + 1 : 0;  // panels r, r + CL, ...
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double* loc = smem_d;                                  // my panels: column (lp, jj) at loc + (lp kLuB + jj) mu
  double* pub = loc + (size_t)maxp * kLuB * mu;          // published panel, kLuB x mu
  int* pub_piv = reinterpret_cast<int*>(pub + (size_t)kLuB * mu);  // kLuB ints
  double* cur = pub + (size_t)kLuB * mu + kLuB;          // copy of the panel being applied
  for (int lp = 0; lp < myp; ++lp)
    for (int jj = 0; jj < kLuB; ++jj) {
      const int g = (lp * CL + r) * kLuB + jj;
      if (g >= mu) break;
      double* dst = loc + (size_t)(lp * kLuB + jj) * mu;
      const double* src = M + (size_t)g * ld;
      for (int i = tid; i < mu; i += blockDim.x) dst[i] = src[i];
    }
  if (tid == 0) s_ld = 0.0;
  __syncthreads();
  // factors panel Q in this (its owner's) CTA and copies it to the publish buffer
  auto factor = [&](int Q) {
    const int lpq = Q / CL, q0 = Q * kLuB;
    const int wq = mu - q0 < kLuB ? mu - q0 : kLuB;
    double* pc = loc + (size_t)lpq * kLuB * mu;
    for (int jj = 0; jj < wq; ++jj) {
      const int j = q0 + jj;
      double* cj = pc + (size_t)jj * mu;
      // largest |a| (ties to the smallest row) compared on the bit patterns: for
      // non-negative doubles the unsigned order of the bits is the order of the
      // values, and the integer pipe has none of the FP64 latency; NaNs are skipped
      unsigned long long best = 0;
      int bi = mu;
      for (int i = j + tid; i < mu; i += blockDim.x) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(cj[i]) & 0x7FFFFFFFFFFFFFFFull;
        if (key <= 0x7FF0000000000000ull && (key > best || bi == mu)) {
          best = key;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        rk[warp] = best;
        ri[warp] = bi;
      }
      __syncthreads();
      unsigned long long bb = 0;
      int p = mu;
      for (int w = 0; w < nw; ++w)
        if (rk[w] > bb || (rk[w] == bb && ri[w] < p)) {
          bb = rk[w];
          p = ri[w];
        }
      if (p < j || p >= mu) {  // only with non-finite entries
        p = j;
        if (tid == 0) st->status = FAB_ENUMERIC;
      }
      if (tid < wq && p != j) {  // the panel's rows j and p
        double* c2 = pc + (size_t)tid * mu;
        const double t = c2[j];
        c2[j] = c2[p];
        c2[p] = t;
      }
      if (tid == 0) s_piv[j] = p;
      __syncthreads();
      const double pv = cj[j];
      if (tid == 0 && (pv == 0.0 || !isfinite(pv))) st->status = FAB_ENUMERIC;
      const double pinv = pv != 0.0 ? 1.0 / pv : 0.0;  // log|pv| is summed after the factorization
      for (int i = j + 1 + tid; i < mu; i += blockDim.x) cj[i] *= pinv;
      __syncthreads();
      for (int j2 = jj + 1 + warp; j2 < wq; j2 += nw) {
        double* c2 = pc + (size_t)j2 * mu;
        const double u = c2[j];
        for (int i = j + 1 + lane; i < mu; i += 32) c2[i] = fma(-cj[i], u, c2[i]);
      }
      __syncthreads();
    }
    for (int idx = tid; idx < wq * mu; idx += blockDim.x) pub[idx] = pc[idx];
    if (tid < wq) pub_piv[tid] = s_piv[q0 + tid];
    __syncthreads();
  };
  // applies the panel in cur (columns c0.., width wP, pivots s_pp) to my local column lc
  auto apply = [&](int lc, int c0, int wP) {
    const int g = ((lc / kLuB) * CL + r) * kLuB + lc % kLuB;
    double* col = loc + (size_t)lc * mu;
    if (lane == 0)
      for (int t = 0; t < wP; ++t) {
        const int pr = s_pp[t], jr = c0 + t;
        if (pr != jr && pr > jr && pr < mu) {
          const double x = col[jr];
          col[jr] = col[pr];
          col[pr] = x;
        }
      }
    __syncwarp();
    if (g >= c0 + wP) {
      for (int t = 0; t < wP; ++t) {  // U block: unit-lower solve with the panel's top wP x wP, lanes t+1..wP-1
        const double x = col[c0 + t];
        __syncwarp();
        if (lane > t && lane < wP) col[c0 + lane] = fma(-cur[(size_t)t * mu + c0 + lane], x, col[c0 + lane]);
        __syncwarp();
      }
      double u[kLuB];
#pragma unroll
      for (int t = 0; t < kLuB; ++t) u[t] = t < wP ? col[c0 + t] : 0.0;
      for (int i = c0 + wP + lane; i < mu; i += 32) {
        double a = col[i];
#pragma unroll
        for (int t = 0; t < kLuB; ++t)
          if (t < wP) a = fma(-cur[(size_t)t * mu + i], u[t], a);
        col[i] = a;
      }
    }
    __syncwarp();
  };
  if (r == 0) factor(0);  // panel 0's owner
  for (int P = 0; P < np; ++P) {
    const int owner = P % CL, lpo = P / CL, c0 = P * kLuB;
    const int wP = mu - c0 < kLuB ? mu - c0 : kLuB;
    cluster.sync();  // panel P is published
    {
      const double* rp = cluster.map_shared_rank(pub, owner);
      const int* rpp = cluster.map_shared_rank(pub_piv, owner);
      for (int idx = tid; idx < wP * mu; idx += blockDim.x)
        if (idx % mu >= c0) cur[idx] = rp[idx];
      if (tid < wP) s_pp[tid] = rpp[tid];
    }
    __syncthreads();
    // the owner of panel P+1 brings that panel up to date and factors and publishes it
    // before updating its other columns (the cluster barrier still waits for every
    // CTA's updates: measured, this order costs nothing and gains nothing)
    const int nxt = P + 1 < np ? (P + 1) % CL : -1, lpn = (P + 1) / CL;
    if (r == nxt) {
      for (int jj = warp; jj < kLuB; jj += nw)
        if ((P + 1) * kLuB + jj < mu) apply(lpn * kLuB + jj, c0, wP);
      __syncthreads();
      factor(P + 1);
    }
    for (int lc = warp; lc < myp * kLuB; lc += nw) {
      const int lp = lc / kLuB;
      const int g = (lp * CL + r) * kLuB + lc % kLuB;
      if (g >= mu || (r == owner && lp == lpo) || (r == nxt && lp == lpn)) continue;
      apply(lc, c0, wP);
    }
    __syncthreads();  // cur and s_pp are refilled for the next panel
  }
  {  // log|U_jj| of my panels' columns, in parallel, summed in a fixed order
    double a = 0.0;
    for (int lc = tid; lc < myp * kLuB; lc += blockDim.x) {
      const int g = ((lc / kLuB) * CL + r) * kLuB + lc % kLuB;
      if (g < mu) {
        const double d = loc[(size_t)lc * mu + g];
        if (d != 0.0 && isfinite(d)) a += log(fabs(d));
      }
    }
    a = warp_sum(a);
    if (lane == 0) rv[warp] = a;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += rv[w];
      s_ld = t;
    }
  }
  cluster.sync();
  for (int lp = 0; lp < myp; ++lp)
    for (int jj = 0; jj < kLuB; ++jj) {
      const int g = (lp * CL + r) * kLuB + jj;
      if (g >= mu) break;
      const double* srcl = loc + (size_t)(lp * kLuB + jj) * mu;
      double* dst = M + (size_t)g * ld;
      for (int i = tid; i < mu; i += blockDim.x) dst[i] = srcl[i];
      if (tid == 0) piv[g] = s_piv[g];
    }
  if (r == 0 && tid == 0 && logdet) {  // partial sums in rank order: deterministic
    double a = 0.0;
    for (int q = 0; q < CL; ++q) a += *cluster.map_shared_rank(&s_ld, q);
    *logdet = a;
  }
  cluster.sync();  // no CTA exits while rank 0 may still read its s_ld
}

cudaError_t launch_lu_fast(double* M, int ld, const int* mdev, int max_m, int* piv, double* logdet, DevState* st,
                           cudaStream_t s) {
  {  // blocked: my panels, the publish buffer (+ pivots) and the applied copy
    const int np = (max_m + kLuB - 1) / kLuB;
    const size_t smem = ((size_t)((np + 15) / 16) * kLuB * max_m + 2 * (size_t)kLuB * max_m + kLuB) * sizeof(double);
    if (smem <= 200 * 1024) {
      void* args[] = {&M, &ld, (void*)&mdev, &piv, &logdet, &st};
      cudaError_t e = launch_cluster(k_lu_blocked<16>, 16, smem, s, args);
      if (e == cudaSuccess) return e;
      cudaGetLastError();
    }
  }
  for (int cl : {16, 8}) {
    const size_t smem = ((size_t)((max_m + cl - 1) / cl) + 1) * max_m * sizeof(double);
    if (smem > 200 * 1024) continue;
    void* args[] = {&M, &ld, (void*)&mdev, &piv, &logdet, &st};
    cudaError_t e = cl == 16 ? launch_cluster(k_lu_cluster<16>, 16, smem, s, args)
                             : launch_cluster(k_lu_cluster<8>, 8, smem, s, args);
    if (e == cudaSuccess) return e;
    cudaGetLastError();
  }
  return launch_lu(M, ld, mdev, piv, logdet, st, s);
}

}  // namespace fab
