// Launchers of the small dense FP64 kernels (small.cu). Internal.
#pragma once

#include "fab_internal.cuh"

namespace fab {

struct LsqrVecs {
  double* v;
  double* w;
  double* x;
  double* z;
  double* coef;
  double* q;  // sigma_j <W_j, ustore> from the GEMV-T reduction
};

cudaError_t launch_householder_qr(double* A, int lda, int rows, const int* mdev, int extra, double* tau,
                                  cudaStream_t s);
// Cluster (DSMEM) versions when the matrix fits a cluster's shared memory.
// Householder QR of the rows x (mu + extra) matrix A (R in the upper triangle, v_j below
// the diagonal, tau_j in tau). start > 0: columns below start hold an earlier call's
// factorization, columns start .. fresh-1 already carry its reflectors (its extra
// column), columns from fresh on are new; only the rest is factored (cluster path
// only: qr_cluster_fits).
cudaError_t launch_qr(double* A, int lda, int rows, const int* mdev, int max_cols, int extra, double* tau,
                      DevState* st, cudaStream_t s, int start = 0, int fresh = 0);
bool qr_cluster_fits(int rows, int ncols);
// st->kappa = max |r_ii| / min |r_ii| over the first min(*mdev, ncols) columns of the
// factored QR buffer (a lower bound on kappa_2 of the factored matrix).
cudaError_t launch_kappa_diag(const double* R, int lda, const int* mdev, int ncols, DevState* st, cudaStream_t s);
cudaError_t launch_lu_fast(double* M, int ld, const int* mdev, int max_m, int* piv, double* logdet, DevState* st,
                           cudaStream_t s);
// mmax: largest *mdev (R's triangle is staged in shared memory when mmax <= 150; 0: never)
cudaError_t launch_trsv(const double* R, int ldr, const int* mdev, const double* xin, double* xout, int trans,
                        const double* pre, cudaStream_t s, int mmax = 0);
cudaError_t launch_build_hhat(const double* H, int ldh, const int* mdev, const double* y, double scale, double* M,
                              int ldm, int mmax, cudaStream_t s);
cudaError_t launch_norm1(const double* M, int ldm, const int* mdev, double* out, cudaStream_t s);
cudaError_t launch_gemm(double* C, const double* A, const double* B, int ld, const int* mdev, int mmax, double alpha,
                        double beta, cudaStream_t s);
cudaError_t launch_lincomb(double* out, const double* X0, const double* X1, const double* X2, const double* X3,
                           double a0, double a1, double a2, double a3, double d, int ld, const int* mdev, int mmax,
                           cudaStream_t s);
cudaError_t launch_lu(double* M, int ld, const int* mdev, int* piv, double* logdet, DevState* st, cudaStream_t s);
cudaError_t launch_lu_solve(const double* LU, int ld, const int* piv, const int* mdev, int mmax, double* B, int ldb,
                            int identity_rhs, cudaStream_t s);
// One Denman-Beavers step over several blocks (part: gridDim doubles of partials,
// counter: a zeroed last-block counter, left zeroed).
cudaError_t launch_db_update(double* M, const double* Minv, int ld, const int* mdev, double* y, const double* logdet,
                             int scale_on, DevState* st, cudaStream_t s, int mmax, double* part, unsigned* counter);
cudaError_t launch_first_column(const double* M, const int* mdev, double* y, cudaStream_t s);
cudaError_t launch_prep_coef(const double* c, const double* sigma, const int* mdev, const DevState* st, double* coef,
                             cudaStream_t s);
cudaError_t launch_lsqr_start(const double* R, int ldr, const int* mdev, const double* sigma, const double* unorm2,
                              const LsqrVecs& lv, double tol, DevState* st, cudaStream_t s, int mmax = 0);
cudaError_t launch_lsqr_step(const double* R, int ldr, const int* mdev, const double* sigma, const double* unorm2,
                             const LsqrVecs& lv, DevState* st, cudaStream_t s, int mmax = 0);
template <typename TV>
cudaError_t launch_lsqr_u(int n, const TV* W, int64_t ld, int nc, const double* coef, double* u, int keep_zero,
                          double* part, unsigned* counter, double* unorm2, const DevState* st, cudaStream_t s);

// Step c of Alg. 1 on the sketches (see k_bg_orth) and R = I for Alg. 3's LSQR.
// Ri (ld ldr): R^{-1} of a basis whitened at st->wh columns (FAB_WHITEN), else NULL;
// gate: see gate_closed.
cudaError_t launch_bg_orth(double* SV, int lds, int c, double* H, int ldh, double* coef, ColScale cs, DevState* st,
                           cudaStream_t s, const double* Ri = nullptr, int ldr = 0, int gate = 0);
// Whitening (FAB_WHITEN, see k_wh_check): the condition check of step c and, at the
// first kappa_1 > kmax, the whitening of H and the sketch; the LSQR preconditioner
// of a whitened basis; whitened coordinates to stored columns.
cudaError_t launch_wh_check(double* SV, int lds, int c, double* Q, double* R, double* Ri, double* T, int ldr,
                            double* H, int ldh, double kmax, double* wcoef, double* nrm, ColScale cs, DevState* st,
                            cudaStream_t s);
cudaError_t launch_wh_precond(const double* R, int ldr, int wh, double* P, int rows, const int* mdev, int mmax,
                              cudaStream_t s);
cudaError_t launch_wh_coef(const double* Ri, int ldr, int wh, const int* mdev, double* cv, cudaStream_t s);
cudaError_t launch_set_identity(double* R, int rows, const int* mdev, int mmax, cudaStream_t s);
// out[0] = ||SV c_new - SV c_old||, out[1] = ||SV c_new|| (growing m to a target).
cudaError_t launch_sketch_change(const double* SV, int lds, const int* mdev, const double* c_new, int m_old,
                                 const double* c_old, double* out, cudaStream_t s);

// One solve's small stage for the batched path: everything between the basis
// and the combine, done by one CTA (k_small_fused).
struct SmallJob {
  int method, f, m, s;
  double t;
  const double* H;  // (m+1) x m, ld ldh
  int ldh;
  const double* SV;     // s x (m+1) sketch of the basis (sketched_fast)
  const double* sigma;  // column scales of the raw basis
  DevState* st;
  double* qr;    // s x (m+1)
  double* tau;   // m+1
  double* y;     // m+1
  double* mats;  // 9 m x m, ld m
  int* piv;      // m+1
  double* cvec;  // m+1: f(H) e_1
  double* scal;  // 16 scalars
  double* coef;  // m+1: output, ||b|| sigma_j c_j (zero when b = 0)
};
struct PadeCoef {
  double b[14];  // [13/13] numerator coefficients (denominator: alternating signs)
  double theta;  // largest 1-norm for which the unscaled approximant is used
};

// One CTA of 256 threads per listed job (ids[i] indexes jobs; ids NULL = 0..count-1).
cudaError_t launch_small_fused(const SmallJob* jobs, const int* ids, int count, int mmax, const PadeCoef& pd,
                               cudaStream_t s);
// Sets the kernel's shared-memory limit for m <= mmax (before a graph capture).
cudaError_t small_fused_prepare(int mmax);

}  // namespace fab
