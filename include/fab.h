/*
 * fab.h - C ABI of libfab: randomized Krylov approximations of f(A)b on one
 * GB300 GPU (sm_103a), after Cortinovis, Kressner and Nakatsukasa,
 * "Speeding up Krylov subspace methods for computing f(A)b via randomization"
 * (arXiv 2212.12758).
 *
 * Problem (paper §1): given a sparse nonsymmetric A (n x n, CSR) and b, compute
 * x ~ f(A) b for f in {exp(tz), z^{1/2}, z^{-1/2}} from an m-dimensional Krylov
 * space K_m(A, b) = span{b, Ab, ..., A^{m-1} b} (eq. krylovspace).
 *
 * Methods (enum fab_method):
 *   FAB_ARNOLDI        eq. standardfm: ||b|| U_m f(K_m) e_1 with an orthonormal
 *                      Arnoldi basis (classical Gram-Schmidt applied twice).
 *   FAB_SKETCHED_LS    Alg. 4: Alg. 2 basis, y = argmin ||V_m z - v_{m+1}|| by
 *                      Blendenpik (QR of Theta V_m as preconditioner, LSQR), then
 *                      ||b|| V_m f(H_m + h_{m+1,m} y e_m^T) e_1 (eq. relationxx).
 *   FAB_SKETCHED_FAST  eq. sFOM in its sketch-and-solve form (Remark after eq. sFOM):
 *                      y = argmin ||Theta (V_m z - v_{m+1})||, then as above.
 *   FAB_NOPROJ         Alg. 5: ||b|| V_m f(H_m) e_1 (eq. noproj).
 *   FAB_BG_LS          Alg. 3: Alg. 1 basis (sketched Gram-Schmidt: S = Theta V
 *                      kept orthonormal, the same coefficients applied to the
 *                      long vectors), y by LSQR on V_m (no preconditioner), then
 *                      r_11 V_m f(H_m + h_{m+1,m} y e_m^T) e_1. k is ignored; the
 *                      sketch is SRHT or sparse sign (it is applied to every new
 *                      vector before its orthogonalization).
 *   FAB_WHITEN         Alg. 2 with whitening and a switch to Alg. 1 (§2.1.2, §5.1.3):
 *                      after every new column the condition number
 *                      kappa_1(R_i) = ||R_i||_1 ||R_i^{-1}||_1 of the thin QR
 *                      Theta V_i = Q_i R_i (diag R_i > 0) is updated exactly. At the
 *                      first kappa_1 > whiten_kappa the basis becomes V_i R_i^{-1},
 *                      H_{i-1} becomes R_i H_{i-1} R_{i-1}^{-1}, and Alg. 1 builds
 *                      the remaining columns with the same Theta; the solve then
 *                      ends as FAB_BG_LS (Alg. 3, gamma_b = ||b|| r_11). A basis
 *                      that is never whitened ends as FAB_NOPROJ (Alg. 5), as §6
 *                      recommends. Sketch SRHT or sparse sign; fixed m only.
 * The Alg. 2 basis orthogonalizes A v_{i-1} against the last k basis vectors
 * only (§2.1.2); the sketch Theta (s x n) is applied in the same pass that
 * produces each basis vector.
 *
 * Sketches (enum fab_sketch), all generated on the device from (seed, index)
 * by SplitMix64 (stream 1 sparse-sign rows, 2 signs, 3 SRHT D, 4 SRHT P):
 *   FAB_SK_SPARSE_SIGN  zeta nonzeros +-1/sqrt(zeta) per column (paper §2.1.1).
 *   FAB_SK_SRHT         s^{-1/2} P H D on the input zero-padded to n' = 2^ceil(log2 n)
 *                       (paper §2.1.1).
 *   FAB_SK_GAUSSIAN     dense N(0, 1/s) entries, rounded to BF16 (stream 5, Box-Muller);
 *                       applied to a BF16 copy of the basis on the tensor cores with FP32
 *                       accumulation. fab_apply accepts it with FAB_MIXED and m+1 <= 256.
 *
 * Conventions for every entry point:
 *   - Return FAB_OK (0) or a negative FAB_E* code; nothing throws across the ABI.
 *   - Pointers flagged "on device" are CUDA device pointers of the current
 *     device; otherwise host pointers. All arrays are caller-owned and are not
 *     retained after the call returns, except as stated for handles.
 *   - Handles are not thread-safe; use one handle per host thread.
 *   - A fab_params.stream of NULL means the legacy default stream.
 */
#ifndef FAB_H
#define FAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FAB_OK = 0,
  FAB_EINVAL = -1,    /* invalid argument: bad CSR, k < 1, s < m+1, sizes out of range */
  FAB_ENOMEM = -2,    /* device or host allocation failed (nothing leaked)             */
  FAB_ECUDA = -3,     /* a CUDA call failed                                            */
  FAB_ENUMERIC = -4,  /* NaN/Inf in the basis, or no principal square root             */
  FAB_ETIMEOUT = -5,  /* a bounded wait expired                                        */
  FAB_ENOTCONV = -6   /* LSQR or the square-root iteration hit its iteration limit     */
};

/* FAB_F_SIGN: sign(A) b computed as (A^2)^{-1/2} (A b) (§5.1.3): the method runs on A^2
 * (formed once per handle on the host and kept on the device) from the starting
 * vector A b with f = inverse square root. Single solves only (FAB_EINVAL in a
 * batch or a server); fab_last_state / fab_last_basis then describe nothing. */
typedef enum { FAB_F_EXP = 0, FAB_F_SQRT = 1, FAB_F_INVSQRT = 2, FAB_F_SIGN = 3 } fab_func;
typedef enum {
  FAB_ARNOLDI = 0,
  FAB_SKETCHED_LS = 1,
  FAB_SKETCHED_FAST = 2,
  FAB_NOPROJ = 3,
  FAB_BG_LS = 4,
  FAB_WHITEN = 5
} fab_method;
typedef enum { FAB_SK_SPARSE_SIGN = 0, FAB_SK_SRHT = 1, FAB_SK_GAUSSIAN = 2 } fab_sketch;
typedef enum { FAB_FP64 = 0, FAB_MIXED = 1 } fab_precision;

/* Parameters of one solve. Fill with fab_params_default() and override. */
typedef struct fab_params {
  int f;             /* fab_func                                                   */
  double t;          /* f(z) = exp(t z) for FAB_F_EXP; ignored otherwise           */
  int m;             /* Krylov dimension, 1 <= m <= 1024                            */
  int k;             /* truncation window of Alg. 2, 1 <= k <= 8 (ignored by Arnoldi) */
  int s;             /* sketch rows, m+1 <= s <= 4096 (sketched methods)            */
  int zeta;          /* nonzeros per column of the sparse-sign sketch, 1..min(s,16) */
  int sketch;        /* fab_sketch                                                 */
  uint64_t seed;     /* sketch seed                                                */
  int method;        /* fab_method                                                 */
  int precision;     /* fab_precision: FAB_FP64, or FAB_MIXED (FP32 A and basis, BF16 */
                     /* Gaussian sketch, FP64 small stage)                          */
  double lsqr_tol;   /* LSQR stopping tolerance (paper §5 uses 1e-6)               */
  int lsqr_maxit;    /* LSQR iteration limit (0: 4m)                               */
  void* stream;      /* cudaStream_t to run on, or NULL                            */
  /* Growing m to a target accuracy (0 = off, the fixed m above). The basis is */
  /* extended by m_step columns at a time, up to m_max, until the sketched    */
  /* relative change ||Theta V (c_m - c_{m-step})|| / ||Theta V c_m|| of two  */
  /* successive solutions is at most target_rel_err (the sketch embeds x_m -  */
  /* x_{m-step}, §2.1.1). Sketched methods only; s >= m_max + 1. If m_max is  */
  /* reached first the call returns FAB_ENOTCONV with the m_max solution in x. */
  double target_rel_err;
  int m_step;
  int m_max;
  /* FAB_WHITEN: whiten when kappa_1 of the sketched basis exceeds this (0: 1000, */
  /* the threshold of §5.1.3; +Inf: never, i.e. Alg. 5 with the check running)   */
  double whiten_kappa;
} fab_params;

/* Diagnostics of the last solve (all optional for the caller). */
typedef struct fab_stats {
  int m_used;           /* basis dimension actually used (< m after a breakdown) */
  int lsqr_iters;       /* LSQR iterations (FAB_SKETCHED_LS)                     */
  int fh_iters;         /* squarings (exp) or Denman-Beavers iterations           */
  int launches;         /* kernel launches issued by this solve                  */
  double h_last;        /* h_{m+1,m}                                             */
  double beta;          /* ||b||_2 (gamma_b = ||Theta b|| for Alg. 1 and whitening) */
  double ms_basis;      /* device time of the basis (+ fused sketch) loop        */
  double ms_small;      /* device time of QR / LSQR / f(H)                       */
  double ms_combine;    /* device time of x = ||b|| V_m c                        */
  double ms_total;      /* device time of the whole solve                        */
  double err_est;       /* last sketched relative change (target mode), else 0   */
  int whiten_at;        /* FAB_WHITEN: basis columns when it was whitened, 0: never */
  double kappa_est;     /* sketched methods with a sketch QR (FAB_SKETCHED_FAST,      */
                        /* FAB_SKETCHED_LS): max|r_ii| / min|r_ii| of Theta V_m = Q R, */
                        /* a lower bound on kappa_2(Theta V_m), which tracks kappa_2 */
                        /* of the basis within the sketch's distortion (§2.1.2); 0   */
                        /* for the other methods                                     */
} fab_stats;

typedef struct fab_handle fab_handle;

/* Default parameters: exp with t = 1, m = 30, k = 2, s = 4m... set explicitly. */
void fab_params_default(fab_params* p);

/* Message for an error code (static string). */
const char* fab_strerror(int code);

/* Detail of the last FAB_ECUDA returned on this host thread: the kernel class
 * whose launch (or, with FAB_SYNC_CHECK=1 in the environment, whose execution)
 * failed and the CUDA error string. Empty if none. fab_server_poll returning
 * FAB_ECUDA sets it to the detail of the slot thread that ran the solve. */
const char* fab_last_error(void);

/*
 * fab_create - copy A (CSR) into a new handle.
 *   n       matrix order, 1 <= n < 2^31
 *   nnz     number of stored entries, 0 <= nnz < 2^31
 *   rowptr  n+1 row offsets (int64), rowptr[0] = 0, nondecreasing, rowptr[n] = nnz
 *   colind  nnz column indices (int32), each in [0, n)
 *   vals    nnz FP64 values
 *   inputs_on_device  nonzero if the three arrays are device pointers
 * The handle owns its device copy of A and all solve workspace; the caller keeps
 * ownership of its arrays. Validation (monotone rowptr, column range) is done on
 * the host copy; invalid input returns FAB_EINVAL and *out is left NULL.
 * The matrix is the operator A of the paper's problem statement (§1).
 */
int fab_create(fab_handle** out, int64_t n, int64_t nnz, const int64_t* rowptr,
               const int32_t* colind, const double* vals, int inputs_on_device);

/*
 * fab_apply - x ~ f(A) b with the method, basis and sketch given in *p.
 *   b, x           n-vectors (FP64), device pointers if bx_on_device else host
 *   st             optional diagnostics (may be NULL); also filled when the call
 *                  returns FAB_ENOTCONV or FAB_ENUMERIC from f(H) (x is then not
 *                  written; m_used, the iteration counts and kappa_est say how far
 *                  the solve got)
 * Runs on p->stream; returns after x is written (the call synchronizes that
 * stream). Workspace grows on demand and is kept by the handle. A breakdown of
 * the basis (h_{c,c-1} <= 64 eps ||A v_{c-1}||, the norm taken as
 * (h_{c,c-1}^2 + sum_j h_{j,c-1}^2)^(1/2) over the orthogonalized columns) is not
 * an error: the space is invariant and the result uses m_used = c basis vectors.
 * b = 0 gives x = 0.
 */
int fab_apply(fab_handle* h, const fab_params* p, const double* b, double* x,
              int bx_on_device, fab_stats* st);

/* Release a handle and everything it owns. NULL-safe. */
void fab_destroy(fab_handle* h);

/*
 * fab_last_state - copy the last solve's small quantities to host arrays.
 *   H      (m+1) x m Hessenberg, column-major, ld = m+1 (paper's underline H_m)
 *   SV     s x (m+1) sketch Theta V_{m+1}, column-major (sketched methods; else untouched)
 *   y      m-vector of eq. leastsquares (sketched methods; zero for the others)
 *   coeffs m-vector c with x = ||b|| V_m c
 * Any pointer may be NULL. Sizes are those of the last fab_apply's m and s.
 * Returns FAB_EINVAL if no solve has run on this handle.
 */
int fab_last_state(fab_handle* h, double* H, double* SV, double* y, double* coeffs);

/*
 * fab_last_basis - copy the last solve's basis V_{m+1} (n x (m+1), column-major,
 * ld = n) to a host or device array (dst_on_device). The library stores each
 * column unnormalized with a separate scale; the copy holds the normalized v_j.
 */
int fab_last_basis(fab_handle* h, double* V, int dst_on_device);

/*
 * fab_sketch_apply - out = Theta V for ncols device columns.
 *   sketch, s, zeta, seed  as in fab_params (Theta is s x n)
 *   V_dev   device array, column j at V_dev + j*ldv, ldv >= n
 *   out_dev device array s x ncols, column-major, ld = s
 *   stream  cudaStream_t or NULL
 * Sign sketches use the same fused kernels as the basis loop (exact int64 block
 * transform per 4096-row chunk, FP64 cross-chunk sums); the Gaussian sketch
 * rounds the columns to BF16 and multiplies on the tensor cores (ncols <= 256).
 * Allocates its scratch with cudaMallocAsync on the stream and synchronizes the
 * stream before returning.
 */
int fab_sketch_apply(int sketch, int64_t n, int s, int zeta, uint64_t seed,
                     const double* V_dev, int64_t ldv, int ncols, double* out_dev, void* stream);

/*
 * fab_sketch_apply_noalloc - the same out = Theta V as fab_sketch_apply (same
 * arguments, same kernels, same result), but it allocates no device memory:
 * its scratch lives in one fixed array inside the library.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate while they run: a host application that pre-reserves or caps all
 * device memory for its own allocator, or a latency-sensitive loop where a
 * cudaMalloc/cudaFree (which may synchronize the device) is not acceptable.
 *
 * Limits: the fixed scratch holds ceil(n/4096) * s <= 1,048,576 chunk partial
 * sums (8 MiB) plus the SRHT row sample (s <= 4096); larger sizes return
 * FAB_EINVAL without touching the device. Every GPU that loads the library
 * keeps this scratch (about 8.02 MiB) until the process exits.
 * Set-up: the first call on each device looks up the scratch address on that
 * device (the device must be current); make that first call before any stream
 * capture. The address is kept for the life of the process: a caller that runs
 * cudaDeviceReset must not call this entry point on that device afterwards.
 * Sharing: all calls on a device use the same scratch and it keeps the last
 * call's contents (each call clears what it needs); calls whose work overlaps
 * on the GPU (different streams or host threads) race on it, so serialize them.
 * Returns after synchronizing `stream`.
 */
int fab_sketch_apply_noalloc(int sketch, int64_t n, int s, int zeta, uint64_t seed,
                             const double* V_dev, int64_t ldv, int ncols, double* out_dev, void* stream);

/*
 * Serving (continuous batching). A server owns `slots` worker threads on the
 * current device, each with its own CUDA stream and its own device workspace,
 * so requests of different n, m, f and method run concurrently and their bases
 * and sketches stay resident between requests. Requests leave the queue in
 * submission order as soon as a slot is free and the request's workspace fits
 * both the device-memory budget and the memory the device reports free.
 * This runtime is not part of the paper; it serves the paper's solves.
 *
 * fab_server_create  hbm_budget_bytes: device bytes all slot workspaces may
 *                    hold together (0: 90 % of the free memory now); slots 1..64.
 * fab_server_submit  b: host n-vector, copied before the call returns; *p is
 *                    copied (its stream is ignored). h must outlive its requests;
 *                    the server never modifies h except to add its FP32 matrix
 *                    copy for FAB_MIXED. FAB_ENOMEM if the request alone exceeds
 *                    the budget. Thread-safe.
 * fab_server_poll    waits up to timeout_ms for the ticket: FAB_ETIMEOUT if not
 *                    done (the request stays); otherwise copies x (host n-vector),
 *                    the stats and the latency from submission to completion
 *                    (ms), releases the ticket and returns the solve's code.
 * fab_server_destroy finishes the solves in progress, drops queued requests,
 *                    frees everything. NULL-safe.
 */
typedef struct fab_server fab_server;
typedef struct fab_server_stats {
  int64_t submitted, completed, queued, in_flight;
  double bytes_in_use;  /* device bytes held by the slot workspaces */
  double bytes_budget;
} fab_server_stats;

int fab_server_create(fab_server** out, size_t hbm_budget_bytes, int slots);
int fab_server_submit(fab_server* srv, fab_handle* h, const fab_params* p, const double* b, uint64_t* ticket);
int fab_server_poll(fab_server* srv, uint64_t ticket, double* x, fab_stats* st, double* latency_ms,
                    int timeout_ms);
int fab_server_stats_get(fab_server* srv, fab_server_stats* out);
void fab_server_destroy(fab_server* srv);

/*
 * SpMV tiling of a matrix (the work unit of the SpMV + window-dot kernel, Alg. 2).
 * The rows are cut into tiles of consecutive rows with at most rows_max (<= 256)
 * rows and at most nnz_cap nonzeros each (a longer row is a tile of its own);
 * a tile with R rows runs 256 / pow2ceil(R) lanes per row, so short rows get a
 * thread each and a long row the whole block. staged = 1 copies a tile's
 * nonzeros into shared memory (bulk copies) when they fit 2048 entries.
 * staged = 2 stages the same way and processes a staged tile of at least 32 rows
 * by nonzeros: each thread takes 8 consecutive entries whatever their rows, and
 * the row sums are assembled in a fixed order (for short rows of uneven length,
 * such as a power-law graph's); tiles cut by the nonzero cap then keep any row
 * count. fab_create uses (256, 2048, 1), or (256, 2048, 2) when the row-per-lane form
 * would leave more than a fifth of the lanes idle (each group of 32 consecutive rows
 * runs for its longest row). The tiling fixes the order of the SpMV
 * additions, so results differ within rounding between tilings (and are
 * reproducible for a given one).
 * fab_set_tiling  sets it; FAB_EINVAL for rows_max outside 1..256, nnz_cap < 1,
 *                 staged outside 0..2 or a workspace clone.
 * fab_tune        times the kernel on h's matrix (precision FAB_FP64 or
 *                 FAB_MIXED, window k) for rows_max in {256, 128, 64}, nnz_cap
 *                 in {2048, 1024, 512} and staged in {2, 1, 0}, keeps the fastest
 *                 and writes it to choice[3] (nullable). Uses a temporary device
 *                 buffer of about (k+1) n words; `stream` is a cudaStream_t or NULL.
 * Neither may run while a solve, batch or server request uses h.
 */
int fab_set_tiling(fab_handle* h, int rows_max, int nnz_cap, int staged);
/*
 * fab_set_fusion - one-pass basis steps of the FP32 basis (FAB_MIXED; Alg. 2 with a
 * sign sketch or none: FAB_SKETCHED_FAST, FAB_SKETCHED_LS, FAB_NOPROJ). A pass updates,
 * normalizes and sketches column c-1 (the window update of Alg. 2) and multiplies it by
 * A with the window dots of step c, so each basis step reads A and the window once;
 * values of column c-1 outside a block's 4096-row chunk are recomputed from the
 * previous SpMV output and the window by the same FMAs their owner runs. Used only
 * when every row of A has at most 8 nonzeros. on = 1 allows it; 0 (the default) keeps
 * the two-pass loop (SpMV + dots, then update + norm + sketch), which is faster on
 * GB300 (the one-pass form moves fewer bytes but hides less latency). The two forms
 * differ only in the grouping of the FP32 partial sums of the dot products and norms.
 * FAB_EINVAL for a NULL handle. Not while a solve, batch or server request uses h.
 */
int fab_set_fusion(fab_handle* h, int on);
/*
 * fab_inject_wait_timeout - failure-detection hook for tests (not part of the paper).
 * In the next solve on h that runs the one-pass steps (fab_set_fusion), the SpMV tasks
 * of basis step `pass` (1 <= pass <= m) wait for a chunk flag value that no task sets
 * and give up after `polls` polls of it (each about a microsecond): the kernel records
 * FAB_ETIMEOUT and returns, no copy is in flight and nothing faults, and fab_apply
 * returns FAB_ETIMEOUT. The hook is one-shot; later solves on h run normally.
 * pass = 0 disarms it. FAB_EINVAL for a NULL handle, pass < 0, or polls < 1.
 */
int fab_inject_wait_timeout(fab_handle* h, int pass, int polls);
int fab_tune(fab_handle* h, int precision, int k, int* choice, void* stream);

/*
 * Batched solves: many f(A)b of uneven size (different matrices, n, m, k, s, f)
 * as one CUDA graph of three kernels. The basis build of every solve (Alg. 2 with
 * the sketch of §2.1.1: per step the SpMV + window dots, then the window update +
 * norm + fused sketch; the sketch's partials are reduced once per solve at the end)
 * is one persistent launch: its blocks claim work items (one block's share of one
 * phase of one solve) in plan order from a device counter and wait, with a bounded
 * wait, only for their own solve's previous phase. A solve's SpMV tiles are grouped
 * at least 32 to a block (a batched solve shares the GPU), so its results equal
 * fab_apply's up to the grouping of partial sums (same bodies, same tiles, same
 * sketch). Then one launch runs every solve's small stage as one CTA (Householder
 * QR of the sketch, the sketch-and-solve projection of eq. sFOM, or none for Alg.
 * 5; f(H)e_1 by Pade scaling and squaring or Denman-Beavers) and one the combines
 * x = ||b|| V_m c. A solve whose phase wait expires reports FAB_ETIMEOUT.
 *
 * fab_batch_create  plans `count` solves (hs[i], ps[i]) and allocates every
 *                   workspace at once (one device allocation; FAB_ENOMEM if it
 *                   does not fit), then captures and instantiates the graph.
 *                   Supported: method FAB_SKETCHED_FAST (sketch SRHT or sparse
 *                   sign) or FAB_NOPROJ; precision the same for all solves
 *                   (FAB_FP64 or FAB_MIXED); fixed m (target_rel_err = 0);
 *                   anything else FAB_EINVAL. A
 *                   handle may appear several times; handles must outlive the
 *                   batch and must not be destroyed or used concurrently while
 *                   it runs. ps[0].stream is used for set-up.
 * fab_batch_exec    one run: copies bs[i] (n_i FP64, host or device; NULL bs =
 *                   inputs already written to fab_batch_input(bt, i)), launches
 *                   the graph on `stream` (cudaStream_t or NULL), copies each
 *                   result to xs[i] (NULL xs or xs[i] = leave it at
 *                   fab_batch_output(bt, i)), waits, and fills sts[i]
 *                   (nullable). Returns the first non-FAB_OK solve status
 *                   (the other solves' results are valid) or FAB_OK.
 * fab_batch_input / fab_batch_output  device addresses (n_i FP64) of solve i's
 *                   start vector and result; NULL for a bad index.
 * fab_batch_kernels number of kernel launches in the graph.
 * fab_batch_destroy NULL-safe.
 * fab_batch_run     create + exec + destroy in one call (bs, xs required).
 */
typedef struct fab_batch fab_batch;
int fab_batch_create(fab_batch** out, fab_handle* const* hs, const fab_params* ps, int count);
int fab_batch_exec(fab_batch* bt, const double* const* bs, double* const* xs, fab_stats* sts, void* stream);
double* fab_batch_input(fab_batch* bt, int i);
double* fab_batch_output(fab_batch* bt, int i);
int fab_batch_kernels(const fab_batch* bt);
void fab_batch_destroy(fab_batch* bt);
int fab_batch_run(fab_handle* const* hs, const fab_params* ps, const double* const* bs, double* const* xs, int count,
                  fab_stats* sts);

/*
 * Kernel-level device timing (measurement support, not needed for solving).
 * fab_profile_enable(1) resets the accumulators and makes every later
 * fab_apply record CUDA events, on the solve's stream, around each launch of
 * the kernel classes below; fab_profile_enable(0) stops recording.
 * fab_profile_query returns the accumulated device time (ms) and the number of
 * launches of one class:
 *   "spmv_dots"      SpMV fused with the window dot products (Alg. 2)
 *   "update"         window update + norm + fused sketch of the new vector
 *   "sketch_reduce"  cross-block reduction of the sketch (per step, or once per
 *                    pass where nothing reads the sketch before the pass ends)
 *   "gemv_t"         V^T w passes (Arnoldi, LSQR)
 *   "small"          QR / LSQR scalar steps / f(H) kernels
 *   "combine"        x = ||b|| V_m c and the LSQR vector update
 *   "fused_step"     one-pass basis step of the FP32 basis (window update, norm and
 *                    sketch of column c-1 with the SpMV and window dots of step c)
 * fab_profile_only(name) restricts the recording to that class (NULL or ""
 * restores every class): each event pair adds a little device time between
 * launches, so a throughput measurement brackets only the kernel it needs.
 * Unknown names return FAB_EINVAL. Process-wide; not thread-safe.
 */
/*
 * fab_fma_peak - measured fused multiply-add throughput of this GPU (measurement
 * support: the arithmetic bound of the FP64 basis kernels, which do about one FP64
 * FMA per 4 to 8 bytes they move). Runs independent chains of FMAs on every SM, in
 * three operand patterns (the rate depends on how operands fall on the register
 * banks), times each with CUDA events at the clocks the GPU runs now (it changes no
 * clock) and reports the fastest.
 *   precision  FAB_FP64 (FP64 FMAs) or FAB_MIXED (FP32 FMAs)
 *   gflops     2 x FMAs / second / 1e9 (one FMA counts two flops)
 *   ms         nullable: duration of the fastest timed launch (at least about 50 ms)
 *   stream     cudaStream_t or NULL; the call synchronizes it
 * FAB_EINVAL for another precision or a NULL gflops.
 */
int fab_fma_peak(int precision, double* gflops, double* ms, void* stream);

int fab_profile_enable(int on);
int fab_profile_only(const char* name);
int fab_profile_query(const char* name, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* FAB_H */
