// C ABI of libfab (include/fab.h): handle lifetime, workspace, and the host
// orchestration of one f(A)b solve. Every arithmetic step runs in the kernels
// of basis.cu and small.cu; this file only validates arguments, allocates,
// and enqueues launches on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "fab_internal.cuh"
#include "gauss.cuh"
#include "handle.cuh"
#include "small.cuh"

using namespace fab;

namespace {

// Pade [13/13] approximant of exp (Higham, "The scaling and squaring method for the
// matrix exponential revisited", SIAM J. Matrix Anal. Appl. 26 (2005)):
// coefficients c_j = (2m-j)! m! / ((2m)! j! (m-j)!), m = 13, and the backward-error
// threshold theta_13 of that paper's Table 2.3.
constexpr double kTheta13 = 5.371920351148152;
constexpr int64_t kCsrPad = 4;  // spare CSR entries for the aligned tile copies
constexpr int kLsqrPoll = 8;    // LSQR iterations between host reads of the convergence flag

// Bump allocator over a caller-provided device buffer (256-byte aligned pieces).
struct Arena8 {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

struct Pade13 {
  double b[14];
  Pade13() {
    const int m = 13;
    double c = 1.0;
    double raw[14];
    raw[0] = 1.0;
    for (int j = 0; j < m; ++j) {
      c = c * (double)(m - j) / ((double)(2 * m - j) * (double)(j + 1));
      raw[j + 1] = c;
    }
    for (int j = 0; j <= m; ++j) b[j] = raw[j] / raw[m];
  }
};


// Host-side allocation fault injection for tests: FAB_FAULT=alloc:N makes the N-th
// workspace allocation counted from the moment the variable took its current value
// fail (the variable is read at every allocation, so a test can re-arm it between
// calls). The count is kept under a lock: server slot threads allocate concurrently.
std::mutex g_fault_mu;
bool fault_hit() {
  std::lock_guard<std::mutex> lock(g_fault_mu);
  static std::string seen;  // the FAB_FAULT value the count belongs to
  static int target = -1, count = 0;
  const char* e = getenv("FAB_FAULT");
  const std::string now = e ? e : "";
  if (now != seen) {
    seen = now;
    count = 0;
    target = now.compare(0, 6, "alloc:") == 0 ? atoi(now.c_str() + 6) : -1;
  }
  if (target < 1) return false;
  return ++count == target;
}

// ------------------------------------------------------------ profiling
enum ProfKind { PK_SPMV = 0, PK_UPDATE, PK_SKRED, PK_GEMVT, PK_SMALL, PK_COMBINE, PK_FUSED, PK_COUNT };
const char* kProfNames[PK_COUNT] = {"spmv_dots", "update", "sketch_reduce", "gemv_t", "small", "combine", "fused_step"};

struct Profiler {
  bool on = false;
  int only = -1;  // record one class only (-1: every class)
  bool wants(int kind) const { return on && (only < 0 || only == kind); }
  double total_ms[PK_COUNT] = {0};
  long long launches[PK_COUNT] = {0};
  std::vector<cudaEvent_t> pool;
  std::vector<int> kinds;  // kind of each recorded (start, end) pair
  size_t used = 0;         // events taken from the pool in the current solve
  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin_solve() {
    used = 0;
    kinds.clear();
  }
  // Called after the solve's stream has been synchronized.
  void end_solve() {
    for (size_t i = 0; i + 1 < used && i / 2 < kinds.size(); i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pool[i], pool[i + 1]) == cudaSuccess) {
        total_ms[kinds[i / 2]] += ms;
        launches[kinds[i / 2]] += 1;
      }
    }
    cudaGetLastError();
    used = 0;
    kinds.clear();
  }
};
Profiler g_prof;

}  // namespace


extern "C" {

void fab_params_default(fab_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->f = FAB_F_EXP;
  p->t = 1.0;
  p->m = 30;
  p->k = 2;
  p->s = 120;
  p->zeta = 8;
  p->sketch = FAB_SK_SPARSE_SIGN;
  p->seed = 1;
  p->method = FAB_SKETCHED_FAST;
  p->precision = FAB_FP64;
  p->lsqr_tol = 1e-6;
  p->lsqr_maxit = 0;
  p->stream = nullptr;
}

const char* fab_strerror(int code) {
  switch (code) {
    case FAB_OK: return "ok";
    case FAB_EINVAL: return "invalid argument";
    case FAB_ENOMEM: return "device allocation failed";
    case FAB_ECUDA: return "CUDA error";
    case FAB_ENUMERIC: return "non-finite value or no principal square root";
    case FAB_ETIMEOUT: return "bounded wait expired";
    case FAB_ENOTCONV: return "iteration limit reached";
    default: return "unknown error";
  }
}

int fab_create(fab_handle** out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
               const double* vals, int inputs_on_device) try {
  if (!out) return FAB_EINVAL;
  *out = nullptr;
  if (n < 1 || n >= (int64_t)1 << 31 || nnz < 0 || nnz >= (int64_t)1 << 31 || !rowptr || (nnz > 0 && (!colind || !vals)))
    return FAB_EINVAL;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(nnz);
  std::vector<double> va(nnz);
  if (inputs_on_device) {
    if (cudaMemcpy(rp.data(), rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (nnz > 0 && cudaMemcpy(ci.data(), colind, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (nnz > 0 && cudaMemcpy(va.data(), vals, nnz * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)) {
      cudaGetLastError();
      return FAB_ECUDA;
    }
  } else {
    memcpy(rp.data(), rowptr, (n + 1) * sizeof(int64_t));
    if (nnz > 0) {
      memcpy(ci.data(), colind, nnz * sizeof(int32_t));
      memcpy(va.data(), vals, nnz * sizeof(double));
    }
  }
  if (rp[0] != 0 || rp[n] != nnz) return FAB_EINVAL;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return FAB_EINVAL;
  for (int64_t e = 0; e < nnz; ++e)
    if (ci[e] < 0 || ci[e] >= n) return FAB_EINVAL;
  std::vector<int> rp32(n + 1);
  for (int64_t i = 0; i <= n; ++i) rp32[i] = (int)rp[i];
  fab_handle* h = new fab_handle();
  // Destroys the handle on every early return and on an exception (a host
  // allocation below), so that a create that fails leaves nothing behind.
  struct Owner {
    fab_handle* h;
    ~Owner() {
      if (h) fab_destroy(h);
    }
  } owner{h};
  h->n = (int)n;
  h->nnz = (int)nnz;
  h->ld = ((n + 31) / 32) * 32;
  if (fault_hit() || cudaMalloc(&h->d_rowptr, (n + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_colind, (nnz + kCsrPad) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_vals, (nnz + kCsrPad) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ENOMEM;
  }
  // the spare entries past nnz are read (never used) by the 16-byte aligned tile copies
  if (cudaMemset(h->d_colind + nnz, 0, kCsrPad * sizeof(int)) != cudaSuccess ||
      cudaMemset(h->d_vals + nnz, 0, kCsrPad * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(h->d_rowptr, rp32.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      (nnz > 0 && cudaMemcpy(h->d_colind, ci.data(), nnz * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) ||
      (nnz > 0 && cudaMemcpy(h->d_vals, va.data(), nnz * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  h->h_rowptr = new int[n + 1];
  memcpy(h->h_rowptr, rp32.data(), (n + 1) * sizeof(int));
  for (int64_t i = 0; i < n; ++i) h->max_row_nnz = std::max(h->max_row_nnz, rp32[i + 1] - rp32[i]);
  if (h->max_row_nnz >= 1 && h->max_row_nnz <= 8) {  // the one-pass steps' plan
    std::vector<int> tasks;
    std::vector<int2> crange;
    fab::fused_plan((int)n, rp32.data(), ci.data(), fab::sm_count() * 3 / 2, tasks, crange);
    if (cudaMalloc(&h->d_ftasks, tasks.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->d_fcrange, crange.size() * sizeof(int2)) != cudaSuccess ||
        cudaMemcpy(h->d_ftasks, tasks.data(), tasks.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_fcrange, crange.data(), crange.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return FAB_ENOMEM;
    }
  }
  // A warp of the row-per-lane form runs each group of 32 rows for its longest row; where
  // that leaves more than a fifth of the lanes idle (short rows of uneven length, as in a
  // power-law graph) the staged tiles are processed by nonzeros instead.
  double busy = 0.0, slots = 0.0;
  for (int64_t r0 = 0; r0 < n; r0 += 32) {
    int longest = 0;
    for (int64_t r = r0; r < std::min<int64_t>(n, r0 + 32); ++r) longest = std::max(longest, rp32[r + 1] - rp32[r]);
    busy += (double)(rp32[std::min<int64_t>(n, r0 + 32)] - rp32[r0]);
    slots += 32.0 * longest;
  }
  const int rc = fab::build_tiles(h, 256, kSpmvCap, busy < 0.8 * slots ? 2 : 1);
  if (rc != FAB_OK) return rc;
  owner.h = nullptr;
  *out = h;
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

void fab_destroy(fab_handle* h) {
  if (!h) return;
  if (h->owns_matrix) {
    cudaFree(h->d_rowptr);
    cudaFree(h->d_colind);
    cudaFree(h->d_vals);
    cudaFree(h->d_vals32);
    cudaFree(h->d_tiles);
    cudaFree(h->d_ftasks);
    cudaFree(h->d_fcrange);
    cudaFree(h->d_ell_col);
    cudaFree(h->d_ell_val);
    delete[] h->h_rowptr;
  }
  Buf* bufs[] = {&h->spat, &h->W32, &h->Wbf, &h->G, &h->shf, &h->scl, &h->W,     &h->H,   &h->sigma, &h->coef, &h->part, &h->counter, &h->gpart,
                 &h->skpart, &h->SV, &h->P,     &h->qr,  &h->tau,  &h->y,    &h->cvec,    &h->dense,
                 &h->piv,   &h->scal, &h->lsq,  &h->u,   &h->xbuf, &h->state, &h->whm, &h->wbuf, &h->fflags};
  for (Buf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->sbuf.p) cudaFree(h->sbuf.p);
  if (h->sq) fab_destroy(h->sq);
  cudaGetLastError();
  delete h;
}

}  // extern "C"

namespace {

#define CK(call)                              \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) {                  \
      cudaGetLastError();                     \
      return FAB_ECUDA;                       \
    }                                         \
  } while (0)

// Enqueue one kernel launch of class `kind`: counted, and bracketed by profiling
// events when profiling is on.
#define LK(kind, call)                                            \
  do {                                                            \
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;                     \
    if (g_prof.wants(kind)) {                                     \
      e0_ = g_prof.take();                                        \
      e1_ = g_prof.take();                                        \
      if (e0_ && e1_) cudaEventRecord(e0_, s);                    \
    }                                                             \
    cudaError_t e_ = (call);                                      \
    if (e_ == cudaSuccess && sync_check()) e_ = cudaStreamSynchronize(s); \
    if (e_ != cudaSuccess) {                                      \
      note_error(kind, e_, __LINE__);                             \
      cudaGetLastError();                                         \
      return FAB_ECUDA;                                           \
    }                                                             \
    if (e0_ && e1_) {                                             \
      cudaEventRecord(e1_, s);                                    \
      g_prof.kinds.push_back(kind);                               \
    }                                                             \
    ++g_launches;                                                 \
  } while (0)

// Debug aid: FAB_SYNC_CHECK=1 synchronizes after every launch so that a failing
// kernel is named by fab_last_error() instead of surfacing at a later call.
bool sync_check() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("FAB_SYNC_CHECK");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}
thread_local char g_errmsg[256] = "";
void note_error(int kind, cudaError_t e, int line) {
  snprintf(g_errmsg, sizeof(g_errmsg), "%s launch (fab_api.cu:%d): %s", kProfNames[kind], line, cudaGetErrorString(e));
}

thread_local int g_launches = 0;

// Host waits of a solve. A serving slot waits on a blocking-sync event so that
// its thread sleeps instead of spinning on a core the other slots need.
thread_local cudaEvent_t g_wait_event = nullptr;
cudaError_t wait_stream(cudaStream_t s) {
  if (!g_wait_event) return cudaStreamSynchronize(s);
  cudaError_t e = cudaEventRecord(g_wait_event, s);
  return e == cudaSuccess ? cudaEventSynchronize(g_wait_event) : e;
}

bool sketched(int method) {
  return method == FAB_SKETCHED_FAST || method == FAB_SKETCHED_LS || method == FAB_BG_LS || method == FAB_WHITEN;
}
// LSQR-based methods (Alg. 4, Alg. 3; whitening ends in Alg. 3 once whitened)
bool uses_lsqr(int method) { return method == FAB_SKETCHED_LS || method == FAB_BG_LS || method == FAB_WHITEN; }
// Whitening threshold of a FAB_WHITEN solve (0 selects the paper's 1000).
double whiten_kappa(const fab_params* p) { return p->whiten_kappa > 0.0 ? p->whiten_kappa : 1000.0; }

int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

int validate(const fab_handle* h, const fab_params* p) {
  if (p->f < 0 || p->f > 3) return FAB_EINVAL;
  if (p->method < 0 || p->method > 5) return FAB_EINVAL;
  if (p->m < 1 || p->m > kMaxM) return FAB_EINVAL;
  if (p->precision != FAB_FP64 && p->precision != FAB_MIXED) return FAB_EINVAL;
  if (p->method != FAB_ARNOLDI && (p->k < 1 || p->k > kMaxWindow)) return FAB_EINVAL;
  if (p->f == FAB_F_EXP && !isfinite(p->t)) return FAB_EINVAL;
  if (sketched(p->method)) {
    if (p->s < p->m + 1 || p->s > kMaxS) return FAB_EINVAL;
    if (p->sketch == FAB_SK_SPARSE_SIGN) {
      if (p->zeta < 1 || p->zeta > kMaxZeta || p->zeta > p->s) return FAB_EINVAL;
    } else if (p->sketch == FAB_SK_SRHT) {
      if (p->s > next_pow2(h->n)) return FAB_EINVAL;
    } else if (p->sketch == FAB_SK_GAUSSIAN) {
      if (p->precision != FAB_MIXED || p->m + 1 > kGaussMaxCols) return FAB_EINVAL;  // BF16 tensor-core sketch
    } else {
      return FAB_EINVAL;
    }
    if (uses_lsqr(p->method) && !(p->lsqr_tol > 0.0)) return FAB_EINVAL;
    // Alg. 1 and whitening need Theta w at every step (the Gaussian sketch is applied once, at the end)
    if ((p->method == FAB_BG_LS || p->method == FAB_WHITEN) && p->sketch == FAB_SK_GAUSSIAN) return FAB_EINVAL;
  }
  if (p->method == FAB_WHITEN && (!(p->whiten_kappa >= 0.0) || p->target_rel_err != 0.0)) return FAB_EINVAL;
  if (p->target_rel_err != 0.0) {  // growing m to a target: sketched methods, s embeds m_max + 1 columns
    if (!(p->target_rel_err > 0.0) || !sketched(p->method) || p->m_step < 1 || p->m_max < p->m ||
        p->m_max > kMaxM || p->s < p->m_max + 1)
      return FAB_EINVAL;
    if (p->sketch == FAB_SK_GAUSSIAN && p->m_max + 1 > kGaussMaxCols) return FAB_EINVAL;
  }
  return FAB_OK;
}

// Largest Krylov dimension a solve may reach (workspace sizing).
int m_cap(const fab_params* p) { return p->target_rel_err > 0.0 ? p->m_max : p->m; }

struct Ws {
  ColScale cs;
  float *W32, *wbuf;
  int* fflags;
  __nv_bfloat16 *Wbf, *G;
  double *W, *H, *sigma, *coef, *part, *gpart, *skpart, *SV, *qr, *tau, *y, *cvec, *scal, *u, *xbuf;
  double* mats[9];
  double *lv_v, *lv_w, *lv_x, *lv_z, *lv_coef, *lv_q, *unorm2, *one;
  double *wR, *wRi, *wT, *wcoef, *wnrm;  // FAB_WHITEN (ld m+1)
  unsigned* counter;
  int *P, *piv;
  DevState* st;
  // pinned host copies: the status word and a few scalars (a copy to pageable
  // memory would go through the CUDA runtime's shared staging buffer)
  DevState* hs;
  double* hd;
};
constexpr size_t kPinnedBytes = 512;  // DevState + 16 doubles

struct Need {
  Buf* b;
  size_t bytes;
};

// Doubles of one column's block partials of the sketch: k_update runs at most
// min(chunks, 8 blocks per SM) blocks of 256 threads.
size_t skpart_col_doubles(int n, int s) {
  const int nchunks = (n + kChunk - 1) / kChunk;
  return (size_t)std::max(1, std::min(nchunks, sm_count() * 8)) * (size_t)s;
}

// Where nothing reads the sketch before a pass of the basis loop ends (the Alg. 2
// paths of sketched_fast and sketched_ls with a sparse-sign or SRHT sketch), every
// column keeps its own block partials and one launch reduces the pass's columns,
// in place of a small latency-bound launch per step. Used while the partials take
// at most a quarter of the basis' bytes.
bool defer_sketch_reduce(const fab_handle* h, const fab_params* p) {
  if (p->method != FAB_SKETCHED_FAST && p->method != FAB_SKETCHED_LS) return false;
  if (p->sketch == FAB_SK_GAUSSIAN) return false;
  const int m = m_cap(p);
  const size_t bytes = (size_t)(m + 1) * skpart_col_doubles(h->n, p->s) * 8;
  const size_t basis = (size_t)h->ld * (m + 1) * (p->precision == FAB_MIXED ? 4 : 8);
  return bytes <= basis / 4;
}

// One-pass basis steps (fused.cu): the FP32 basis of Alg. 2 (sketched_fast, sketched_ls,
// Alg. 5) with a sign sketch or none, rows of at most 8 nonzeros, and the handle's switch on.
bool fused_steps(const fab_handle* h, const fab_params* p) {
  if (p->precision != FAB_MIXED || !h->fuse || h->max_row_nnz > 8 || h->max_row_nnz < 1 || !h->d_ftasks)
    return false;
  if (p->method == FAB_NOPROJ) return true;
  if (p->method != FAB_SKETCHED_FAST && p->method != FAB_SKETCHED_LS) return false;
  return p->sketch == FAB_SK_SRHT || p->sketch == FAB_SK_SPARSE_SIGN;
}

// The workspace a solve needs (buffer, bytes), shared by allocation and admission.
int ws_needs(fab_handle* h, const fab_params* p, Need* out) {
  const int m = m_cap(p), s = sketched(p->method) ? p->s : 1;
  const int n = h->n;
  const size_t ld = (size_t)h->ld;
  const int ntiles = (n + kTileRows - 1) / kTileRows;
  const int nchunks = (n + kChunk - 1) / kChunk;
  const size_t part_blocks = (size_t)sm_count() * kMaxPartBlocks;
  const bool gauss = p->precision == FAB_MIXED && p->sketch == FAB_SK_GAUSSIAN && sketched(p->method);
  const Need need[] = {
      {p->precision == FAB_MIXED ? &h->W32 : &h->W, ld * (m + 1) * (p->precision == FAB_MIXED ? 4 : 8)},
      {&h->Wbf, gauss ? gauss_B_bytes(n, m + 1) : 0},  // hi and lo terms, K-blocked
      {&h->G, gauss ? gauss_G_bytes(n, s) : 0},
      {&h->H, (size_t)(m + 1) * m * 8},
      {&h->sigma, (size_t)(m + 1) * 8},
      {&h->shf, (size_t)(m + 1) * 4},
      {&h->scl, (size_t)(m + 1) * 8},
      {&h->coef, (size_t)(m + 1) * 8},
      {&h->part, part_blocks * (kMaxWindow + 1) * 8},
      {&h->counter, 64},
      {&h->gpart, std::max((size_t)ntiles * (m + 1) * 8, gauss ? gauss_partial_bytes(n, s, m + 1) : (size_t)0)},
      {&h->skpart, defer_sketch_reduce(h, p) ? (size_t)(m + 1) * skpart_col_doubles(n, s) * 8 : (size_t)nchunks * s * 8},
      {&h->SV, (size_t)s * (m + 1) * 8},
      {&h->P, (size_t)s * 4},
      {&h->spat, (sketched(p->method) && p->sketch == FAB_SK_SPARSE_SIGN) ? sparse_table_bytes(n, s, p->zeta) : 0},
      {&h->qr, (size_t)s * (m + 1) * 8},
      {&h->tau, (size_t)(m + 1) * 8},
      {&h->y, (size_t)(m + 1) * 8},
      {&h->cvec, (size_t)2 * (m + 1) * 8},  // c and, growing m, the previous c
      {&h->dense, (size_t)9 * m * m * 8},
      {&h->piv, (size_t)(m + 1) * 4},
      {&h->scal, 64 * 8},
      {&h->lsq, (size_t)6 * (m + 1) * 8},
      {&h->state, sizeof(DevState)},
      {&h->u, uses_lsqr(p->method) ? (size_t)n * 8 : 0},
      {&h->xbuf, (size_t)n * 8},
      {&h->whm, p->method == FAB_WHITEN ? (3 * (size_t)(m + 1) * (m + 1) + (m + 1) + 8) * 8 : 0},
      {&h->wbuf, fused_steps(h, p) ? ld * 2 * 4 : 0},
      {&h->fflags, fused_steps(h, p) ? (size_t)nchunks * 4 : 0},
  };
  const int cnt = (int)(sizeof(need) / sizeof(need[0]));
  for (int i = 0; i < cnt; ++i) out[i] = need[i];
  return cnt;
}

int ensure_ws(fab_handle* h, const fab_params* p, Ws& ws) {
  Need need[64];
  const int cnt = ws_needs(h, p, need);
  const int n = h->n;
  const int m = m_cap(p);
  for (int i = 0; i < cnt; ++i) {
    auto& q = need[i];
    if (q.bytes == 0 && (q.b == &h->u || q.b == &h->xbuf || q.b == &h->whm || q.b == &h->wbuf || q.b == &h->fflags))
      continue;  // allocated on demand
    const bool grow = q.b->bytes < (q.bytes ? q.bytes : 16);
    if (grow) {
      // a regrown buffer starts uninitialized (and a failed growth leaves none):
      // the contents cached with the handle are drawn again
      if (q.b == &h->P) h->P_npad = -1;
      if (q.b == &h->spat) h->spat_n = -1;
      if (q.b == &h->G) h->G_n = -1;
      if (fault_hit()) {  // as a cudaMalloc that fails after ensure() freed the old buffer
        cudaFree(q.b->p);
        q.b->p = nullptr;
        q.b->bytes = 0;
        return FAB_ENOMEM;
      }
    }
    if (!ensure(*q.b, q.bytes)) return FAB_ENOMEM;
    if (grow && q.b == &h->counter) CK(cudaMemset(h->counter.p, 0, h->counter.bytes));
  }
  (void)n;
  ws.W = ptr<double>(h->W);
  ws.W32 = ptr<float>(h->W32);
  ws.wbuf = ptr<float>(h->wbuf);
  ws.fflags = ptr<int>(h->fflags);
  ws.Wbf = ptr<__nv_bfloat16>(h->Wbf);
  ws.G = ptr<__nv_bfloat16>(h->G);
  ws.H = ptr<double>(h->H);
  ws.sigma = ptr<double>(h->sigma);
  ws.cs = ColScale{ptr<double>(h->sigma), ptr<int>(h->shf), ptr<double>(h->scl)};
  ws.coef = ptr<double>(h->coef);
  ws.part = ptr<double>(h->part);
  ws.gpart = ptr<double>(h->gpart);
  ws.skpart = ptr<double>(h->skpart);
  ws.SV = ptr<double>(h->SV);
  ws.qr = ptr<double>(h->qr);
  ws.tau = ptr<double>(h->tau);
  ws.y = ptr<double>(h->y);
  ws.cvec = ptr<double>(h->cvec);
  ws.scal = ptr<double>(h->scal);
  ws.u = ptr<double>(h->u);
  for (int i = 0; i < 9; ++i) ws.mats[i] = ptr<double>(h->dense) + (size_t)i * m * m;
  double* l = ptr<double>(h->lsq);
  ws.lv_v = l;
  ws.lv_w = l + (m + 1);
  ws.lv_x = l + 2 * (m + 1);
  ws.lv_z = l + 3 * (m + 1);
  ws.lv_coef = l + 4 * (m + 1);
  ws.lv_q = l + 5 * (m + 1);
  ws.unorm2 = ws.scal + 8;
  ws.one = ws.scal + 9;
  {
    double* w = ptr<double>(h->whm);
    const size_t sq = (size_t)(m + 1) * (m + 1);
    ws.wR = w;
    ws.wRi = w ? w + sq : nullptr;
    ws.wT = w ? w + 2 * sq : nullptr;
    ws.wcoef = w ? w + 3 * sq : nullptr;
    ws.wnrm = w ? w + 3 * sq + (m + 1) : nullptr;
  }
  ws.counter = ptr<unsigned>(h->counter);
  ws.P = ptr<int>(h->P);
  ws.piv = ptr<int>(h->piv);
  ws.st = ptr<DevState>(h->state);
  if (!h->h_pinned) {
    if (cudaHostAlloc(&h->h_pinned, kPinnedBytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      h->h_pinned = nullptr;
      return FAB_ENOMEM;
    }
  }
  ws.hs = reinterpret_cast<DevState*>(h->h_pinned);
  ws.hd = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(h->h_pinned) + 256);
  return FAB_OK;
}

// exp(M) e_1 into c; M (ld m) is overwritten. Scaling and squaring with the [13/13]
// Pade approximant r_13 (Higham 2005): X = M / 2^sq with ||X||_1 <= theta_13, exp(M) =
// (r_13(X))^(2^sq), r_13 = (V - U)^{-1} (V + U), U odd and V even in X, both formed from
// X^2, X^4, X^6 (6 many-block GEMMs). The solve is the blocked cluster LU of the
// Denman-Beavers path with an m-column substitution; the squarings are GEMMs.
int expm_e1(Ws& ws, int m, const int* mdev, double* c, int* squarings, cudaStream_t s) {
  const double* b = pade13_b();
  double *X = ws.mats[0], *X2 = ws.mats[1], *X4 = ws.mats[2], *X6 = ws.mats[3], *T = ws.mats[4], *U = ws.mats[5],
         *V = ws.mats[6], *R = ws.mats[7], *R2 = ws.mats[8];
  LK(PK_SMALL, launch_norm1(X, m, mdev, ws.scal + 10, s));
  CK(cudaMemcpyAsync(ws.hd, ws.scal + 10, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(wait_stream(s));
  const double nrm = ws.hd[0];
  if (!isfinite(nrm)) return FAB_ENUMERIC;
  const int sq = nrm > kTheta13 ? (int)ceil(log2(nrm / kTheta13)) : 0;
  if (sq > 0) LK(PK_SMALL, launch_lincomb(X, X, nullptr, nullptr, nullptr, ldexp(1.0, -sq), 0, 0, 0, 0.0, m, mdev, m, s));
  LK(PK_SMALL, launch_gemm(X2, X, X, m, mdev, m, 1.0, 0.0, s));
  LK(PK_SMALL, launch_gemm(X4, X2, X2, m, mdev, m, 1.0, 0.0, s));
  LK(PK_SMALL, launch_gemm(X6, X4, X2, m, mdev, m, 1.0, 0.0, s));
  // U = X (X^6 (b13 X^6 + b11 X^4 + b9 X^2) + b7 X^6 + b5 X^4 + b3 X^2 + b1 I)
  LK(PK_SMALL, launch_lincomb(T, X6, X4, X2, nullptr, b[13], b[11], b[9], 0, 0.0, m, mdev, m, s));
  LK(PK_SMALL, launch_gemm(R, X6, T, m, mdev, m, 1.0, 0.0, s));
  LK(PK_SMALL, launch_lincomb(R, R, X6, X4, X2, 1.0, b[7], b[5], b[3], b[1], m, mdev, m, s));
  LK(PK_SMALL, launch_gemm(U, X, R, m, mdev, m, 1.0, 0.0, s));
  // V = X^6 (b12 X^6 + b10 X^4 + b8 X^2) + b6 X^6 + b4 X^4 + b2 X^2 + b0 I
  LK(PK_SMALL, launch_lincomb(T, X6, X4, X2, nullptr, b[12], b[10], b[8], 0, 0.0, m, mdev, m, s));
  LK(PK_SMALL, launch_gemm(V, X6, T, m, mdev, m, 1.0, 0.0, s));
  LK(PK_SMALL, launch_lincomb(V, V, X6, X4, X2, 1.0, b[6], b[4], b[2], b[0], m, mdev, m, s));
  // (V - U) R = V + U
  LK(PK_SMALL, launch_lincomb(T, V, U, nullptr, nullptr, 1.0, -1.0, 0, 0, 0.0, m, mdev, m, s));
  LK(PK_SMALL, launch_lincomb(R, V, U, nullptr, nullptr, 1.0, 1.0, 0, 0, 0.0, m, mdev, m, s));
  LK(PK_SMALL, launch_lu_fast(T, m, mdev, m, ws.piv, ws.scal + 11, ws.st, s));
  LK(PK_SMALL, launch_lu_solve(T, m, ws.piv, mdev, m, R, m, 0, s));
  for (int i = 0; i < sq; ++i) {
    LK(PK_SMALL, launch_gemm(R2, R, R, m, mdev, m, 1.0, 0.0, s));
    std::swap(R, R2);
  }
  CK(cudaMemcpyAsync(c, R, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (squarings) *squarings = sq;
  return FAB_OK;
}

// f(M) e_1 for f = sqrt (want_sqrt) or inverse sqrt by the scaled product-form
// Denman-Beavers iteration; M (ld m) is overwritten.
int sqrtm_e1(Ws& ws, int m, const int* mdev, double* c, int want_sqrt, int* iters, cudaStream_t s) {
  double *M = ws.mats[0], *T = ws.mats[1], *Minv = ws.mats[2];
  LK(PK_SMALL, launch_first_column(want_sqrt ? M : nullptr, mdev, c, s));
  const int maxit = 100;
  double err = INFINITY;
  int extra = -1;
  for (int it = 0; it < maxit; ++it) {
    CK(cudaMemcpyAsync(T, M, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    LK(PK_SMALL, launch_lu_fast(T, m, mdev, m, ws.piv, ws.scal + 11, ws.st, s));
    LK(PK_SMALL, launch_lu_solve(T, m, ws.piv, mdev, m, Minv, m, 1, s));
    LK(PK_SMALL, launch_db_update(M, Minv, m, mdev, c, ws.scal + 11, err > 1e-2 ? 1 : 0, ws.st, s, m, ws.part,
                                  ws.counter));
    DevState& hs = *ws.hs;
    CK(cudaMemcpyAsync(&hs, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(wait_stream(s));
    if (hs.status != FAB_OK) return hs.status;
    err = hs.scal[1];
    if (iters) *iters = it + 1;
    if (extra >= 0) return FAB_OK;
    if (err <= 1e-13 * sqrt((double)m)) extra = 0;  // one more step after convergence
  }
  return FAB_ENOTCONV;
}

}  // namespace

// One solve with the basis stored as TV (double: FP64 path; float: mixed path).
template <typename TV>
int apply_impl(fab_handle* h, const fab_params* p, const double* b, double* x, int bx_on_device, fab_stats* stats,
               Ws& ws, TV* W, const void* vals) {
  int rc = FAB_OK;
  cudaStream_t s = (cudaStream_t)p->stream;
  constexpr bool kMixed = sizeof(TV) == 4;
  // every device buffer this solve touches must exist before the first launch
  if (!W || !vals || !ws.H || !ws.st || !ws.SV || !ws.part || !ws.gpart ||
      (p->sketch == FAB_SK_GAUSSIAN && sketched(p->method) && (!ws.Wbf || !ws.G)) ||
      (uses_lsqr(p->method) && !ws.u) || (p->method == FAB_WHITEN && !ws.wR))
    return FAB_ENOMEM;
  const int n = h->n, k = p->k;
  const int mcap = m_cap(p);   // largest dimension this solve may grow to
  const bool grow = p->target_rel_err > 0.0;
  int m = p->m;                // current dimension
  const int64_t ld = h->ld;
  const int ldh = mcap + 1;
  const bool sk_on = sketched(p->method);
  const bool whiten = p->method == FAB_WHITEN;
  const int ldr = mcap + 1;  // whitening: R, R^{-1} and scratch are ldr x ldr
  const int* mdev = &ws.st->m_used;
  Csr A{h->n, h->nnz, h->d_rowptr, h->d_colind, vals, h->d_tiles, h->ntiles, h->tile_staged};
  h->has_state = 0;
  g_launches = 0;
  if (g_prof.on) g_prof.begin_solve();

  cudaEvent_t ev[4];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
    }
  } guard{ev};

  CK(cudaEventRecord(ev[0], s));
  LK(PK_SMALL, launch_state_reset(ws.st, m, s));
  CK(cudaMemsetAsync(ws.counter, 0, 64, s));
  CK(cudaMemsetAsync(ws.H, 0, (size_t)ldh * mcap * sizeof(double), s));
  CK(cudaMemsetAsync(ws.y, 0, (size_t)(mcap + 1) * sizeof(double), s));
  if (kMixed) {  // b is FP64 (host or device): stage it, then round to FP32 in column 0
    if ((h->xbuf.bytes < (size_t)n * 8 && fault_hit()) || !ensure(h->xbuf, (size_t)n * 8)) return FAB_ENOMEM;
    CK(cudaMemcpyAsync(h->xbuf.p, b, (size_t)n * sizeof(double), cudaMemcpyDefault, s));
    LK(PK_SMALL, launch_to_f32(n, ptr<double>(h->xbuf), reinterpret_cast<float*>(W), s));
  } else {
    CK(cudaMemcpyAsync(W, b, (size_t)n * sizeof(double), cudaMemcpyDefault, s));
  }

  SketchDev sk;
  memset(&sk, 0, sizeof(sk));
  sk.kind = SK_NONE;
  double sk_scale = 1.0;
  if (sk_on) {
    sk.kind = p->sketch == FAB_SK_SRHT ? SK_SRHT : (p->sketch == FAB_SK_GAUSSIAN ? SK_GAUSS : SK_SPARSE);
    sk.s = p->s;
    sk.zeta = p->zeta;
    sk.chunk_log2 = kChunkLog2;
    sk.nchunks = (n + kChunk - 1) / kChunk;
    sk.st_rows = rng_state(p->seed, 1);
    sk.st_signs = rng_state(p->seed, 2);
    sk.st_D = rng_state(p->seed, 3);
    sk.P = ws.P;
    sk.part = ws.skpart;
    if (sk.kind == SK_SRHT) {
      const int64_t npad = next_pow2(n);
      if (h->P_npad != npad || h->P_s != p->s || h->P_seed != p->seed) {
        LK(PK_SMALL, launch_srht_sample(npad, p->s, rng_state(p->seed, 4), ws.P, s));
        h->P_npad = npad;
        h->P_s = p->s;
        h->P_seed = p->seed;
      }
      sk_scale = 1.0 / sqrt((double)p->s);
    } else if (sk.kind == SK_GAUSS) {
      sk.Wbf = ws.Wbf;
      sk.bf_cpad = gauss_cpad(mcap + 1);
      // the copy's rows past n (the end of the last K block) enter the products: zero them
      CK(cudaMemsetAsync(ws.Wbf + (size_t)(gauss_nkb(n) - 1) * 2 * sk.bf_cpad * 64, 0,
                         (size_t)2 * sk.bf_cpad * 64 * sizeof(__nv_bfloat16), s));
      if (h->G_n != n || h->G_s != p->s || h->G_seed != p->seed) {  // G (BF16, s x n) cached per handle
        LK(PK_SMALL, launch_gauss_generate(p->s, n, rng_state(p->seed, 5), ws.G, s));
        h->G_n = n;
        h->G_s = p->s;
        h->G_seed = p->seed;
      }
    } else {
      sk_scale = 1.0 / sqrt((double)p->zeta);
      unsigned short* pat = ptr<unsigned short>(h->spat);
      if (h->spat_n != n || h->spat_s != p->s || h->spat_zeta != p->zeta || h->spat_seed != p->seed) {
        h->spat_n = -1;  // (re)drawn once per (n, s, zeta, seed) and kept with the handle
        LK(PK_SMALL, launch_sparse_pattern(n, sk, pat, s));
        h->spat_n = n;
        h->spat_s = p->s;
        h->spat_zeta = p->zeta;
        h->spat_seed = p->seed;
      }
      sk.pat = pat;
    }
  }
  SketchDev none;
  memset(&none, 0, sizeof(none));
  none.kind = SK_NONE;
  // deferred sketch reduce: column c's partials at ws.skpart + c * colstride, and the
  // number of blocks that wrote them
  const bool defer = sk_on && sk.kind != SK_GAUSS && defer_sketch_reduce(h, p);
  const size_t colstride = defer ? skpart_col_doubles(n, p->s) : 0;
  std::vector<int> col_parts(defer ? m_cap(p) + 1 : 0, 0);
  int red_from = 0;  // first column whose deferred reduce is pending

  if (p->method == FAB_BG_LS) {  // Alg. 1 start: p = Theta b, r_11 = ||p||, sigma_0 = 1 / r_11
    LK(PK_UPDATE, launch_update(n, W, ld, 0, 0, 0, ws.coef, ws.H, ldh, ws.cs, 0, ws.part, ws.counter, sk,
                                ws.st, s));
    LK(PK_SKRED, launch_sketch_reduce(sk, nullptr, 0, sk_scale, ws.SV, ws.st, s));
    LK(PK_SMALL, launch_bg_orth(ws.SV, p->s, 0, ws.H, ldh, ws.coef, ws.cs, ws.st, s));
  } else {
    // start vector: ||b||, sigma_0, sketch of b (Gaussian: its BF16 copy)
    LK(PK_UPDATE, launch_update(n, W, ld, 0, 0, 0, ws.coef, ws.H, ldh, ws.cs, 1 | 2, ws.part, ws.counter,
                                sk_on ? sk : none, ws.st, s));
    if (defer)
      col_parts[0] = sk.nparts;
    else if (sk_on && sk.kind != SK_GAUSS)
      LK(PK_SKRED, launch_sketch_reduce(sk, ws.sigma, 0, sk_scale, ws.SV, ws.st, s));
    if (whiten)  // R = (||Theta v_1||), Q = Theta v_1 / r_11
      LK(PK_SMALL, launch_wh_check(ws.SV, p->s, 0, ws.qr, ws.wR, ws.wRi, ws.wT, ldr, ws.H, ldh, whiten_kappa(p),
                                   ws.wcoef, ws.wnrm, ws.cs, ws.st, s));
  }

  const int ntiles = (n + kTileRows - 1) / kTileRows;
  int c_done = 0;          // basis columns 1..c_done are built
  int m_prev = 0;          // dimension of the previous solution (growing m)
  int qr_cols = 0;         // columns of ws.qr already factored by this solve's previous pass
  double err_est = 0.0;
  int rc_final = FAB_OK;
  int lsqr_iters = 0, fh_iters = 0;
  DevState& hs = *ws.hs;
  int mu = 0;
  int wh = 0;  // FAB_WHITEN: > 0 once the basis was whitened at wh columns
  // one-pass basis steps: the FP32 Alg. 2 loop on a matrix with short rows
  const bool fused = kMixed && fused_steps(h, p) && ws.wbuf && ws.fflags && h->d_ell_col &&
                     (!sk_on || sk.kind == SK_SRHT || sk.kind == SK_SPARSE);
  const FusePlan fplan{ws.fflags,   h->d_ftasks, h->d_fcrange,     h->d_ell_col,
                       h->d_ell_val, h->ld,       h->max_row_nnz,    fused ? h->stall_pass : 0,
                       h->stall_polls};
  if (fused) h->stall_pass = 0;  // the hook is one-shot
  if (fused) CK(cudaMemsetAsync(ws.fflags, 0, (size_t)((n + kChunk - 1) / kChunk) * sizeof(int), s));
  for (;;) {  // one pass per dimension m (a single pass unless m grows to a target)
  if constexpr (kMixed) {
    if (fused && c_done < m) {
      // Pass c updates column c-1 (from the second pass of this run on) and multiplies
      // it by A; the run's last column gets its update, norm and sketch from k_update.
      const int c0 = c_done + 1;
      float* wb[2] = {ws.wbuf, ws.wbuf + ld};
      SketchDev& skf = sk_on ? sk : none;
      for (int c = c0; c <= m; ++c) {
        const bool upd = c > c0;
        const int j0 = std::max(0, c - k), kw = c - j0;
        const int j0u = std::max(0, c - 1 - k), kwu = upd ? (c - 1) - j0u : 0;
        const float* wprev = upd ? wb[(c - 1) & 1] : W + (size_t)(c - 1) * ld;
        float* wnext = c == m ? W + (size_t)c * ld : wb[c & 1];
        if (defer) skf.part = ws.skpart + (size_t)(c - 1) * colstride;
        LK(PK_FUSED, launch_fused_step(A, W, ld, c, upd ? 1 : 0, j0u, kwu, j0, kw, wprev, wnext, ws.cs, ws.H, ldh,
                                       ws.coef, ws.part, ws.counter, skf, ws.st, fplan, s));
        if (upd && sk_on) {
          if (defer)
            col_parts[c - 1] = skf.nparts;
          else
            LK(PK_SKRED, launch_sketch_reduce(sk, ws.sigma, c - 1, sk_scale, ws.SV + (size_t)(c - 1) * p->s, ws.st, s));
        }
      }
      const int j0 = std::max(0, m - k), kw = m - j0;
      if (sk_on) {
        if (defer) sk.part = ws.skpart + (size_t)m * colstride;
        LK(PK_UPDATE, launch_update(n, W, ld, m, j0, kw, ws.coef, ws.H, ldh, ws.cs, 1, ws.part, ws.counter, sk,
                                    ws.st, s));
        if (defer)
          col_parts[m] = sk.nparts;
        else
          LK(PK_SKRED, launch_sketch_reduce(sk, ws.sigma, m, sk_scale, ws.SV + (size_t)m * p->s, ws.st, s));
      } else {
        LK(PK_UPDATE, launch_update_plain(n, W, ld, m, j0, kw, ws.coef, ws.H, ldh, ws.cs, 1, ws.part, ws.counter,
                                          ws.st, s));
      }
      c_done = m;
    }
  }
  for (int c = c_done + 1; c <= m; ++c) {
    if (p->method == FAB_BG_LS) {
      // Alg. 1: w = A v_{c-1}; p = Theta w; sketched Gram-Schmidt step; the same
      // coefficients on the long vector: W_c <- W_c - sum_j coef_j W_j
      LK(PK_SPMV, launch_spmv_dots(A, W, ld, c, 0, 0, ws.cs, ws.H, ldh, ws.coef, ws.part, ws.counter, ws.st, s));
      LK(PK_UPDATE, launch_update(n, W, ld, c, 0, 0, ws.coef, ws.H, ldh, ws.cs, 0, ws.part, ws.counter, sk,
                                  ws.st, s));
      LK(PK_SKRED, launch_sketch_reduce(sk, ws.cs.scl, c, sk_scale, ws.SV + (size_t)c * p->s, ws.st, s));
      LK(PK_SMALL, launch_bg_orth(ws.SV, p->s, c, ws.H, ldh, ws.coef, ws.cs, ws.st, s));
      LK(PK_UPDATE, launch_update(n, W, ld, c, 0, c, ws.coef, ws.H, ldh, ws.cs, 0, ws.part, ws.counter, none,
                                  ws.st, s));
    } else if (whiten) {
      // Both step sequences are queued; the gates let one of them run (1: Alg. 2
      // until the basis is whitened, 2: Alg. 1 afterwards), so the switch needs
      // no host round trip.
      const int j0 = std::max(0, c - k), kw = c - j0;
      LK(PK_SPMV, launch_spmv_dots(A, W, ld, c, j0, kw, ws.cs, ws.H, ldh, ws.coef, ws.part, ws.counter, ws.st,
                                   s, 1));
      LK(PK_UPDATE, launch_update(n, W, ld, c, j0, kw, ws.coef, ws.H, ldh, ws.cs, 1, ws.part, ws.counter, sk,
                                  ws.st, s, 1));
      LK(PK_SKRED, launch_sketch_reduce(sk, ws.sigma, c, sk_scale, ws.SV + (size_t)c * p->s, ws.st, s, 1));
      LK(PK_SMALL, launch_wh_check(ws.SV, p->s, c, ws.qr, ws.wR, ws.wRi, ws.wT, ldr, ws.H, ldh, whiten_kappa(p),
                                   ws.wcoef, ws.wnrm, ws.cs, ws.st, s));
      LK(PK_COMBINE, launch_whiten_column(n, W, ld, c, ws.wcoef, ws.st, s));
      LK(PK_SPMV, launch_spmv_dots(A, W, ld, c, 0, 0, ws.cs, ws.H, ldh, ws.coef, ws.part, ws.counter, ws.st,
                                   s, 2));
      LK(PK_UPDATE, launch_update(n, W, ld, c, 0, 0, ws.coef, ws.H, ldh, ws.cs, 0, ws.part, ws.counter, sk,
                                  ws.st, s, 2));
      LK(PK_SKRED, launch_sketch_reduce(sk, ws.cs.scl, c, sk_scale, ws.SV + (size_t)c * p->s, ws.st, s, 2));
      LK(PK_SMALL, launch_bg_orth(ws.SV, p->s, c, ws.H, ldh, ws.coef, ws.cs, ws.st, s, ws.wRi, ldr, 2));
      LK(PK_UPDATE, launch_update(n, W, ld, c, 0, c, ws.coef, ws.H, ldh, ws.cs, 0, ws.part, ws.counter, none,
                                  ws.st, s, 2));
    } else if (p->method == FAB_ARNOLDI) {
      LK(PK_SPMV, launch_spmv_dots(A, W, ld, c, 0, 0, ws.cs, ws.H, ldh, ws.coef, ws.part, ws.counter, ws.st, s));
      double* Hcol = ws.H + (size_t)ldh * (c - 1);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        LK(PK_GEMVT, launch_gemv_t(n, (const TV*)W, ld, 0, c, (const TV*)W + (size_t)c * ld, ws.gpart, ntiles, ws.st, s));
        LK(PK_GEMVT, launch_reduce_cols(ws.gpart, ntiles, c, ws.sigma, 0, ws.cs.scl + c, Hcol, pass, ws.coef,
                                        ws.st, s));
        LK(PK_UPDATE, launch_update(n, W, ld, c, 0, c, ws.coef, ws.H, ldh, ws.cs, pass == 1 ? 1 : 0, ws.part,
                         ws.counter, none, ws.st, s));
      }
    } else {
      const int j0 = std::max(0, c - k), kw = c - j0;
      LK(PK_SPMV, launch_spmv_dots(A, W, ld, c, j0, kw, ws.cs, ws.H, ldh, ws.coef, ws.part, ws.counter, ws.st,
                          s));
      if (sk_on) {  // window update, norm and the sketch of the new column in one pass
        if (defer) sk.part = ws.skpart + (size_t)c * colstride;
        LK(PK_UPDATE, launch_update(n, W, ld, c, j0, kw, ws.coef, ws.H, ldh, ws.cs, 1, ws.part, ws.counter, sk,
                                    ws.st, s));
        if (defer)
          col_parts[c] = sk.nparts;
        else if (sk.kind != SK_GAUSS)
          LK(PK_SKRED, launch_sketch_reduce(sk, ws.sigma, c, sk_scale, ws.SV + (size_t)c * p->s, ws.st, s));
      } else {  // no sketch (Alg. 5): the lean kernel, all of a row group's loads in flight at once
        LK(PK_UPDATE, launch_update_plain(n, W, ld, c, j0, kw, ws.coef, ws.H, ldh, ws.cs, 1, ws.part,
                                          ws.counter, ws.st, s));
      }
    }
  }
  c_done = m;
  if (defer) {  // the pass's sketch columns, one launch per run of equal block counts
    sk.part = ws.skpart;
    for (int c0 = red_from; c0 <= m;) {
      int c1 = c0;
      while (c1 < m && col_parts[c1 + 1] == col_parts[c0]) ++c1;
      LK(PK_SKRED, launch_sketch_reduce_cols(sk, colstride, c0, c1 - c0 + 1, col_parts[c0], ws.sigma, sk_scale, ws.SV,
                                             ws.st, s));
      c0 = c1 + 1;
    }
    red_from = m + 1;
  }
  if (sk_on && sk.kind == SK_GAUSS)  // Theta V_{m+1} = G (BF16 basis) on the tensor cores, FP64 finish
    LK(PK_SKRED, launch_gauss_sketch(ws.G, ws.Wbf, gauss_cpad(mcap + 1), n, p->s, m + 1, ws.sigma, ws.gpart, ws.SV,
                                     ws.st, s));
  CK(cudaEventRecord(ev[1], s));
  CK(cudaMemcpyAsync(&hs, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(wait_stream(s));
  if (hs.status != FAB_OK) return hs.status;
  mu = hs.m_used;
  h->last_m = m;
  h->last_ldh = ldh;
  h->last_s = sk_on ? p->s : 0;
  h->last_sketched = sk_on ? 1 : 0;
  h->last_mixed = kMixed ? 1 : 0;
  h->has_state = 1;  // the basis, H and the sketch can be inspected from here on
  if (mu == 0) {  // b = 0
    CK(cudaMemsetAsync(ws.cvec, 0, (size_t)m * sizeof(double), s));
    if (bx_on_device) {
      CK(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), s));
    } else {
      memset(x, 0, (size_t)n * sizeof(double));
    }
    CK(wait_stream(s));
    h->has_state = 1;
    if (stats) {
      memset(stats, 0, sizeof(*stats));
    }
    return FAB_OK;
  }
  const bool breakdown = mu < m;
  wh = whiten ? hs.wh : 0;
  const bool lsqr = !breakdown && (p->method == FAB_SKETCHED_LS || p->method == FAB_BG_LS || wh > 0);
  const double* yptr = nullptr;
  if (!breakdown && p->method == FAB_SKETCHED_FAST) {
    // y = argmin || Theta V_m z - Theta v_{m+1} || (sketch-and-solve form of eq. sFOM).
    // Growing m: the previous pass's columns stay factored and its extra column
    // (Theta v_{m_prev+1}, already transformed) is the next column to factor, so only
    // the new sketch columns are copied and the QR continues at column m_prev.
    const bool inc = qr_cols > 0 && qr_cols <= mu && qr_cluster_fits(p->s, m + 1);
    const int q0 = inc ? qr_cols : 0, fresh = inc ? qr_cols + 1 : 0;
    CK(cudaMemcpyAsync(ws.qr + (size_t)fresh * p->s, ws.SV + (size_t)fresh * p->s,
                       (size_t)p->s * (mu + 1 - fresh) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    LK(PK_SMALL, launch_qr(ws.qr, p->s, p->s, mdev, m, 1, ws.tau, ws.st, s, q0, fresh));
    LK(PK_SMALL, launch_kappa_diag(ws.qr, p->s, mdev, m, ws.st, s));
    qr_cols = mu;
    LK(PK_SMALL, launch_trsv(ws.qr, p->s, mdev, ws.qr + (size_t)mu * p->s, ws.y, 0, nullptr, s, m));
    yptr = ws.y;
  } else if (lsqr) {
    if (p->method == FAB_SKETCHED_LS) {
      // Blendenpik: R from the QR of Theta V_m; LSQR on V_m R^{-1} u ~ v_{m+1}; y = R^{-1} u
      // (growing m: the previous pass's columns stay factored, as above)
      const bool inc = qr_cols > 0 && qr_cols <= mu && qr_cluster_fits(p->s, m);
      const int q0 = inc ? qr_cols : 0;
      CK(cudaMemcpyAsync(ws.qr + (size_t)q0 * p->s, ws.SV + (size_t)q0 * p->s, (size_t)p->s * (mu - q0) * sizeof(double),
                         cudaMemcpyDeviceToDevice, s));
      LK(PK_SMALL, launch_qr(ws.qr, p->s, p->s, mdev, m, 0, ws.tau, ws.st, s, q0, q0));
      LK(PK_SMALL, launch_kappa_diag(ws.qr, p->s, mdev, m, ws.st, s));
      qr_cols = mu;
    } else if (wh > 0) {
      // Alg. 3 on the whitened basis: LSQR on the stored columns with the implicit
      // R_{wh-1}^{-1} as right preconditioner; u is y in whitened coordinates
      LK(PK_SMALL, launch_wh_precond(ws.wR, ldr, wh, ws.qr, p->s, mdev, m, s));
    } else {
      // Alg. 3: LSQR on V_m itself (the Alg. 1 basis is well conditioned): R = I
      LK(PK_SMALL, launch_set_identity(ws.qr, p->s, mdev, m, s));
    }
    ws.hd[8] = 1.0;
    CK(cudaMemcpyAsync(ws.one, ws.hd + 8, sizeof(double), cudaMemcpyHostToDevice, s));
    LK(PK_SMALL, launch_state_clear_flag(ws.st, s));  // a previous pass (growing m) left it set
    LK(PK_COMBINE, launch_lsqr_u(n, (const TV*)W + (size_t)mu * ld, ld, 1, ws.one, ws.u, 1, ws.part, ws.counter, ws.unorm2, ws.st, s));
    LK(PK_GEMVT, launch_gemv_t(n, (const TV*)W, ld, 0, mu, ws.u, ws.gpart, ntiles, ws.st, s));
    LK(PK_GEMVT, launch_reduce_cols(ws.gpart, ntiles, mu, ws.sigma, 0, nullptr, ws.lv_q, 0, nullptr, ws.st, s));
    LsqrVecs lv{ws.lv_v, ws.lv_w, ws.lv_x, ws.lv_z, ws.lv_coef, ws.lv_q};
    LK(PK_SMALL, launch_lsqr_start(ws.qr, p->s, mdev, ws.sigma, ws.unorm2, lv, p->lsqr_tol, ws.st, s, m));
    const int maxit = p->lsqr_maxit > 0 ? p->lsqr_maxit : 4 * mu;
    bool converged = false;
    for (int it = 0; it < maxit; ++it) {
      LK(PK_COMBINE, launch_lsqr_u(n, (const TV*)W, ld, mu, ws.lv_coef, ws.u, 0, ws.part, ws.counter, ws.unorm2, ws.st, s));
      LK(PK_GEMVT, launch_gemv_t(n, (const TV*)W, ld, 0, mu, ws.u, ws.gpart, ntiles, ws.st, s));
      LK(PK_GEMVT, launch_reduce_cols(ws.gpart, ntiles, mu, ws.sigma, 0, nullptr, ws.lv_q, 0, nullptr, ws.st, s));
      LK(PK_SMALL, launch_lsqr_step(ws.qr, p->s, mdev, ws.sigma, ws.unorm2, lv, ws.st, s, m));
      // iterations after convergence are no-ops on the device, so the host reads
      // the flag only every kLsqrPoll iterations
      if ((it + 1) % kLsqrPoll != 0 && it + 1 != maxit) continue;
      CK(cudaMemcpyAsync(&hs, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
      CK(wait_stream(s));
      if (hs.status != FAB_OK) return hs.status;
      if (hs.flag) {
        converged = true;
        break;
      }
    }
    lsqr_iters = hs.iters;
    if (!converged) return FAB_ENOTCONV;
    if (wh > 0) {
      yptr = ws.lv_x;
    } else {
      LK(PK_SMALL, launch_trsv(ws.qr, p->s, mdev, ws.lv_x, ws.y, 0, nullptr, s, m));
      yptr = ws.y;
    }
  }
  // f(H_m + h y e_m^T) e_1
  if (p->f == FAB_F_EXP) {
    LK(PK_SMALL, launch_build_hhat(ws.H, ldh, mdev, yptr, p->t, ws.mats[0], m, m, s));
    rc = expm_e1(ws, m, mdev, ws.cvec, &fh_iters, s);
  } else {
    LK(PK_SMALL, launch_build_hhat(ws.H, ldh, mdev, yptr, 1.0, ws.mats[0], m, m, s));
    rc = sqrtm_e1(ws, m, mdev, ws.cvec, p->f == FAB_F_SQRT, &fh_iters, s);
  }
  if (rc != FAB_OK) {  // no x; the diagnostics say how far the solve got
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->m_used = mu;
      stats->lsqr_iters = lsqr_iters;
      stats->fh_iters = fh_iters;
      stats->launches = g_launches;
      stats->beta = hs.beta;
      if (cudaMemcpyAsync(&hs, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
          wait_stream(s) == cudaSuccess)
        stats->kappa_est = hs.kappa;
      cudaGetLastError();
    }
    return rc;
  }
  if (!grow || mu < m) break;  // fixed m, or an invariant subspace: nothing to gain
  if (m_prev > 0) {  // sketched relative change of the solution since the previous m
    LK(PK_SMALL, launch_sketch_change(ws.SV, p->s, mdev, ws.cvec, m_prev, ws.cvec + (mcap + 1), ws.scal + 12, s));
    double* e2 = ws.hd + 2;
    CK(cudaMemcpyAsync(e2, ws.scal + 12, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(wait_stream(s));
    err_est = e2[1] > 0.0 ? e2[0] / e2[1] : 0.0;
    if (err_est <= p->target_rel_err) break;
  }
  if (m >= mcap) {  // the cap is reached before the target: best solution, flagged
    rc_final = FAB_ENOTCONV;
    break;
  }
  CK(cudaMemcpyAsync(ws.cvec + (mcap + 1), ws.cvec, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  m_prev = m;
  m = std::min(m + p->m_step, mcap);
  LK(PK_SMALL, launch_state_set_m(ws.st, m, s));
  }  // growing m
  CK(cudaEventRecord(ev[2], s));
  if (wh > 0) LK(PK_SMALL, launch_wh_coef(ws.wRi, ldr, wh, mdev, ws.cvec, s));  // to the stored columns
  // x = ||b|| V_m c  (gamma_b for Alg. 1 and a whitened basis)
  LK(PK_COMBINE, launch_prep_coef(ws.cvec, ws.sigma, mdev, ws.st, ws.coef, s));
  double* xdst = x;
  if (!bx_on_device) {
    if ((h->xbuf.bytes < (size_t)n * 8 && fault_hit()) || !ensure(h->xbuf, (size_t)n * 8)) return FAB_ENOMEM;
    xdst = ptr<double>(h->xbuf);
  }
  LK(PK_COMBINE, launch_combine(n, (const TV*)W, ld, mu, ws.coef, xdst, 0.0, s));
  CK(cudaEventRecord(ev[3], s));
  if (!bx_on_device) CK(cudaMemcpyAsync(x, xdst, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hs, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(wait_stream(s));
  if (g_prof.on) g_prof.end_solve();
  if (hs.status != FAB_OK) return hs.status;
  h->has_state = 1;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->err_est = err_est;
    stats->m_used = mu;
    stats->lsqr_iters = lsqr_iters;
    stats->fh_iters = fh_iters;
    stats->whiten_at = wh;
    stats->launches = g_launches;
    stats->beta = hs.beta;
    stats->kappa_est = hs.kappa;
    double hl = 0.0;
    if (mu == m) CK(cudaMemcpy(&hl, ws.H + m + (size_t)ldh * (m - 1), sizeof(double), cudaMemcpyDeviceToHost));
    stats->h_last = hl;
    float t01 = 0, t12 = 0, t23 = 0, t03 = 0;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    cudaEventElapsedTime(&t03, ev[0], ev[3]);
    stats->ms_basis = t01;
    stats->ms_small = t12;
    stats->ms_combine = t23;
    stats->ms_total = t03;
  }
  return rc_final;
}

namespace {
// A^2 of h's matrix on the host (row by row, a dense accumulator over the touched
// columns, columns sorted), as a handle of its own.
int build_square(fab_handle* h) {
  const int n = h->n, nnz = h->nnz;
  std::vector<int> ci(nnz);
  std::vector<double> va(nnz);
  if ((nnz > 0 && cudaMemcpy(ci.data(), h->d_colind, (size_t)nnz * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (nnz > 0 && cudaMemcpy(va.data(), h->d_vals, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  const int* rp = h->h_rowptr;
  std::vector<int64_t> rp2(n + 1, 0);
  std::vector<int32_t> ci2;
  std::vector<double> va2;
  std::vector<double> acc(n, 0.0);
  std::vector<char> seen(n, 0);
  std::vector<int> cols;
  for (int i = 0; i < n; ++i) {
    cols.clear();
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int k = ci[e];
      const double a = va[e];
      for (int f = rp[k]; f < rp[k + 1]; ++f) {
        const int j = ci[f];
        if (!seen[j]) {
          seen[j] = 1;
          cols.push_back(j);
        }
        acc[j] = fma(a, va[f], acc[j]);
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) {
      ci2.push_back(j);
      va2.push_back(acc[j]);
      acc[j] = 0.0;
      seen[j] = 0;
    }
    rp2[i + 1] = (int64_t)ci2.size();
  }
  if (ci2.size() >= ((size_t)1 << 31)) return FAB_EINVAL;
  fab_handle* sq = nullptr;
  const int rc = fab_create(&sq, n, (int64_t)ci2.size(), rp2.data(), ci2.data(), va2.data(), 0);
  if (rc != FAB_OK) return rc;
  h->sq = sq;
  return FAB_OK;
}
}  // namespace

extern "C" int fab_apply(fab_handle* h, const fab_params* p, const double* b, double* x, int bx_on_device,
                         fab_stats* stats) try {
  if (!h || !p || !b || !x) return FAB_EINVAL;
  // The inspectable state (fab_last_state / fab_last_basis) describes the last
  // successful solve only: any later call may regrow or overwrite its buffers.
  h->has_state = 0;
  int rc = validate(h, p);
  if (rc != FAB_OK) return rc;
  if (p->f == FAB_F_SIGN) {  // sign(A) b = (A^2)^{-1/2} (A b)
    if (!h->owns_matrix) return FAB_EINVAL;  // not on workspace clones (serving)
    if (!h->sq && (rc = build_square(h)) != FAB_OK) return rc;
    cudaStream_t s = (cudaStream_t)p->stream;
    const size_t n = (size_t)h->n;
    if (!ensure(h->sbuf, 2 * n * sizeof(double))) return FAB_ENOMEM;
    double* db = ptr<double>(h->sbuf);
    double* dab = db + n;
    if (cudaMemcpyAsync(db, b, n * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess ||
        launch_csr_spmv(h->n, h->d_rowptr, h->d_colind, h->d_vals, db, dab, s) != cudaSuccess) {
      cudaGetLastError();
      return FAB_ECUDA;
    }
    fab_params q = *p;
    q.f = FAB_F_INVSQRT;
    double* xd = bx_on_device ? x : db;  // b is no longer needed: its buffer takes x
    rc = fab_apply(h->sq, &q, dab, xd, 1, stats);
    h->has_state = 0;
    if ((rc == FAB_OK || rc == FAB_ENOTCONV) && !bx_on_device) {
      if (cudaMemcpyAsync(x, xd, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FAB_ECUDA;
      }
    }
    return rc;
  }
  Ws ws;
  rc = ensure_ws(h, p, ws);
  if (rc != FAB_OK) return rc;
  if (p->precision == FAB_MIXED) {
    rc = fab::ensure_vals32(h, (cudaStream_t)p->stream);
    if (rc != FAB_OK) return rc;
    return apply_impl<float>(h, p, b, x, bx_on_device, stats, ws, ws.W32, h->d_vals32);
  }
  return apply_impl<double>(h, p, b, x, bx_on_device, stats, ws, ws.W, h->d_vals);
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_last_state(fab_handle* h, double* H, double* SV, double* y, double* coeffs) try {
  if (!h || !h->has_state) return FAB_EINVAL;
  const int m = h->last_m;
  if (H && cudaMemcpy2D(H, (size_t)(m + 1) * 8, h->H.p, (size_t)h->last_ldh * 8, (size_t)(m + 1) * 8, m,
                        cudaMemcpyDeviceToHost) != cudaSuccess)
    return FAB_ECUDA;
  if (SV && h->last_sketched &&
      cudaMemcpy(SV, h->SV.p, (size_t)h->last_s * (m + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return FAB_ECUDA;
  if (y && cudaMemcpy(y, h->y.p, (size_t)m * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return FAB_ECUDA;
  if (coeffs && cudaMemcpy(coeffs, h->cvec.p, (size_t)m * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return FAB_ECUDA;
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_last_basis(fab_handle* h, double* V, int dst_on_device) try {
  if (!h || !h->has_state || !V) return FAB_EINVAL;
  const int m = h->last_m, n = h->n;
  double* dst = V;
  void* tmp = nullptr;
  if (!dst_on_device) {
    if (cudaMalloc(&tmp, (size_t)n * (m + 1) * 8) != cudaSuccess) {
      cudaGetLastError();
      return FAB_ENOMEM;
    }
    dst = (double*)tmp;
  }
  int rc = FAB_OK;
  const cudaError_t e = h->last_mixed
                            ? launch_scale_columns(n, (const float*)ptr<float>(h->W32), h->ld, m + 1,
                                                   ptr<double>(h->sigma), dst, n, 0)
                            : launch_scale_columns(n, (const double*)ptr<double>(h->W), h->ld, m + 1,
                                                   ptr<double>(h->sigma), dst, n, 0);
  if (e != cudaSuccess) rc = FAB_ECUDA;
  if (rc == FAB_OK && !dst_on_device &&
      cudaMemcpy(V, dst, (size_t)n * (m + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FAB_ECUDA;
  if (rc == FAB_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FAB_ECUDA;
  if (tmp) cudaFree(tmp);
  cudaGetLastError();
  return rc;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_sketch_apply(int sketch, int64_t n, int s, int zeta, uint64_t seed, const double* V_dev,
                                int64_t ldv, int ncols, double* out_dev, void* stream) try {
  if (n < 1 || n >= (int64_t)1 << 31 || s < 1 || s > kMaxS || ncols < 0 || ldv < n || !V_dev || !out_dev)
    return FAB_EINVAL;
  if (sketch == FAB_SK_SPARSE_SIGN) {
    if (zeta < 1 || zeta > kMaxZeta || zeta > s) return FAB_EINVAL;
  } else if (sketch == FAB_SK_SRHT) {
    if (s > next_pow2(n)) return FAB_EINVAL;
  } else if (sketch == FAB_SK_GAUSSIAN) {
    if (ncols > kGaussMaxCols) return FAB_EINVAL;
  } else {
    return FAB_EINVAL;
  }
  if (ncols == 0) return FAB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (sketch == FAB_SK_GAUSSIAN) {  // G and the BF16 columns in scratch, GEMM on the tensor cores
    __nv_bfloat16 *G = nullptr, *B = nullptr;
    double *part = nullptr, *ones = nullptr;
    DevState* ds = nullptr;
    int rc = FAB_OK;
    if (cudaMallocAsync((void**)&G, gauss_G_bytes(n, s), st) != cudaSuccess ||
        cudaMallocAsync((void**)&B, gauss_B_bytes(n, ncols), st) != cudaSuccess ||
        cudaMallocAsync((void**)&part, gauss_partial_bytes((int)n, s, ncols) + 16, st) != cudaSuccess ||
        cudaMallocAsync((void**)&ones, (size_t)ncols * 8, st) != cudaSuccess ||
        cudaMallocAsync((void**)&ds, sizeof(DevState), st) != cudaSuccess)
      rc = FAB_ENOMEM;
    std::vector<double> h1((size_t)ncols, 1.0);
    if (rc == FAB_OK && (cudaMemcpyAsync(ones, h1.data(), (size_t)ncols * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                         launch_state_reset(ds, 0, st) != cudaSuccess ||
                         launch_gauss_generate(s, (int)n, rng_state(seed, 5), G, st) != cudaSuccess ||
                         launch_to_bf16((int)n, ncols, V_dev, ldv, B, st) != cudaSuccess ||
                         launch_gauss_sketch(G, B, gauss_cpad(ncols), (int)n, s, ncols, ones, part, out_dev, ds, st) !=
                             cudaSuccess))
      rc = FAB_ECUDA;
    DevState hs;
    if (rc == FAB_OK && cudaMemcpyAsync(&hs, ds, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = FAB_ECUDA;
    for (void* q : {(void*)G, (void*)B, (void*)part, (void*)ones, (void*)ds})
      if (q) cudaFreeAsync(q, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = FAB_ECUDA;
    if (rc == FAB_OK && hs.status != FAB_OK) rc = hs.status;
    cudaGetLastError();
    return rc;
  }
  const int nchunks = (int)((n + kChunk - 1) / kChunk);
  double* part = nullptr;
  int* P = nullptr;
  DevState* ds = nullptr;
  if (cudaMallocAsync((void**)&part, (size_t)nchunks * s * 8, st) != cudaSuccess ||
      cudaMallocAsync((void**)&P, (size_t)s * 4, st) != cudaSuccess ||
      cudaMallocAsync((void**)&ds, sizeof(DevState), st) != cudaSuccess) {
    cudaGetLastError();
    if (part) cudaFreeAsync(part, st);
    if (P) cudaFreeAsync(P, st);
    cudaStreamSynchronize(st);
    return FAB_ENOMEM;
  }
  int rc = FAB_OK;
  SketchDev sk;
  memset(&sk, 0, sizeof(sk));
  sk.kind = sketch == FAB_SK_SRHT ? SK_SRHT : SK_SPARSE;
  sk.s = s;
  sk.zeta = zeta;
  sk.chunk_log2 = kChunkLog2;
  sk.nchunks = nchunks;
  sk.st_rows = rng_state(seed, 1);
  sk.st_signs = rng_state(seed, 2);
  sk.st_D = rng_state(seed, 3);
  sk.P = P;
  sk.part = part;
  const double scale = sk.kind == SK_SRHT ? 1.0 / sqrt((double)s) : 1.0 / sqrt((double)zeta);
  if (launch_state_reset(ds, 0, st) != cudaSuccess) rc = FAB_ECUDA;
  if (rc == FAB_OK && sk.kind == SK_SRHT && launch_srht_sample(next_pow2(n), s, rng_state(seed, 4), P, st) != cudaSuccess)
    rc = FAB_ECUDA;
  for (int j = 0; j < ncols && rc == FAB_OK; ++j) {
    if (launch_update((int)n, const_cast<double*>(V_dev), ldv, j, 0, 0, nullptr, nullptr, 1, ColScale{}, 0,
                      nullptr, nullptr, sk, ds, st) != cudaSuccess ||
        launch_sketch_reduce(sk, nullptr, 0, scale, out_dev + (size_t)j * s, ds, st) != cudaSuccess)
      rc = FAB_ECUDA;
  }
  cudaFreeAsync(part, st);
  cudaFreeAsync(P, st);
  cudaFreeAsync(ds, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = FAB_ECUDA;
  cudaGetLastError();
  return rc;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_profile_enable(int on) {
  g_prof.on = on != 0;
  for (int i = 0; i < PK_COUNT; ++i) {
    g_prof.total_ms[i] = 0.0;
    g_prof.launches[i] = 0;
  }
  g_prof.begin_solve();
  return FAB_OK;
}

extern "C" int fab_profile_only(const char* name) {
  if (!name || !*name) {
    g_prof.only = -1;
    return FAB_OK;
  }
  for (int i = 0; i < PK_COUNT; ++i) {
    if (strcmp(name, kProfNames[i]) == 0) {
      g_prof.only = i;
      return FAB_OK;
    }
  }
  return FAB_EINVAL;
}

extern "C" int fab_profile_query(const char* name, double* total_ms, int64_t* launches) {
  if (!name) return FAB_EINVAL;
  for (int i = 0; i < PK_COUNT; ++i) {
    if (strcmp(name, kProfNames[i]) == 0) {
      if (total_ms) *total_ms = g_prof.total_ms[i];
      if (launches) *launches = g_prof.launches[i];
      return FAB_OK;
    }
  }
  return FAB_EINVAL;
}

extern "C" int fab_fma_peak(int precision, double* gflops, double* ms, void* stream) try {
  if (!gflops || (precision != FAB_FP64 && precision != FAB_MIXED)) return FAB_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return FAB_ECUDA;
  }
  auto run = [&](int pattern, int iters, double* fmas, float* t) -> bool {
    if (cudaEventRecord(e0, s) != cudaSuccess) return false;
    const cudaError_t e = precision == FAB_FP64 ? launch_fma_peak<double>(pattern, 4, iters, s, fmas)
                                                : launch_fma_peak<float>(pattern, 4, iters, s, fmas);
    return e == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(t, e0, e1) == cudaSuccess;
  };
  // calibrate on a short launch, then time each operand pattern on launches of at least
  // 50 ms (after a warm-up of the same length) and keep the fastest
  double fmas = 0.0;
  float t = 0.f;
  int iters = 64;
  bool ok = true;
  for (int pattern = 0; pattern < 3 && ok; ++pattern) ok = run(pattern, iters, &fmas, &t);  // load the kernels
  if (ok) ok = run(0, iters, &fmas, &t);
  while (ok && t < 5.f && iters < (1 << 24)) {
    iters *= 4;
    ok = run(0, iters, &fmas, &t);
  }
  double best = 0.0;
  float best_t = 0.f;
  if (ok) {
    const double want = 50.0 / (t > 1e-3f ? t : 1e-3f);
    iters = (int)std::min<double>((double)(1 << 26), ceil(iters * want));
    for (int pattern = 0; pattern < 3 && ok; ++pattern) {
      ok = run(pattern, iters, &fmas, &t) && run(pattern, iters, &fmas, &t);
      if (ok && t > 0.f && 2.0 * fmas / ((double)t * 1e6) > best) {
        best = 2.0 * fmas / ((double)t * 1e6);
        best_t = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || !(best > 0.0)) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  *gflops = best;
  if (ms) *ms = best_t;
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_inject_wait_timeout(fab_handle* h, int pass, int polls) {
  if (!h || pass < 0 || (pass > 0 && polls < 1)) return FAB_EINVAL;
  h->stall_pass = pass;
  h->stall_polls = polls;
  return FAB_OK;
}

extern "C" int fab_set_fusion(fab_handle* h, int on) {
  if (!h) return FAB_EINVAL;
  h->fuse = on ? 1 : 0;
  return FAB_OK;
}

extern "C" int fab_set_tiling(fab_handle* h, int rows_max, int nnz_cap, int staged) try {
  if (!h || !h->owns_matrix) return FAB_EINVAL;
  return fab::build_tiles(h, rows_max, nnz_cap, staged);
} catch (...) {
  return fab::abi_error_code();
}

namespace {
// Device time (ms per launch) of the SpMV + window-dot kernel with h's current tiling.
template <typename TV>
int time_spmv(fab_handle* h, const void* vals, int k, unsigned char* scratch, cudaStream_t s, float* ms_out) {
  const int cols = k + 1;
  const size_t ld = (size_t)h->ld;
  Arena8 ar{scratch};
  TV* W = ar.take<TV>(ld * cols);
  ColScale cs{ar.take<double>(cols), ar.take<int>(cols), ar.take<double>(cols + 1)};
  double* H = ar.take<double>((size_t)cols * cols);
  double* coef = ar.take<double>(cols);
  double* part = ar.take<double>((size_t)sm_count() * kMaxPartBlocks * (kMaxWindow + 1));
  unsigned* counter = ar.take<unsigned>(16);
  DevState* st = ar.take<DevState>(1);
  Csr A{h->n, h->nnz, h->d_rowptr, h->d_colind, vals, h->d_tiles, h->ntiles, h->tile_staged};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaGetLastError();
    return FAB_ECUDA;
  }
  const int reps = 5;
  cudaError_t e = launch_spmv_dots<TV>(A, W, ld, k, 0, k, cs, H, cols, coef, part, counter, st, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int i = 0; i < reps && e == cudaSuccess; ++i)
    e = launch_spmv_dots<TV>(A, W, ld, k, 0, k, cs, H, cols, coef, part, counter, st, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  *ms_out = ms / reps;
  return FAB_OK;
}
}  // namespace

extern "C" int fab_tune(fab_handle* h, int precision, int k, int* choice, void* stream) try {
  if (!h || !h->owns_matrix || (precision != FAB_FP64 && precision != FAB_MIXED) || k < 1 || k > kMaxWindow)
    return FAB_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == FAB_MIXED) {
    const int rc = ensure_vals32(h, s);
    if (rc != FAB_OK) return rc;
  }
  const size_t esz = precision == FAB_MIXED ? 4 : 8;
  const int cols = k + 1;
  const size_t bytes = (size_t)h->ld * cols * esz + (size_t)sm_count() * kMaxPartBlocks * (kMaxWindow + 1) * 8 +
                       (size_t)cols * cols * 8 + 64 * 1024;
  unsigned char* scratch = nullptr;
  if (fault_hit() || cudaMalloc(&scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ENOMEM;
  }
  if (cudaMemsetAsync(scratch, 0, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(scratch);
    return FAB_ECUDA;
  }
  // candidates: rows per tile x nonzeros per tile x shared-memory staging
  const int rows_c[] = {256, 128, 64};
  const int nnz_c[] = {kSpmvCap, kSpmvCap / 2, kSpmvCap / 4};
  float best = 1e30f;
  int bi[3] = {256, kSpmvCap, 1};
  int rc = FAB_OK;
  for (int ri = 0; ri < 3 && rc == FAB_OK; ++ri)
    for (int ni = 0; ni < 3 && rc == FAB_OK; ++ni)
      for (int stg = 2; stg >= 0 && rc == FAB_OK; --stg) {
        rc = fab::build_tiles(h, rows_c[ri], nnz_c[ni], stg);
        if (rc != FAB_OK) break;
        float ms = 0.0f;
        rc = precision == FAB_MIXED ? time_spmv<float>(h, h->d_vals32, k, scratch, s, &ms)
                                    : time_spmv<double>(h, h->d_vals, k, scratch, s, &ms);
        if (rc == FAB_OK && ms < best) {
          best = ms;
          bi[0] = rows_c[ri];
          bi[1] = nnz_c[ni];
          bi[2] = stg;
        }
      }
  cudaFree(scratch);
  const int rc2 = fab::build_tiles(h, bi[0], bi[1], bi[2]);
  if (rc == FAB_OK) rc = rc2;
  if (choice) {
    choice[0] = bi[0];
    choice[1] = bi[1];
    choice[2] = bi[2];
  }
  return rc;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" const char* fab_last_error(void) { return g_errmsg; }

namespace fab {
void set_last_error(const char* msg) { snprintf(g_errmsg, sizeof(g_errmsg), "%s", msg ? msg : ""); }
void use_blocking_waits(bool on) {
  if (on && !g_wait_event) {
    if (cudaEventCreateWithFlags(&g_wait_event, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      g_wait_event = nullptr;
    }
  } else if (!on && g_wait_event) {
    cudaEventDestroy(g_wait_event);
    g_wait_event = nullptr;
  }
}
int validate_params(const fab_handle* h, const fab_params* p) { return validate(h, p); }
const double* pade13_b() {
  static const Pade13 pd;
  return pd.b;
}
double pade13_theta() { return kTheta13; }
bool alloc_fault() { return fault_hit(); }
}  // namespace fab

namespace fab {
// FP32 copy of A's values (mixed precision), made once per matrix.
int ensure_vals32(fab_handle* h, cudaStream_t s) {
  if (h->d_vals32) return FAB_OK;
  if (fault_hit() || cudaMalloc(&h->d_vals32, (size_t)(h->nnz + kCsrPad) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    h->d_vals32 = nullptr;
    return FAB_ENOMEM;
  }
  if (launch_to_f32(h->nnz + (int)kCsrPad, h->d_vals, h->d_vals32, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  // the ELL form the one-pass steps read (rows of at most 8 nonzeros); without it the
  // two-pass loop runs
  if (h->d_ftasks && h->max_row_nnz >= 1 && h->max_row_nnz <= 8 && !h->d_ell_col) {
    const size_t cnt = (size_t)h->max_row_nnz * (size_t)h->ld;
    if (cudaMalloc(&h->d_ell_col, cnt * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->d_ell_val, cnt * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(h->d_ell_col);
      cudaFree(h->d_ell_val);
      h->d_ell_col = nullptr;
      h->d_ell_val = nullptr;
      return FAB_OK;
    }
    if (launch_build_ell(h->n, h->d_rowptr, h->d_colind, h->d_vals32, h->max_row_nnz, h->ld, h->d_ell_col,
                         h->d_ell_val, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return FAB_ECUDA;
    }
  }
  return FAB_OK;
}

size_t estimate_ws_bytes(const fab_handle* h, const fab_params* p) {
  Need need[64];
  const int cnt = ws_needs(const_cast<fab_handle*>(h), p, need);
  size_t t = 0;
  for (int i = 0; i < cnt; ++i) t += need[i].bytes;
  if (p->precision == FAB_MIXED) t += (size_t)(h->nnz + kCsrPad) * sizeof(float);
  return t;
}

size_t handle_ws_bytes(const fab_handle* h) {
  const Buf* bufs[] = {&h->spat, &h->W32, &h->Wbf, &h->G,    &h->shf,  &h->scl,  &h->W,   &h->H,     &h->sigma,
                       &h->coef, &h->part, &h->counter, &h->gpart, &h->skpart, &h->SV, &h->P,
                       &h->qr,  &h->tau, &h->y,    &h->cvec, &h->dense, &h->piv, &h->scal, &h->lsq,
                       &h->u,   &h->xbuf, &h->state, &h->whm};
  size_t t = 0;
  for (const Buf* b : bufs) t += b->bytes;
  if (h->d_vals32) t += (size_t)(h->nnz + kCsrPad) * sizeof(float);
  if (h->d_ell_col) t += (size_t)h->max_row_nnz * (size_t)h->ld * 8;
  return t;
}

fab_handle* clone_for_workspace(const fab_handle* h) {
  fab_handle* c = new fab_handle();
  c->owns_matrix = false;
  point_to_matrix(c, h);
  return c;
}

int build_tiles(fab_handle* h, int rows_max, int nnz_cap, int staged) {
  if (!h || !h->h_rowptr || rows_max < 1 || rows_max > kThreads || nnz_cap < 1 || staged < 0 || staged > 2)
    return FAB_EINVAL;
  const int* rp = h->h_rowptr;
  std::vector<int> t;
  t.reserve(h->n / 16 + 2);
  t.push_back(0);
  int r0 = 0;
  while (r0 < h->n) {
    int r1 = r0 + 1;
    // grow while the tile stays within rows_max rows and its 16-byte aligned
    // nonzero range within nnz_cap entries
    while (r1 < h->n && r1 - r0 < rows_max && ((rp[r1 + 1] + 3) & ~3) - (rp[r0] & ~3) <= nnz_cap) ++r1;
    // a tile cut by the nonzero cap keeps a power-of-two row count, so that
    // 256 / rows lanes per row use every thread of the block (not needed when
    // the tile is processed by nonzeros)
    if (staged != 2 && r1 < h->n && r1 - r0 < rows_max) {
      int R = 1;
      while (2 * R <= r1 - r0) R *= 2;
      r1 = r0 + R;
    }
    t.push_back(r1);
    r0 = r1;
  }
  int* d = nullptr;
  if (alloc_fault() || cudaMalloc(&d, t.size() * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ENOMEM;
  }
  if (cudaMemcpy(d, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d);
    return FAB_ECUDA;
  }
  cudaFree(h->d_tiles);
  h->d_tiles = d;
  h->ntiles = (int)t.size() - 1;
  h->tile_rows = rows_max;
  h->tile_nnz = nnz_cap;
  h->tile_staged = staged;
  return FAB_OK;
}

void point_to_matrix(fab_handle* c, const fab_handle* h) {
  c->d_tiles = h->d_tiles;
  c->ntiles = h->ntiles;
  c->tile_rows = h->tile_rows;
  c->tile_nnz = h->tile_nnz;
  c->tile_staged = h->tile_staged;
  c->max_row_nnz = h->max_row_nnz;
  c->fuse = h->fuse;
  c->d_ftasks = h->d_ftasks;
  c->d_fcrange = h->d_fcrange;
  c->d_ell_col = h->d_ell_col;
  c->d_ell_val = h->d_ell_val;
  c->h_rowptr = h->h_rowptr;
  c->n = h->n;
  c->nnz = h->nnz;
  c->d_rowptr = h->d_rowptr;
  c->d_colind = h->d_colind;
  c->d_vals = h->d_vals;
  c->d_vals32 = h->d_vals32;
  c->ld = h->ld;
  c->has_state = 0;
}
}  // namespace fab
