// One-pass basis step of Alg. 2 for the FP32 basis (mixed precision): the window
// update, norm and fused sketch of column c-1 and the SpMV + window dot products of
// step c run in one launch, so every basis step reads A, the window and the previous
// SpMV output from HBM once and writes two vectors.
//
// Pass c is a list of tasks over the 4096-row chunks (the sketch's transform block):
//   U_i  the update of chunk i of column c-1: u = w_{c-1} - sum_q coef_q W_{j0u+q}
//        (coefficients from pass c-1's reduction), stored as column c-1; its
//        ||u||^2 and int64 sketch go into the block's partials; then flag[i] = c
//        (release);
//   S_j  the SpMV of chunk j: waits (acquire, bounded) until flag[i] = c for every
//        chunk i that the rows of chunk j reference, then w_c[r] = 2^e sum_e a_re
//        u[col_e] (u of the chunk itself from shared memory, of other chunks from
//        L2), the window dots <W_j, w_c> and ||w_c||^2 into the partials, w_c to a
//        scratch vector (double buffered: pass c+1 reads w_c while it writes w_{c+1};
//        the last step writes column m itself).
// Blocks claim tasks from a counter in a fixed order, U_i at position key 2i and S_j at
// key 2(j+H+L)+1, H the farthest chunk any chunk's rows reach ahead and L a lead of about
// half the resident blocks (so that an S task seldom waits). An S task waits only
// for U tasks with smaller keys, which were claimed before it by running blocks, and a
// U task waits for nothing: every claimed task finishes whatever number of blocks is
// resident. The order is a wavefront: chunk i's window columns and u are still in L2
// when S_i and its neighbours read them, so HBM sees each vector once.
// The last block to finish reduces the partials: h_{c-1,c-2}, the breakdown test and
// sigma_{c-1} first, then h_{j,c-1} = sigma_j tau_c d_j and the next coefficients,
// with tau_c = sigma_{c-1} 2^-e. The exact shift e of pass c comes from ||w_{c-1}||
// (pass c-1) instead of ||u_{c-1}|| (not known until pass c ends); a power of two
// changes no rounding, and ||u|| <= ||w|| keeps the new column in range.
//
// Rows with at most 8 nonzeros (stencil matrices): the S tasks read A in ELL form (slot u
// of every row contiguous, so that a warp's loads of a slot are one coalesced stream),
// kFuseRows rows per thread with all their loads in flight; no shared-memory staging.
#include <float.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "chunk.cuh"
#include "fab_internal.cuh"
#include "handle.cuh"

namespace fab {

namespace {

constexpr int kFuseRows = 2;  // rows per thread whose loads are in flight together in an S task
constexpr int kFlagLimit = 1 << 21;  // polls of a chunk flag before FAB_ETIMEOUT

// Shared-memory layout: u of the S task's chunk, the sketch's per-chunk scratch of the
// U tasks (the SRHT transform buffer, or the sparse-sign accumulators and chunk values),
// then the block's sketch accumulators and the SRHT sample, which persist across tasks.
struct FuseSmem {
  size_t su, scratch, acc, P, total;
};
__host__ __device__ inline FuseSmem fuse_layout(int kind, int s) {
  FuseSmem L;
  L.su = 0;
  L.scratch = L.su + (size_t)kChunk * 4;
  size_t scr = 0;
  if (kind == SK_SRHT) scr = (size_t)(kChunk + kChunk / 16) * 8;
  if (kind == SK_SPARSE_TAB) scr = ((size_t)s * 8 + 15) / 16 * 16 + (size_t)kChunk * 8;
  L.acc = (L.scratch + scr + 15) / 16 * 16;
  const bool sk = kind == SK_SRHT || kind == SK_SPARSE_TAB;
  L.P = L.acc + (sk ? ((size_t)s * 8 + 15) / 16 * 16 : 0);
  L.total = (L.P + (kind == SK_SRHT ? (size_t)s * 4 : 0) + 15) / 16 * 16;
  return L;
}

struct FuseArgs {
  Csr A;               // FP32 values; 256-row tiles implied (A.tiles unused)
  float* W;            // raw basis columns (ld)
  int64_t ld;
  int c;               // this pass: update of column c-1 (when upd) and SpMV of step c
  int upd;             // 1: column c-1 is still w_{c-1} (in wprev) and gets its update here
  int j0u, kwu;        // the update's window: columns j0u .. j0u+kwu-1
  int j0, kw;          // step c's window for the dots: columns j0 .. c-1
  const float* wprev;  // w_{c-1} (upd) or column c-1 itself
  float* wnext;        // destination of w_c
  ColScale cs;
  double* H;
  int ldh;
  double* coef;        // in: the update's coefficients; out (last block): step c's
  double* part;
  unsigned* counter;   // [0] last-block counter, [1] task counter
  DevState* st;
  SketchDev sk;        // sketch of column c-1 (kind SK_NONE: none)
  int* flags;          // per chunk: the last pass whose update of that chunk is stored
  const int* tasks;    // 2 nchunks task codes in claim order: 2i = U_i, 2j+1 = S_j
  const int2* crange;  // per chunk: first and last chunk its rows reference (and itself)
  const int* ell_col;  // the matrix in ELL form: slot u of row r at u ell_ld + r (ell_k <= 8 slots)
  const float* ell_val;
  int64_t ell_ld;
  int ell_k;
  int flag_extra;      // an S task waits for flag >= c + flag_extra (1: a value no task sets)
  int flag_limit;      // polls of a flag before FAB_ETIMEOUT
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int SK, int KU>
__global__ __launch_bounds__(kThreads, 3) void k_fused_step(FuseArgs a) {
  extern __shared__ __align__(16) unsigned char smem_f[];
  constexpr int NV = KU + 3;  // dots (kw <= KU + 1), ||u_{c-1}||^2, ||w_c||^2
  __shared__ volatile int s_fail;
  __shared__ int s_task;
  __shared__ double sh[32 * NV];
  __shared__ double tot[NV];
  __shared__ int s_int[32];
  DevState* st = a.st;
  if (st->stop) return;
  const FuseSmem L = fuse_layout(SK, a.sk.s);
  float* su = reinterpret_cast<float*>(smem_f + L.su);
  long long* buf = reinterpret_cast<long long*>(smem_f + L.scratch);
  unsigned long long* sacc = reinterpret_cast<unsigned long long*>(smem_f + L.scratch);
  double* s_acc = reinterpret_cast<double*>(smem_f + L.acc);
  int* s_P = reinterpret_cast<int*>(smem_f + L.P);
  const SketchDev& sk = a.sk;
  const Csr& A = a.A;
  const int n = A.n, tid = threadIdx.x, lane = tid & 31;
  const int nchunks = (n + kChunk - 1) / kChunk;
  const int ntasks = 2 * nchunks;
  const int c = a.c;
  const bool upd = a.upd != 0;
  const int kwu = upd ? KU : 0;
  const size_t ld = (size_t)a.ld;
  // the update's coefficients (FP32, as the two-pass update uses them)
  float cf[KU > 0 ? KU : 1];
#pragma unroll
  for (int q = 0; q < KU; ++q) cf[q] = upd ? (float)a.coef[q] : 0.f;
  const float* Wu0 = a.W + (size_t)a.j0u * ld;  // the update's window column q at Wu0 + q ld
  const float* Wd0 = a.W + (size_t)a.j0 * ld;   // step c's window column q at Wd0 + q ld
  float* ucol = a.W + (size_t)(c - 1) * ld;
  const int kw = a.kw;       // KU or KU + 1
  const int jlast = kw - 1;  // the dot with W_{c-1} = u (read from shared memory)
  const int ksh = a.cs.shf[c - 1];
  double p2k_lo;
  const double p2k_hi = pow2_split(ksh, &p2k_lo);
  const float p2k = (float)(p2k_hi * p2k_lo);
  if (SK == SK_SRHT || SK == SK_SPARSE_TAB)
    for (int q = tid; q < sk.s; q += kThreads) s_acc[q] = 0.0;
  if (SK == SK_SRHT)
    for (int q = tid; q < sk.s; q += kThreads) s_P[q] = sk.P[q];
  if (tid == 0) s_fail = 0;
  __syncthreads();

  double nrm_u = 0.0, nrm_w = 0.0;
  double accd[KU + 1];
#pragma unroll
  for (int q = 0; q <= KU; ++q) accd[q] = 0.0;
  // Thread 0 claims the next task when the current one starts, so the claim's latency
  // overlaps the work. A pre-claimed task only waits on tasks with smaller keys (claimed
  // earlier still), so claiming ahead adds no cycle.
  int next = 0;
  if (tid == 0) next = (int)atomicAdd(a.counter + 1, 1u);
  for (;;) {
    if (tid == 0) s_task = next;
    __syncthreads();
    const int tk = s_task;
    __syncthreads();  // every thread has the task before thread 0 overwrites s_task
    if (tk >= ntasks || s_fail) break;
    if (tid == 0) next = (int)atomicAdd(a.counter + 1, 1u);
    const int code = a.tasks[tk];
    const int ch = code >> 1;
    const int base = ch * kChunk;
    if ((code & 1) == 0) {
      // ---------------- U_ch: u = w_{c-1} - sum_q coef_q W_{j0u+q} on the chunk's rows
      if (!upd) continue;  // column c-1 is final: nothing to update, nothing to wait for
      float v[kRowsPerThread];
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) v[i] = __ldg(a.wprev + min(base + i * kThreads + tid, n - 1));
#pragma unroll
      for (int q = 0; q < KU; ++q) {
        float w[kRowsPerThread];
#pragma unroll
        for (int i = 0; i < kRowsPerThread; ++i) w[i] = __ldg(Wu0 + q * ld + min(base + i * kThreads + tid, n - 1));
#pragma unroll
        for (int i = 0; i < kRowsPerThread; ++i) v[i] = fma(-cf[q], w[i], v[i]);
      }
      float nrm_c = 0.f;
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        const int r = base + i * kThreads + tid;
        if (r >= n) v[i] = 0.f;
        if (r < n) ucol[r] = v[i];
        nrm_c = fma(v[i], v[i], nrm_c);
      }
      nrm_u += (double)nrm_c;
      if (SK == SK_SPARSE_TAB) {  // its accumulators share the region the tile ring used
        for (int q = tid; q < sk.s; q += kThreads) sacc[q] = 0ull;
        __syncthreads();
      }
      if (SK == SK_SRHT) sketch_chunk_srht(v, ch, sk, buf, s_P, s_acc, s_int);
      if (SK == SK_SPARSE_TAB) sketch_chunk_sparse<float, true>(v, ch, n, sk, sacc, s_acc, s_int);
      __syncthreads();  // every row of the chunk is stored
      if (tid == 0) {
        __threadfence();
        st_release(a.flags + ch, c);
      }
      continue;
    }
    // ---------------- S_ch: wait for the chunks it references, then the chunk's rows
    if (upd) {
      const int2 rg = a.crange[ch];
      for (int i = rg.x + tid; i <= rg.y; i += kThreads) {
        int it = 0;
        while (ld_acquire(a.flags + i) < c + a.flag_extra && ++it < a.flag_limit) __nanosleep(64);
        if (it >= a.flag_limit) s_fail = 1;
      }
      __syncthreads();
      if (s_fail) continue;  // uniform: the loop ends at the next claim
    }
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) {  // u of the chunk (stored by another block: from L2)
      const int r = base + i * kThreads + tid;
      su[i * kThreads + tid] = r < n ? __ldcg(ucol + r) : 0.f;
    }
    __syncthreads();
    float accf[KU + 1];
#pragma unroll
    for (int q = 0; q <= KU; ++q) accf[q] = 0.f;
    float nrm_wc = 0.f;
    // kFuseRows rows per thread at a time, every slot's loads in flight together; the ELL
    // slots of a row hold its nonzeros in CSR order, then zeros on the row's own column
    for (int i0 = 0; i0 < kRowsPerThread; i0 += kFuseRows) {
      int col[kFuseRows][8];
      float am[kFuseRows][8], g[kFuseRows][8], wv[kFuseRows][KU + 1];
#pragma unroll
      for (int j = 0; j < kFuseRows; ++j) {
        const int r = min(base + (i0 + j) * kThreads + tid, n - 1);  // clamped: loads stay in the matrix
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          col[j][u] = u < a.ell_k ? __ldg(a.ell_col + (size_t)u * a.ell_ld + r) : r;
          am[j][u] = u < a.ell_k ? __ldg(a.ell_val + (size_t)u * a.ell_ld + r) : 0.f;
        }
#pragma unroll
        for (int q = 0; q <= KU; ++q) wv[j][q] = q < jlast ? __ldg(Wd0 + q * ld + r) : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kFuseRows; ++j) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {  // u[col]: shared memory inside the chunk, L2 outside it
          const bool outside = (unsigned)(col[j][u] - base) >= (unsigned)kChunk;
          g[j][u] = u >= a.ell_k ? 0.f : (outside ? __ldcg(ucol + col[j][u]) : su[col[j][u] - base]);
        }
      }
#pragma unroll
      for (int j = 0; j < kFuseRows; ++j) {
        const int r = base + (i0 + j) * kThreads + tid;
        float y = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < a.ell_k) y = fma(am[j][u], g[j][u], y);
        if (r < n) {
          y = scale_pow2(y, ksh, p2k);
          a.wnext[r] = y;
          const float ur = su[(i0 + j) * kThreads + tid];  // u[r]
#pragma unroll
          for (int q = 0; q <= KU; ++q)
            if (q < kw) accf[q] = fma(q == jlast ? ur : wv[j][q], y, accf[q]);
          nrm_wc = fma(y, y, nrm_wc);
        }
      }
    }
#pragma unroll
    for (int q = 0; q <= KU; ++q) accd[q] += (double)accf[q];
    nrm_w += (double)nrm_wc;
    __syncthreads();  // su and the sketch scratch are reused by the next task
  }
  (void)kwu;
  (void)lane;
  if (s_fail) {
    // a chunk flag was never set (its update did not finish in time): record it
    if (tid == 0) {
      st->status = FAB_ETIMEOUT;
      st->stop = 1;
    }
    return;
  }
  if ((SK == SK_SRHT || SK == SK_SPARSE_TAB) && upd) {  // this block's share of the sketch of column c-1
    double* out = sk.part + (size_t)blockIdx.x * sk.s;
    for (int q = tid; q < sk.s; q += kThreads) out[q] = s_acc[q];
  }
  // ---- block partials: dots, ||u_{c-1}||^2, ||w_c||^2
  double vals[NV];
#pragma unroll
  for (int q = 0; q <= KU; ++q) vals[q] = accd[q];
  vals[KU + 1] = nrm_u;
  vals[KU + 2] = nrm_w;
  block_sum_multi<NV>(vals, sh, tot);
  if (tid < NV) a.part[(size_t)blockIdx.x * NV + tid] = tot[tid];
  if (!last_block(a.counter, gridDim.x)) return;
  sum_partials_multi<NV>(a.part, gridDim.x, tot, sh);
  if (tid == 0) {
    const ColScale& cs = a.cs;
    bool stop = false;
    if (upd) {  // column c-1: h_{c-1,c-2}, breakdown test, sigma_{c-1} (as column_norm_tail)
      const int cu = c - 1;
      const double h = sqrt(tot[KU + 1]);
      const double hc = cs.scl[cu] * h;
      a.H[cu + (size_t)a.ldh * (cu - 1)] = hc;
      double av2 = hc * hc;
      for (int j = a.j0u; j < cu; ++j) {
        const double hj = a.H[j + (size_t)a.ldh * (cu - 1)];
        av2 = fma(hj, hj, av2);
      }
      if (!isfinite(hc)) {
        st->status = FAB_ENUMERIC;
        st->stop = 1;
        stop = true;
      } else if (!(hc > 64.0 * DBL_EPSILON * sqrt(av2))) {
        st->m_used = cu;  // the basis spans an invariant subspace
        st->stop = 1;
        cs.sigma[cu] = 0.0;
        stop = true;
      } else {
        cs.sigma[cu] = 1.0 / h;
      }
    }
    if (!stop) {  // step c: h_{j,c-1} = sigma_j tau d_j, the next update's coefficients, the next shift
      const double tau = column_tau(cs.sigma[c - 1], ksh);
      for (int q = 0; q < kw; ++q) {
        const int j = a.j0 + q;
        const double d = tot[q];
        a.H[j + (size_t)a.ldh * (c - 1)] = cs.sigma[j] * tau * d;
        a.coef[q] = cs.sigma[j] * cs.sigma[j] * d;
      }
      cs.scl[c] = tau;
      const double wn = sqrt(tot[KU + 2]);
      if (!isfinite(wn)) {
        st->status = FAB_ENUMERIC;
        st->stop = 1;
      }
      cs.shf[c] = (wn > 0.0 && isfinite(wn)) ? exponent_of(1.0 / wn) : 0;
    }
    a.counter[1] = 0;  // every block has stopped claiming tasks
    *a.counter = 0;
  }
}

template <int SK>
const void* fused_fn(int ku) {
  static const void* fns[kMaxWindow + 1] = {
      (const void*)k_fused_step<SK, 0>, (const void*)k_fused_step<SK, 1>, (const void*)k_fused_step<SK, 2>,
      (const void*)k_fused_step<SK, 3>, (const void*)k_fused_step<SK, 4>, (const void*)k_fused_step<SK, 5>,
      (const void*)k_fused_step<SK, 6>, (const void*)k_fused_step<SK, 7>, (const void*)k_fused_step<SK, 8>};
  return fns[ku];
}

const void* fused_kernel(int kind, int ku) {
  switch (kind) {
    case SK_SRHT: return fused_fn<SK_SRHT>(ku);
    case SK_SPARSE_TAB: return fused_fn<SK_SPARSE_TAB>(ku);
    default: return fused_fn<SK_NONE>(ku);
  }
}

// ELL copy of the FP32 CSR matrix: slot u of row r holds the row's u-th nonzero (CSR
// order) or, past the row's end, a zero on the row's own column.
__global__ void k_build_ell(int n, const int* __restrict__ rowptr, const int* __restrict__ colind,
                            const float* __restrict__ vals, int k, int64_t ld, int* __restrict__ ecol,
                            float* __restrict__ eval) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int e0 = rowptr[r], e1 = rowptr[r + 1];
    for (int u = 0; u < k; ++u) {
      const int e = e0 + u;
      ecol[(size_t)u * ld + r] = e < e1 ? colind[e] : r;
      eval[(size_t)u * ld + r] = e < e1 ? vals[e] : 0.f;
    }
  }
}

}  // namespace

cudaError_t launch_build_ell(int n, const int* rowptr, const int* colind, const float* vals, int k, int64_t ld,
                             int* ecol, float* eval, cudaStream_t s) {
  const int grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_build_ell<<<grid < 1 ? 1 : grid, 256, 0, s>>>(n, rowptr, colind, vals, k, ld, ecol, eval);
  return cudaGetLastError();
}

int fused_grid(int kind, int n, int s, size_t* smem_out) {
  const FuseSmem L = fuse_layout(kind, s);
  if (smem_out) *smem_out = L.total;
  // blocks per SM, the same for every window width (one partial layout per solve),
  // found once per (sketch kind, shared-memory size)
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  int occ_min;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({kind, L.total});
    if (it != cache.end()) {
      occ_min = it->second;
    } else {
      occ_min = 1 << 30;
      for (int ku = 0; ku <= kMaxWindow; ++ku) {
        const void* fn = fused_kernel(kind, ku);
        if (ensure_smem_limit(fn, L.total) != cudaSuccess) return -1;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, L.total);
        occ_min = occ < occ_min ? occ : occ_min;
      }
      if (occ_min < 1) occ_min = 1;
      cache[{kind, L.total}] = occ_min;
    }
  }
  const int nchunks = (n + kChunk - 1) / kChunk;
  const int grid = sm_count() * occ_min;
  return nchunks < grid ? (nchunks < 1 ? 1 : nchunks) : grid;
}

void fused_plan(int n, const int* rowptr, const int* colind, int lead, std::vector<int>& tasks,
                std::vector<int2>& crange) {
  const int nch = (n + kChunk - 1) / kChunk;
  crange.assign(nch, int2{0, 0});
  int H = 0;
  for (int ch = 0; ch < nch; ++ch) {
    int lo = ch, hi = ch;  // the chunk's own u is read too
    const int r0 = ch * kChunk, r1 = std::min(n, r0 + kChunk);
    for (int e = rowptr[r0]; e < rowptr[r1]; ++e) {
      const int cc = colind[e] / kChunk;
      lo = cc < lo ? cc : lo;
      hi = cc > hi ? cc : hi;
    }
    crange[ch] = int2{lo, hi};
    H = std::max(H, hi - ch);
  }
  // claim order: U_i at key 2i, S_j at key 2 (j + H + lead) + 1: the updates run H + lead
  // chunks ahead, so that S_j is claimed about lead chunks after the last update it needs
  // (that update has finished by then, and the chunk's vectors are still in L2)
  H += lead > 0 ? lead : 0;
  tasks.clear();
  tasks.reserve(2 * (size_t)nch);
  int u = 0, sj = 0;
  while (u < nch || sj < nch) {
    if (u < nch && (sj >= nch || 2 * (long long)u < 2 * ((long long)sj + H) + 1))
      tasks.push_back(2 * u++);
    else
      tasks.push_back(2 * sj++ + 1);
  }
}

cudaError_t launch_fused_step(const Csr& A, float* W, int64_t ld, int c, int upd, int j0u, int kwu, int j0, int kw,
                              const float* wprev, float* wnext, ColScale cs, double* H, int ldh, double* coef,
                              double* part, unsigned* counter, SketchDev& sk, DevState* st, const FusePlan& plan,
                              cudaStream_t s) {
  if (kwu < 0 || kwu > kMaxWindow || kw < 1 || kw > kMaxWindow || (upd && kw != kwu && kw != kwu + 1) ||
      (!upd && kwu != 0) || !plan.flags || !plan.tasks || !plan.crange || !plan.ell_col || !plan.ell_val ||
      plan.ell_k < 1 || plan.ell_k > 8)
    return cudaErrorInvalidValue;
  const int kind = (sk.kind == SK_SPARSE && sk.pat) ? SK_SPARSE_TAB : sk.kind;
  if (kind != SK_SRHT && kind != SK_SPARSE_TAB && kind != SK_NONE) return cudaErrorInvalidValue;
  // the kernel's window array holds KU + 1 dots: KU = the update window, or kw - 1 without an update
  const int ku = upd ? kwu : kw - 1;
  size_t smem = 0;
  const int grid = fused_grid(kind, A.n, sk.s, &smem);
  if (grid < 1) return cudaErrorInvalidValue;
  sk.nparts = grid;
  FuseArgs a;
  a.A = A;
  a.W = W;
  a.ld = ld;
  a.c = c;
  a.upd = upd;
  a.j0u = j0u;
  a.kwu = kwu;
  a.j0 = j0;
  a.kw = kw;
  a.wprev = wprev;
  a.wnext = wnext;
  a.cs = cs;
  a.H = H;
  a.ldh = ldh;
  a.coef = coef;
  a.part = part;
  a.counter = counter;
  a.st = st;
  a.sk = sk;
  a.flags = plan.flags;
  a.tasks = plan.tasks;
  a.crange = reinterpret_cast<const int2*>(plan.crange);
  a.ell_col = plan.ell_col;
  a.ell_val = plan.ell_val;
  a.ell_ld = plan.ell_ld;
  a.ell_k = plan.ell_k;
  const bool stall = plan.stall_pass > 0 && c == plan.stall_pass;  // the failure-detection hook
  a.flag_extra = stall ? 1 : 0;
  a.flag_limit = stall ? plan.stall_polls : kFlagLimit;
  void* args[] = {&a};
  return cudaLaunchKernel(fused_kernel(kind, ku), dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace fab
