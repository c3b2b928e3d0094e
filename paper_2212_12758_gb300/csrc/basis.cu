// Basis-loop kernels of libfab: CSR SpMV fused with the window dot products of
// Alg. 2 (truncated orthogonalization, paper §2.1.2), the window update fused
// with the norm and the sketch of the new vector (paper §2.1.1, §3.3), the
// cross-chunk sketch reduction, the SRHT row sampling, and the classical
// Gram-Schmidt passes of the Arnoldi baseline (eq. arnoldi).
//
// Storage: the basis is kept as raw columns W_j (column-major, leading
// dimension ld) with separate scales sigma_j = 1/||W_j||, so v_j = sigma_j W_j.
// Every consumer folds sigma_j into its coefficients, which saves the pass
// that would otherwise normalize each new vector.
#include <float.h>
#include <limits.h>

#include <cuda_bf16.h>

#include <map>
#include <mutex>

#include "chunk.cuh"
#include "fab_internal.cuh"
#include "gauss.cuh"

namespace fab {

int sm_count();

// ------------------------------------------------------------------- state
__global__ void k_state_reset(DevState* st, int m) {
  st->m_used = m;
  st->stop = 0;
  st->status = FAB_OK;
  st->flag = 0;
  st->iters = 0;
  st->wh = 0;
  st->beta = 0.0;
  for (int i = 0; i < 16; ++i) st->scal[i] = 0.0;
  st->kappa = 0.0;
}

cudaError_t launch_state_reset(DevState* st, int m, cudaStream_t s) {
  k_state_reset<<<1, 1, 0, s>>>(st, m);
  return cudaGetLastError();
}

__global__ void k_state_set_m(DevState* st, int m) { st->m_used = m; }

__global__ void k_state_clear_flag(DevState* st) { st->flag = 0; }

cudaError_t launch_state_clear_flag(DevState* st, cudaStream_t s) {
  k_state_clear_flag<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_state_set_m(DevState* st, int m, cudaStream_t s) {
  k_state_set_m<<<1, 1, 0, s>>>(st, m);
  return cudaGetLastError();
}

// --------------------------------------------- SpMV + window dot products
// W_c = 2^shf[c-1] A W_{c-1} is written to column c (an exact power-of-two rescale
// done on the exponent bits keeps the raw columns near unit norm without FP64
// work); for the window j0..j0+kw-1 the dots d_j = <W_j, W_c> are reduced over the
// grid (recursive halving within a warp: a few additions for all kw dots, not kw
// full warp reductions). With v_j = sigma_j W_j and tau = sigma_{c-1} 2^-shf[c-1]
// (so that A v_{c-1} = tau W_c) the last block writes
//   h_{j,c-1} = sigma_j tau d_j     (into H),
//   coef_q    = sigma_j^2 d_j       (update coefficient of the raw column),
//   scl[c]    = tau
// (no window: block 0 writes scl[c] alone). ||A v_{c-1}|| for the breakdown test
// is formed by the update from h_{j,c-1} and h_{c,c-1} (column_norm_tail).
// The rows are cut into tiles of at most 256 rows and (unless a single row has
// more) at most kSpmvCap nonzeros, so every block iteration has about the same
// work whatever the row lengths. A tile's nonzeros are staged in shared memory
// by bulk copies (double buffered, one tile ahead) when they fit the stage; a
// longer single-row tile is read from global memory with the same order of
// operations.

// With A.staged == 2, staged tiles of at least kSegRows rows are processed by
// nonzeros instead of by rows (the short, uneven rows of a power-law graph leave
// most lanes of a row-per-lane warp idle and make their shared loads conflict).
constexpr int kSegRows = 32;

// The work of block `bid` of `nblk` (a launch of its own, or one solve's share
// of a batched wave) is a function of (bid, nblk) only, so a solve gives the
// same bits whichever way its blocks are launched.
// Loads of the basis columns: through the read-only path, or (kCoh) through L1 with
// the coherence an acquire gives, for a kernel that reads columns its other blocks
// wrote earlier in the same launch (the persistent batch kernel).
template <bool kCoh, typename TV>
__device__ __forceinline__ TV ld_col(const TV* p) {
  if constexpr (kCoh) return *p;
  else return __ldg(p);
}

template <typename TV, int KW, bool SEG = false, bool kCoh = false>
__device__ __forceinline__ void spmv_dots_body(
    const Csr& A, TV* __restrict__ W, int64_t ld, int c, int j0, int kw, const ColScale& cs, double* __restrict__ H,
    int ldh, double* __restrict__ coef, double* __restrict__ part, unsigned* __restrict__ counter, DevState* st,
    int bid, int nblk, unsigned char* smem_raw) {
  constexpr int NV = KW > 0 ? KW : 1;  // window dot products per thread
  constexpr int S = kSpmvStages;
  TV* s_vals = reinterpret_cast<TV*>(smem_raw);                                // [S][kSpmvCap]
  int* s_col = reinterpret_cast<int*>(smem_raw + S * kSpmvCap * sizeof(TV));   // [S][kSpmvCap]
  const TV* Avals = reinterpret_cast<const TV*>(A.vals);
  // full[q]: the tile of stage q is in shared memory (or the stage holds a direct
  // tile); empty[q]: every warp is done with it, so it may be refilled.
  __shared__ __align__(8) uint64_t s_full[S], s_empty[S];
  __shared__ int s_e0[S];
  __shared__ int s_staged[S];
  __shared__ volatile int s_fail;
  __shared__ double sh[32 * NV];
  __shared__ double tot[NV];
  __shared__ TV s_red[kThreads / 32];
  // nonzero-parallel tiles (A.staged == 2): row starts in stage coordinates, and per
  // thread the sums of the row it continues (head) and of the row it leaves open (tail)
  constexpr int kSeg = SEG ? kThreads : 1;
  __shared__ int s_rp[kSeg + 1];
  __shared__ TV s_head[kSeg], s_tail[kSeg], s_yrow[kSeg];
  if (st->stop) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ntiles = A.ntiles;
  const TV* vin = W + (size_t)(c - 1) * ld;
  TV* wout = W + (size_t)c * ld;
  const int ksh = cs.shf[c - 1];
  double p2k_lo;
  const double p2k_hi = pow2_split(ksh, &p2k_lo);
  const TV p2k = (TV)(p2k_hi * p2k_lo);  // 2^ksh (only used for zeros / subnormals)
  TV acc[NV];  // per-thread partial sums (FP32 rows for the mixed path, FP64 across threads)
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = (TV)0;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&s_full[q], 1);
      mbar_init(&s_empty[q], kThreads / 32);
    }
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  // thread 0: fill stage i % S with the tile of iteration i, once every warp has
  // released that stage's previous tile. Staged copies are aligned to 4 entries so
  // that both start and end on 16-byte boundaries (the CSR arrays have 4 spare
  // entries); a tile that does not fit is read directly (full[] still completes).
  int last_it[S];
  for (int q = 0; q < S; ++q) last_it[q] = -1;
  auto issue = [&](int i) {
    const int tile = bid + i * nblk;
    const int stg = i % S;
    if (i >= S && !mbar_wait_bounded(&s_empty[stg], (uint32_t)((i / S - 1) & 1))) {
      s_fail = 1;  // the stage is still in use: leave it; its consumers time out too
      return;
    }
    const int r0 = A.tiles[tile], r1 = A.tiles[tile + 1];
    const int e0 = A.rowptr[r0], e1 = A.rowptr[r1];
    const int e0a = e0 & ~3, e1a = (e1 + 3) & ~3;
    const int cnt = e1a - e0a;
    last_it[stg] = i;
    if (A.staged && cnt > 0 && cnt <= kSpmvCap) {
      s_e0[stg] = e0a;
      s_staged[stg] = 1;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&s_full[stg], (uint32_t)cnt * (uint32_t)(sizeof(TV) + 4));
      bulk_copy_g2s(s_vals + stg * kSpmvCap, Avals + e0a, (uint32_t)cnt * (uint32_t)sizeof(TV), &s_full[stg]);
      bulk_copy_g2s(s_col + stg * kSpmvCap, A.colind + e0a, (uint32_t)cnt * 4u, &s_full[stg]);
    } else {
      s_staged[stg] = 0;
      mbar_arrive(&s_full[stg]);
    }
  };
  if (tid == 0)
    for (int i = 0; i < S - 1 && bid + i * nblk < ntiles; ++i) issue(i);
  // lanes 1..KW of warp 0: the window rows of the tile S-1 iterations ahead, into
  // L2 ahead of their loads (start rounded down, end up, to 16 bytes: within ld)
  auto prefetch_window = [&](int i) {
    const int q = tid - 1;
    const int tile = bid + i * nblk;
    if (q < 0 || q >= KW || tile >= ntiles) return;
    constexpr int kAl = 16 / (int)sizeof(TV);
    const int ra = A.tiles[tile] & ~(kAl - 1), rb = (A.tiles[tile + 1] + kAl - 1) & ~(kAl - 1);
    bulk_prefetch_l2_aligned(W + (size_t)(j0 + q) * ld + ra, (uint32_t)((size_t)(rb - ra) * sizeof(TV)));
  };
  for (int i = 0; i < S - 1; ++i) prefetch_window(i);
  int it = 0;
  for (int tile = bid; tile < ntiles; tile += nblk, ++it) {
    const int stg = it % S;
    if (tid == 0 && bid + (it + S - 1) * nblk < ntiles && !s_fail) issue(it + S - 1);
    prefetch_window(it + S - 1);
    // The tile's rows share the block: L = 256 / pow2ceil(rows) lanes per row
    // (one row per thread for full tiles, the whole block for a single long row);
    // each lane sums every L-th nonzero of its row, then the lanes of a row are
    // combined in a fixed order.
    const int r0 = A.tiles[tile], nr = A.tiles[tile + 1] - r0;
    const bool seg = SEG && A.staged == 2 && nr >= kSegRows;  // block-uniform
    const int lgL = seg ? 0 : 8 - (nr > 1 ? 32 - __clz(nr - 1) : 0);
    const int L = 1 << lgL;
    const int grp = tid >> lgL, lane_r = tid & (L - 1);
    const bool in_tile = grp < nr;
    const int r = r0 + grp;
    // Row bounds and window entries do not need the staged nonzeros. The FP32
    // path issues them before waiting for the tile so that their latency overlaps
    // the copy; the FP64 path (bound by its FP64 pipe) loses more by holding them
    // across the wait and issues them after it.
    constexpr bool kEarly = sizeof(TV) == 4;
    int e0 = 0, e1 = 0;
    TV wv[KW > 0 ? KW : 1];
    auto load_row = [&]() {
      if (in_tile) {
        e0 = A.rowptr[r];
        e1 = A.rowptr[r + 1];
        if (lane_r == 0) {
#pragma unroll
          for (int q = 0; q < KW; ++q) wv[q] = W[(size_t)(j0 + q) * ld + r];
        }
      }
    };
    if (kEarly) load_row();
    bool ok = !s_fail && mbar_wait_bounded(&s_full[stg], (uint32_t)((it / S) & 1));
    if (!kEarly) load_row();
    if (!ok) s_fail = 1;
    const bool staged = ok && s_staged[stg] != 0;
    const bool has_row = ok && in_tile;
    TV y = (TV)0;
    bool done = false;
    if constexpr (SEG) if (seg) {
      // Thread t takes the 8 staged entries 8t..8t+7 whatever rows they belong to
      // (conflict-free 16-byte shared loads, 8 independent gathers, no idle lanes on
      // short rows), sums them per row in order, and the rows are then assembled in a
      // fixed order: a row inside one thread from that thread's sum, a row spread over
      // threads ts..te from tail(ts) + head(ts+1) + ... + head(te).
      const int base = s_e0[stg];
      int rs = 0, re = 0;
      if (in_tile) {
        rs = e0 - base;
        re = e1 - base;
        s_rp[grp] = rs;
        if (grp == nr - 1) s_rp[nr] = re;
      }
      const int bad = __syncthreads_or(!ok);
      if (!bad && s_staged[stg]) {
        const int lo = s_rp[0], hi = s_rp[nr];
        const int a = 8 * tid;
        if (a < hi && a + 8 > lo) {
          int ci[8];
          TV av[8], g[8];
          const int* sc = s_col + stg * kSpmvCap + a;
          const TV* sv = s_vals + stg * kSpmvCap + a;
          *reinterpret_cast<int4*>(ci) = *reinterpret_cast<const int4*>(sc);
          *reinterpret_cast<int4*>(ci + 4) = *reinterpret_cast<const int4*>(sc + 4);
          if constexpr (sizeof(TV) == 4) {
            *reinterpret_cast<float4*>(av) = *reinterpret_cast<const float4*>(sv);
            *reinterpret_cast<float4*>(av + 4) = *reinterpret_cast<const float4*>(sv + 4);
          } else {
#pragma unroll
            for (int u = 0; u < 8; u += 2) *reinterpret_cast<double2*>(av + u) = *reinterpret_cast<const double2*>(sv + u);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) g[u] = (a + u >= lo && a + u < hi) ? ld_col<kCoh>(vin + ci[u]) : (TV)0;
          // the row of the first entry in the tile: the last row starting at or before it
          const int first = a > lo ? a : lo;
          int row = 0, top = nr;
          while (top - row > 1) {
            const int mid = (row + top) >> 1;
            if (s_rp[mid] <= first) row = mid;
            else top = mid;
          }
          int rbeg = s_rp[row], rend = s_rp[row + 1];
          TV sum = (TV)0;
          auto flush = [&]() {
            const bool before = rbeg < a, after = rend > a + 8;
            if (!before && !after) s_yrow[row] = sum;
            if (before) s_head[tid] = sum;
            if (after) s_tail[tid] = sum;
          };
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = a + u;
            if (e < lo || e >= hi) continue;
            while (e >= rend) {  // the current row ends before entry e
              flush();
              ++row;
              rbeg = rend;
              rend = s_rp[row + 1];
              sum = (TV)0;
            }
            sum = fma(av[u], g[u], sum);
          }
          flush();
        }
        __syncthreads();
        if (has_row && re > rs) {
          const int ts = rs >> 3, te = (re - 1) >> 3;
          if (ts == te) {
            y = s_yrow[grp];
          } else {
            y = s_tail[ts];
            for (int t = ts + 1; t < te; ++t) y += s_head[t];
            y += s_head[te];
          }
        }
        done = true;
      }
    }
    if (has_row && !done) {
      int e = e0 + lane_r;
      if (staged) {
        const int base = s_e0[stg];
        const TV* sv = s_vals + stg * kSpmvCap - base;
        const int* sc = s_col + stg * kSpmvCap - base;
        for (; e + 7 * L < e1; e += 8 * L) {  // eight gathers in flight per thread
          TV g[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) g[u] = ld_col<kCoh>(vin + sc[e + u * L]);
#pragma unroll
          for (int u = 0; u < 8; ++u) y = fma(sv[e + u * L], g[u], y);
        }
        if (e < e1) {  // tail: every index is clamped into the row, so no load can leave it
          const int rem = (e1 - e + L - 1) >> lgL;
          TV g[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) g[u] = ld_col<kCoh>(vin + sc[min(e + u * L, e1 - 1)]);
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (u < rem) y = fma(sv[e + u * L], g[u], y);
        }
      } else {  // same order of operations, operands from global memory
        for (; e + 7 * L < e1; e += 8 * L) {
          int cidx[8];
          TV av[8], g[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            cidx[u] = __ldg(A.colind + e + u * L);
            av[u] = __ldg(Avals + e + u * L);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) g[u] = ld_col<kCoh>(vin + cidx[u]);
#pragma unroll
          for (int u = 0; u < 8; ++u) y = fma(av[u], g[u], y);
        }
        for (; e < e1; e += L) y = fma(__ldg(Avals + e), ld_col<kCoh>(vin + __ldg(A.colind + e)), y);
      }
    }
    if (L > 1) {  // block-uniform branch: combine the lanes of each row
      for (int o = (L < 32 ? L : 32) >> 1; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
      if (L > 32) {
        if ((tid & 31) == 0) s_red[tid >> 5] = y;
        __syncthreads();
        if (lane_r == 0) {
          TV t = s_red[tid >> 5];
          for (int q = 1; q < (L >> 5); ++q) t += s_red[(tid >> 5) + q];
          y = t;
        }
        __syncthreads();  // s_red is free for the next such tile
      }
    }
    if (has_row && lane_r == 0) {
      y = scale_pow2(y, ksh, p2k);
      wout[r] = y;
#pragma unroll
      for (int q = 0; q < KW; ++q) acc[q] = fma(wv[q], y, acc[q]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&s_empty[stg]);  // this warp is done with the stage
  }
  __syncthreads();
  if (s_fail) {
    // A tile never arrived or a stage was never released: record it and give every
    // copy issued a bounded wait so that none lands in shared memory after exit.
    if (tid == 0) {
      st->status = FAB_ETIMEOUT;
      st->stop = 1;
      for (int q = 0; q < S; ++q)
        if (last_it[q] >= 0) mbar_wait_bounded(&s_full[q], (uint32_t)((last_it[q] / S) & 1));
    }
    __syncthreads();
    return;
  }
  if constexpr (KW == 0) {  // no window (Alg. 1, Arnoldi): only the scale of the new column
    if (bid == 0 && tid == 0) cs.scl[c] = column_tau(cs.sigma[c - 1], ksh);
    return;
  } else {
    double accd[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) accd[q] = (double)acc[q];
    block_sum_multi<NV>(accd, sh, tot);
    if (tid < NV) part[(size_t)bid * NV + tid] = tot[tid];
    if (!last_block(counter, (unsigned)nblk)) return;
    sum_partials_multi<NV>(part, nblk, tot, sh);
    const double tau = column_tau(cs.sigma[c - 1], ksh);
    if (tid < kw) {
      const int j = j0 + tid;
      const double d = tot[tid];
      H[j + (size_t)ldh * (c - 1)] = cs.sigma[j] * tau * d;
      coef[tid] = cs.sigma[j] * cs.sigma[j] * d;
    }
    if (tid == 0) {
      cs.scl[c] = tau;
      *counter = 0;
    }
  }
}

template <typename TV, int KW, bool SEG>
__global__ __launch_bounds__(kThreads) void k_spmv_dots(Csr A, TV* __restrict__ W, int64_t ld, int c, int j0, int kw,
                                                         ColScale cs, double* __restrict__ H, int ldh,
                                                         double* __restrict__ coef, double* __restrict__ part,
                                                         unsigned* __restrict__ counter, DevState* st, int gate) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (gate_closed(st, c, gate)) return;
  spmv_dots_body<TV, KW, SEG>(A, W, ld, c, j0, kw, cs, H, ldh, coef, part, counter, st, blockIdx.x, gridDim.x,
                              smem_raw);
}

template <typename TV>
const void* spmv_fn(int kw, bool seg) {
  static const void* fns[2][kMaxWindow + 1] = {
      {(const void*)k_spmv_dots<TV, 0, false>, (const void*)k_spmv_dots<TV, 1, false>,
       (const void*)k_spmv_dots<TV, 2, false>, (const void*)k_spmv_dots<TV, 3, false>,
       (const void*)k_spmv_dots<TV, 4, false>, (const void*)k_spmv_dots<TV, 5, false>,
       (const void*)k_spmv_dots<TV, 6, false>, (const void*)k_spmv_dots<TV, 7, false>,
       (const void*)k_spmv_dots<TV, 8, false>},
      {(const void*)k_spmv_dots<TV, 0, true>, (const void*)k_spmv_dots<TV, 1, true>,
       (const void*)k_spmv_dots<TV, 2, true>, (const void*)k_spmv_dots<TV, 3, true>,
       (const void*)k_spmv_dots<TV, 4, true>, (const void*)k_spmv_dots<TV, 5, true>,
       (const void*)k_spmv_dots<TV, 6, true>, (const void*)k_spmv_dots<TV, 7, true>,
       (const void*)k_spmv_dots<TV, 8, true>}};
  return fns[seg ? 1 : 0][kw];
}

// Blocks of one SpMV launch: every resident slot once (the nonzero-parallel form,
// seg, is a kernel of its own with its own occupancy).
template <typename TV>
int spmv_grid(int ntiles, int kw, bool seg) {
  static int occ[2][kMaxWindow + 1] = {{0}};
  int& o_kw = occ[seg ? 1 : 0][kw];
  if (o_kw == 0) {
    const size_t smem = (size_t)kSpmvStages * kSpmvCap * (sizeof(TV) + sizeof(int));
    ensure_smem_limit(spmv_fn<TV>(kw, seg), smem);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, spmv_fn<TV>(kw, seg), kThreads, smem);
    o_kw = o < 1 ? 1 : o;
  }
  const int grid = sm_count() * o_kw;
  return ntiles < grid ? (ntiles < 1 ? 1 : ntiles) : grid;
}
template int spmv_grid<double>(int, int, bool);
template int spmv_grid<float>(int, int, bool);

template <typename TV>
cudaError_t launch_spmv_dots(const Csr& A, TV* W, int64_t ld, int c, int j0, int kw, ColScale cs,
                             double* H, int ldh, double* coef, double* part, unsigned* counter,
                             DevState* st, cudaStream_t s, int gate) {
  if (kw < 0 || kw > kMaxWindow) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kSpmvStages * kSpmvCap * (sizeof(TV) + sizeof(int));
  const bool seg = A.staged == 2;
  const int grid = spmv_grid<TV>(A.ntiles, kw, seg);
  void* args[] = {(void*)&A, &W, &ld, &c, &j0, &kw, &cs, &H, &ldh, &coef, &part, &counter, &st, &gate};
  return cudaLaunchKernel(spmv_fn<TV>(kw, seg), dim3(grid), dim3(kThreads), args, smem, s);
}
template cudaError_t launch_spmv_dots<double>(const Csr&, double*, int64_t, int, int, int, ColScale, double*, int,
                                              double*, double*, unsigned*, DevState*, cudaStream_t, int);
template cudaError_t launch_spmv_dots<float>(const Csr&, float*, int64_t, int, int, int, ColScale, double*, int,
                                             double*, double*, unsigned*, DevState*, cudaStream_t, int);

// The sparse-sign pattern transposed per chunk (one block per 4096-row chunk): count
// the rows that hit each sketch row, scan the counts into the offsets, then place each
// row (and its sign) in its sketch rows' lists. Order inside a list is not fixed; the
// sums taken over it are exact in int64, so the sketch does not depend on it.
__global__ void k_sparse_pattern(int n, SketchDev sk, unsigned char* __restrict__ tab) {
  extern __shared__ int s_cnt[];  // s counts, then s cursors
  int* s_pos = s_cnt + sk.s;
  const int chunk = blockIdx.x;
  unsigned char* rec = tab + (size_t)chunk * sparse_rec_bytes(sk.s, sk.zeta);
  unsigned* off = reinterpret_cast<unsigned*>(rec);
  unsigned short* ent = reinterpret_cast<unsigned short*>(rec + sparse_off_bytes(sk.s));
  for (int q = threadIdx.x; q < sk.s; q += blockDim.x) s_cnt[q] = 0;
  __syncthreads();
  for (int rl = threadIdx.x; rl < kChunk; rl += blockDim.x) {
    const long long j = (long long)chunk * kChunk + rl;
    if (j >= n) break;
    int rows[kMaxZeta];
    sparse_rows(sk, j, rows);
#pragma unroll
    for (int q = 0; q < kMaxZeta; ++q)
      if (q < sk.zeta) atomicAdd(&s_cnt[rows[q]], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned a = 0;
    for (int q = 0; q < sk.s; ++q) {
      off[q] = a;
      s_pos[q] = (int)a;
      a += (unsigned)s_cnt[q];
    }
    off[sk.s] = a;
  }
  __syncthreads();
  for (int rl = threadIdx.x; rl < kChunk; rl += blockDim.x) {
    const long long j = (long long)chunk * kChunk + rl;
    if (j >= n) break;
    int rows[kMaxZeta];
    sparse_rows(sk, j, rows);
    const unsigned long long sg = rng_u(sk.st_signs, (unsigned long long)j);
#pragma unroll
    for (int q = 0; q < kMaxZeta; ++q)
      if (q < sk.zeta) {
        const int p = atomicAdd(&s_pos[rows[q]], 1);
        ent[p] = (unsigned short)(rl | (((sg >> q) & 1ull) << 15));
      }
  }
}

cudaError_t launch_sparse_pattern(int n, const SketchDev& sk, unsigned short* pat, cudaStream_t s) {
  if (sk.s < 1 || sk.s > kMaxS || sk.zeta < 1 || sk.zeta > kMaxZeta) return cudaErrorInvalidValue;
  const int nchunks = (n + kChunk - 1) / kChunk;
  if (nchunks < 1) return cudaSuccess;
  const size_t smem = (size_t)2 * sk.s * sizeof(int);
  if (smem > 48 * 1024) {
    const cudaError_t e = ensure_smem_limit((const void*)k_sparse_pattern, smem);
    if (e != cudaSuccess) return e;
  }
  k_sparse_pattern<<<nchunks, 256, smem, s>>>(n, sk, reinterpret_cast<unsigned char*>(pat));
  return cudaGetLastError();
}

template <int SK, typename TV>
__device__ __forceinline__ void update_body(int n, TV* __restrict__ W, int64_t ld, int c, int j0, int nc,
                                            const double* __restrict__ coef, double* __restrict__ H, int ldh,
                                            const ColScale& cs, int mode,
                                            double* __restrict__ part, unsigned* __restrict__ counter,
                                            const SketchDev& sk, DevState* st, int bid, int nblk,
                                            unsigned char* smem_raw) {
  __shared__ double sh[32];
  __shared__ double tot[1];
  __shared__ int s_int[32];
  if (st->stop) return;
  TV* s_coef = reinterpret_cast<TV*>(smem_raw);  // nc coefficients
  double* s_acc = reinterpret_cast<double*>(smem_raw + ((size_t)nc * 8 + 15) / 16 * 16);  // s doubles
  const bool sk_acc = (SK == SK_SRHT || SK == SK_SPARSE || SK == SK_SPARSE_TAB);
  unsigned char* after = reinterpret_cast<unsigned char*>(s_acc) + ((size_t)(sk_acc ? sk.s : 0) * 8 + 15) / 16 * 16;
  long long* buf = reinterpret_cast<long long*>(after);                     // SRHT: pidx(4096) int64
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(after);   // sparse: s uint64
  int* s_P = reinterpret_cast<int*>(after + (size_t)(kChunk + kChunk / 16) * 8);  // SRHT: s ints
  for (int i = threadIdx.x; i < nc; i += kThreads) s_coef[i] = (TV)coef[i];
  if (sk_acc)
    for (int q = threadIdx.x; q < sk.s; q += kThreads) s_acc[q] = 0.0;
  if (SK == SK_SRHT)
    for (int q = threadIdx.x; q < sk.s; q += kThreads) s_P[q] = sk.P[q];
  if (SK == SK_SPARSE || SK == SK_SPARSE_TAB)
    for (int q = threadIdx.x; q < sk.s; q += kThreads) acc[q] = 0ull;
  __syncthreads();
  TV* wc = W + (size_t)c * ld;
  const TV* Wb = W + (size_t)j0 * ld;
  double nrm = 0.0;
  // FP64 with the SRHT: the norm comes exactly from the sketch's fixed-point integers
  // (sketch_chunk_srht), which frees the FP64 pipe of one FMA per row
  constexpr bool kIntNorm = SK == SK_SRHT && sizeof(TV) == 8;
  const int nchunks = (n + kChunk - 1) / kChunk;
  for (int chunk = bid; chunk < nchunks; chunk += nblk) {
    const int base = chunk * kChunk + threadIdx.x;
    TV v[kRowsPerThread];
    TV nrm_c = (TV)0;  // this chunk's share in the element type, added to nrm in FP64
    if ((chunk + 1) * kChunk <= n) {
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) v[i] = wc[base + i * kThreads];
      for (int q = 0; q < nc; ++q) {
        const TV cf = s_coef[q];
        const TV* col = Wb + (size_t)q * ld + base;
#pragma unroll
        for (int i = 0; i < kRowsPerThread; ++i) v[i] = fma(-cf, col[i * kThreads], v[i]);
      }
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        if (nc > 0) wc[base + i * kThreads] = v[i];
        if (!kIntNorm) nrm_c = fma(v[i], v[i], nrm_c);
      }
    } else {  // last, partial chunk: every load index is clamped to a valid row
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        const TV t = wc[min(base + i * kThreads, n - 1)];
        v[i] = (base + i * kThreads < n) ? t : (TV)0;
      }
      for (int q = 0; q < nc; ++q) {
        const TV cf = s_coef[q];
        const TV* col = Wb + (size_t)q * ld;
#pragma unroll
        for (int i = 0; i < kRowsPerThread; ++i) {
          const TV t = col[min(base + i * kThreads, n - 1)];
          if (base + i * kThreads < n) v[i] = fma(-cf, t, v[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        if (base + i * kThreads < n) {
          if (nc > 0) wc[base + i * kThreads] = v[i];
          if (!kIntNorm) nrm_c = fma(v[i], v[i], nrm_c);
        }
      }
    }
    nrm += (double)nrm_c;
    if (SK == SK_SRHT) sketch_chunk_srht<TV, true>(v, chunk, sk, buf, s_P, s_acc, s_int, kIntNorm ? &nrm : nullptr);
    if (SK == SK_SPARSE) sketch_chunk_sparse<TV, false>(v, chunk, n, sk, acc, s_acc, s_int);
    if (SK == SK_SPARSE_TAB) sketch_chunk_sparse<TV, true>(v, chunk, n, sk, acc, s_acc, s_int);
    if (SK == SK_GAUSS) {  // two-term BF16 copy of the column for the tensor-core Gaussian sketch
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i)
        if (base + i * kThreads < n) {
          const float x = (float)v[i];
          const __nv_bfloat16 hi = __float2bfloat16_rn(x);
          const int64_t r = base + i * kThreads;
          sk.Wbf[gauss_bidx(r, c, 0, sk.bf_cpad)] = hi;
          sk.Wbf[gauss_bidx(r, c, 1, sk.bf_cpad)] = __float2bfloat16_rn(x - __bfloat162float(hi));  // exact in FP32
        }
    }
  }
  if (sk_acc) {  // this block's share of the sketch (its chunks, fixed order)
    double* out = sk.part + (size_t)bid * sk.s;
    for (int q = threadIdx.x; q < sk.s; q += kThreads) out[q] = s_acc[q];
  }
  if (!(mode & kModeNorm)) return;
  column_norm_tail(nrm, c, j0, H, ldh, cs, mode, part, counter, st, bid, nblk, sh, tot);
}

template <int SK, typename TV>
__global__ __launch_bounds__(kThreads, SK == SK_SPARSE ? 2 : 3) void k_update(
    int n, TV* __restrict__ W, int64_t ld, int c, int j0, int nc, const double* __restrict__ coef,
    double* __restrict__ H, int ldh, ColScale cs, int mode, double* __restrict__ part,
    unsigned* __restrict__ counter, SketchDev sk, DevState* st, int gate) {
  extern __shared__ __align__(16) unsigned char smem_upd[];
  if (gate_closed(st, c, gate)) return;
  update_body<SK, TV>(n, W, ld, c, j0, nc, coef, H, ldh, cs, mode, part, counter, sk, st, blockIdx.x, gridDim.x,
                      smem_upd);
}

size_t update_smem_bytes(int kind, int nc, int s) {
  size_t b = ((size_t)nc * 8 + 15) / 16 * 16;
  if (kind == SK_SRHT || kind == SK_SPARSE || kind == SK_SPARSE_TAB) b += ((size_t)s * 8 + 15) / 16 * 16;
  if (kind == SK_SRHT) b += (size_t)(kChunk + kChunk / 16) * 8 + (size_t)s * 4;
  if (kind == SK_SPARSE || kind == SK_SPARSE_TAB) b += ((size_t)s * 8 + 15) / 16 * 16;
  if (kind == SK_SPARSE_TAB) b += (size_t)kChunk * 8;  // the chunk's X for the gather
  return b;
}

template <typename TV>
const void* update_fn(int kind) {
  switch (kind) {
    case SK_SRHT: return (const void*)k_update<SK_SRHT, TV>;
    case SK_SPARSE: return (const void*)k_update<SK_SPARSE, TV>;
    case SK_SPARSE_TAB: return (const void*)k_update<SK_SPARSE_TAB, TV>;
    case SK_GAUSS: return (const void*)k_update<SK_GAUSS, TV>;
    default: return (const void*)k_update<SK_NONE, TV>;
  }
}

template <typename TV>
int update_grid(int kind, int n, int nc, int s, size_t* smem_out) {
  const size_t smem = update_smem_bytes(kind, nc, s);
  if (smem_out) *smem_out = smem;
  const void* fn = update_fn<TV>(kind);
  if (ensure_smem_limit(fn, smem) != cudaSuccess) return -1;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
  if (occ < 1) occ = 1;
  const int nchunks = (n + kChunk - 1) / kChunk;
  const int grid = sm_count() * occ;
  return nchunks < grid ? (nchunks < 1 ? 1 : nchunks) : grid;
}
template int update_grid<double>(int, int, int, int, size_t*);
template int update_grid<float>(int, int, int, int, size_t*);

template <typename TV>
cudaError_t launch_update(int n, TV* W, int64_t ld, int c, int j0, int nc, const double* coef, double* H, int ldh,
                          ColScale cs, int mode, double* part, unsigned* counter, SketchDev& sk,
                          DevState* st, cudaStream_t s, int gate) {
  size_t smem = 0;
  const int kind = (sk.kind == SK_SPARSE && sk.pat) ? SK_SPARSE_TAB : sk.kind;
  const int grid = update_grid<TV>(kind, n, nc, sk.s, &smem);
  if (grid < 1) return cudaErrorInvalidValue;
  const void* fn = update_fn<TV>(kind);
  sk.nparts = grid;  // one sketch partial per block
  void* args[] = {&n, &W, &ld, &c, &j0, &nc, (void*)&coef, &H, &ldh, &cs, &mode, &part, &counter, &sk, &st, &gate};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, s);
}
template cudaError_t launch_update<double>(int, double*, int64_t, int, int, int, const double*, double*, int,
                                           ColScale, int, double*, unsigned*, SketchDev&, DevState*, cudaStream_t,
                                           int);
template cudaError_t launch_update<float>(int, float*, int64_t, int, int, int, const double*, double*, int, ColScale,
                                          int, double*, unsigned*, SketchDev&, DevState*, cudaStream_t, int);

// ------------------------------------------------- window update without a sketch
// W_c <- W_c - sum_q coef_q W_{j0+q} (KW window columns, a compile-time count) and
// ||W_c||^2 with the same bookkeeping as k_update (column_norm_tail). A thread takes
// kPlainU rows per pass and issues all their (KW+1) loads before the first FMA, so a
// row group waits for one memory latency instead of one per column; the FMAs run in
// the same order as in k_update, so the column is bit-identical. Used for the basis
// steps that take no sketch; with a sketch the fused k_update stays faster than this
// kernel followed by a sketch-only pass (measured: 104 against 134 us per FP64 step).
constexpr int kPlainU = 4;
template <typename TV, int KW>
__global__ __launch_bounds__(kThreads) void k_update_plain(int n, TV* __restrict__ W, int64_t ld, int c, int j0,
                                                           const double* __restrict__ coef, double* __restrict__ H,
                                                           int ldh, ColScale cs,
                                                           int mode, double* __restrict__ part,
                                                           unsigned* __restrict__ counter, DevState* st) {
  __shared__ double sh[32];
  __shared__ double tot[1];
  if (st->stop) return;
  TV cf[KW > 0 ? KW : 1];
#pragma unroll
  for (int q = 0; q < KW; ++q) cf[q] = (TV)coef[q];
  TV* wc = W + (size_t)c * ld;
  const TV* Wb = W + (size_t)j0 * ld;
  double nrm = 0.0;
  const int64_t step = (int64_t)gridDim.x * kThreads * kPlainU;
  for (int64_t r0 = (int64_t)blockIdx.x * kThreads * kPlainU + threadIdx.x; r0 < n; r0 += step) {
    TV v[kPlainU], w[kPlainU][KW > 0 ? KW : 1];
#pragma unroll
    for (int u = 0; u < kPlainU; ++u) {
      const int64_t r = r0 + (int64_t)u * kThreads;
      const int64_t rr = r < n ? r : n - 1;  // clamped: every load stays in the column
      v[u] = wc[rr];
#pragma unroll
      for (int q = 0; q < KW; ++q) w[u][q] = Wb[(size_t)q * ld + rr];
    }
    TV nrm_g = (TV)0;
#pragma unroll
    for (int u = 0; u < kPlainU; ++u) {
      const int64_t r = r0 + (int64_t)u * kThreads;
      if (r >= n) continue;
      TV x = v[u];
#pragma unroll
      for (int q = 0; q < KW; ++q) x = fma(-cf[q], w[u][q], x);
      if (KW > 0) wc[r] = x;
      nrm_g = fma(x, x, nrm_g);
    }
    nrm += (double)nrm_g;
  }
  if (!(mode & kModeNorm)) return;
  column_norm_tail(nrm, c, j0, H, ldh, cs, mode, part, counter, st, blockIdx.x, gridDim.x, sh, tot);
}

template <typename TV>
const void* plain_fn(int kw) {
  static const void* fns[kMaxWindow + 1] = {
      (const void*)k_update_plain<TV, 0>, (const void*)k_update_plain<TV, 1>, (const void*)k_update_plain<TV, 2>,
      (const void*)k_update_plain<TV, 3>, (const void*)k_update_plain<TV, 4>, (const void*)k_update_plain<TV, 5>,
      (const void*)k_update_plain<TV, 6>, (const void*)k_update_plain<TV, 7>, (const void*)k_update_plain<TV, 8>};
  return fns[kw];
}

template <typename TV>
cudaError_t launch_update_plain(int n, TV* W, int64_t ld, int c, int j0, int kw, const double* coef, double* H,
                                int ldh, ColScale cs, int mode, double* part, unsigned* counter,
                                DevState* st, cudaStream_t s) {
  if (kw < 0 || kw > kMaxWindow) return cudaErrorInvalidValue;
  static int occ[kMaxWindow + 1] = {0};
  if (occ[kw] == 0) {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, plain_fn<TV>(kw), kThreads, 0);
    occ[kw] = o < 1 ? 1 : o;
  }
  const int64_t need = ((int64_t)n + (int64_t)kThreads * kPlainU - 1) / ((int64_t)kThreads * kPlainU);
  const int cap = sm_count() * occ[kw];
  const int grid = (int)(need < 1 ? 1 : (need < cap ? need : cap));
  void* args[] = {&n, &W, &ld, &c, &j0, (void*)&coef, &H, &ldh, &cs, &mode, &part, &counter, &st};
  return cudaLaunchKernel(plain_fn<TV>(kw), dim3(grid), dim3(kThreads), args, 0, s);
}
template cudaError_t launch_update_plain<double>(int, double*, int64_t, int, int, int, const double*, double*, int,
                                                 ColScale, int, double*, unsigned*, DevState*, cudaStream_t);
template cudaError_t launch_update_plain<float>(int, float*, int64_t, int, int, int, const double*, double*, int,
                                                ColScale, int, double*, unsigned*, DevState*, cudaStream_t);

// ---------------------------------------------- cross-block sketch reduce
// out[q] = scale * sigma[col] * sum_blocks part[block][q] (the per-block partials
// of k_update already carry the cross-chunk Hadamard signs); one warp per
// sketch row, fixed order.
__device__ __forceinline__ void sketch_reduce_body(const SketchDev& sk, int nparts, const double* __restrict__ sigma,
                                                   int col, double scale, double* __restrict__ out, DevState* st,
                                                   int bid) {
  if (st->stop) return;
  const int q = (bid * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= sk.s) return;
  double a = 0.0;
  for (int b = lane; b < nparts; b += 32) a += sk.part[(size_t)b * sk.s + q];
  a = warp_sum(a);
  if (lane == 0) out[q] = a * scale * (sigma ? sigma[col] : 1.0);
}

__global__ void k_sketch_reduce(SketchDev sk, const double* __restrict__ sigma, int col, double scale,
                                double* __restrict__ out, DevState* st, int gate) {
  if (gate_closed(st, col, gate)) return;
  sketch_reduce_body(sk, sk.nparts, sigma, col, scale, out, st, blockIdx.x);
}

cudaError_t launch_sketch_reduce(const SketchDev& sk, const double* sigma, int col, double scale, double* out,
                                 DevState* st, cudaStream_t s, int gate) {
  const int warps_per_block = 8;
  const int grid = (sk.s + warps_per_block - 1) / warps_per_block;
  k_sketch_reduce<<<grid, warps_per_block * 32, 0, s>>>(sk, sigma, col, scale, out, st, gate);
  return cudaGetLastError();
}

// Deferred form: the partials of columns c0..c0+ncols-1 lie colstride doubles apart
// (nparts blocks each) and one launch reduces them all, one warp per (column,
// sketch row), with the arithmetic and order of sketch_reduce_body. Only the columns
// the per-step reduce would have written are written: those below m_used, and
// m_used itself unless the basis loop stopped there (a breakdown or an error).
__global__ void k_sketch_reduce_cols(SketchDev sk, size_t colstride, int c0, int ncols, int nparts,
                                     const double* __restrict__ sigma, double scale, double* __restrict__ SV,
                                     const DevState* st) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)ncols * sk.s) return;
  const int col = c0 + (int)(wid / sk.s), q = (int)(wid % sk.s);
  const int mu = st->m_used;
  if (!(col < mu || (col == mu && !st->stop))) return;
  const double* part = sk.part + (size_t)col * colstride;
  double a = 0.0;
  for (int b = lane; b < nparts; b += 32) a += part[(size_t)b * sk.s + q];
  a = warp_sum(a);
  if (lane == 0) SV[(size_t)col * sk.s + q] = a * scale * sigma[col];
}

cudaError_t launch_sketch_reduce_cols(const SketchDev& sk, size_t colstride, int c0, int ncols, int nparts,
                                      const double* sigma, double scale, double* SV, const DevState* st,
                                      cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const int warps_per_block = 8;
  const long long warps = (long long)ncols * sk.s;
  const int grid = (int)((warps + warps_per_block - 1) / warps_per_block);
  k_sketch_reduce_cols<<<grid, warps_per_block * 32, 0, s>>>(sk, colstride, c0, ncols, nparts, sigma, scale, SV, st);
  return cudaGetLastError();
}

// ------------------------------------------------------ SRHT row sampling
// Floyd's algorithm: for i = 0..s-1, j = n'-s+i, t = floor(u(seed,4,i) (j+1) / 2^64);
// take t unless already taken, else j. Then the rows are sorted (bitonic).
__global__ void k_srht_sample(int64_t npad, int s, uint64_t stP, int* __restrict__ P) {
  __shared__ int S[kMaxS];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = 0; i < s; ++i) {
      const long long j = npad - s + i;
      const unsigned long long t = __umul64hi(rng_u(stP, (unsigned long long)i), (unsigned long long)(j + 1));
      bool found = false;
      for (int q = lane; q < i; q += 32) found |= (S[q] == (int)t);
      found = __any_sync(0xffffffffu, found);
      if (lane == 0) S[i] = found ? (int)j : (int)t;
      __syncwarp();
    }
  }
  __syncthreads();
  int L = 1;
  while (L < s) L <<= 1;
  for (int i = s + threadIdx.x; i < L; i += blockDim.x) S[i] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= L; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const int a = S[i], b = S[ixj];
          if ((a > b) == up) {
            S[i] = b;
            S[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) P[i] = S[i];
}

cudaError_t launch_srht_sample(int64_t npad, int s, uint64_t stP, int* P, cudaStream_t st) {
  k_srht_sample<<<1, 1024, 0, st>>>(npad, s, stP, P);
  return cudaGetLastError();
}

// ------------------------------------------------------------- GEMV-T pass
// part[tile][q] = sum over the tile's rows of W_{j0+q}[r] x[r]; one warp per column.
template <typename TV, typename TX>
__global__ __launch_bounds__(kThreads) void k_gemv_t(int n, const TV* __restrict__ W, int64_t ld, int j0, int nc,
                                                      const TX* __restrict__ x, double* __restrict__ part,
                                                      DevState* st) {
  __shared__ TV xs[kTileRows];
  if (st && (st->stop || st->flag)) return;  // flag: an LSQR loop has converged
  const int tile = blockIdx.x;
  const int r0 = tile * kTileRows;
  const int rows = min(kTileRows, n - r0);
  for (int i = threadIdx.x; i < rows; i += kThreads) xs[i] = (TV)x[r0 + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int col = warp; col < nc; col += kThreads / 32) {
    const TV* wcol = W + (size_t)(j0 + col) * ld + r0;
    TV a0 = (TV)0, a1 = (TV)0;
    int i = lane;
    for (; i + 32 < rows; i += 64) {
      a0 = fma(wcol[i], xs[i], a0);
      a1 = fma(wcol[i + 32], xs[i + 32], a1);
    }
    if (i < rows) a0 = fma(wcol[min(i, rows - 1)], xs[min(i, rows - 1)], a0);
    const double a = warp_sum((double)a0 + (double)a1);
    if (lane == 0) part[(size_t)tile * nc + col] = a;
  }
}

template <typename TV, typename TX>
cudaError_t launch_gemv_t(int n, const TV* W, int64_t ld, int j0, int nc, const TX* x, double* part, int ntiles,
                          DevState* st, cudaStream_t s) {
  k_gemv_t<TV, TX><<<ntiles, kThreads, 0, s>>>(n, W, ld, j0, nc, x, part, st);
  return cudaGetLastError();
}
template cudaError_t launch_gemv_t<double, double>(int, const double*, int64_t, int, int, const double*, double*, int,
                                                   DevState*, cudaStream_t);
template cudaError_t launch_gemv_t<float, float>(int, const float*, int64_t, int, int, const float*, double*, int,
                                                 DevState*, cudaStream_t);
template cudaError_t launch_gemv_t<float, double>(int, const float*, int64_t, int, int, const double*, double*, int,
                                                  DevState*, cudaStream_t);

// d_q = sum over tiles of part[tile][q] (fixed order), then with j = j0+q:
//   Hcol[j] = sigma_j sig_col d_q (or += when h_accumulate; sig_col = 1 when NULL),
//   coef[q] = sigma_j^2 d_q (update coefficient of a raw column).
__global__ void k_reduce_cols(const double* __restrict__ part, int ntiles, int nc, const double* __restrict__ sigma,
                              int j0, const double* __restrict__ sig_col, double* __restrict__ Hcol, int h_accumulate,
                              double* __restrict__ coef, DevState* st) {
  if (st && (st->stop || st->flag)) return;  // flag: an LSQR loop has converged
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nc) return;
  double a = 0.0;
  for (int t = lane; t < ntiles; t += 32) a += part[(size_t)t * nc + q];
  a = warp_sum(a);
  if (lane == 0) {
    const int j = j0 + q;
    const double h = sigma[j] * (sig_col ? *sig_col : 1.0) * a;
    if (Hcol) Hcol[j] = h_accumulate ? Hcol[j] + h : h;
    if (coef) coef[q] = sigma[j] * sigma[j] * a;
  }
}

cudaError_t launch_reduce_cols(const double* part, int ntiles, int nc, const double* sigma, int j0,
                               const double* sig_col, double* Hcol, int h_accumulate, double* coef, DevState* st,
                               cudaStream_t s) {
  const int grid = (nc + 7) / 8;
  k_reduce_cols<<<grid, 256, 0, s>>>(part, ntiles, nc, sigma, j0, sig_col, Hcol, h_accumulate, coef, st);
  return cudaGetLastError();
}

// ---------------------------------------------------- FMA throughput probe
// Eight independent chains x = fma(x, a, b) per thread, 16 rounds per loop trip, on
// every SM: the FP64 (or FP32) pipe's fused multiply-add rate at the clocks the GPU
// runs now. a and b arrive as arguments, so nothing folds; |a| < 1 keeps every chain
// bounded (x tends to b / (1 - a)); the sum is stored only if it equals an impossible
// value, which the compiler cannot prove false.
__device__ double g_fma_sink;
// The FMA pipe's rate depends on how the operands of an FMA fall on the register
// banks, so the kernel comes in three operand patterns and the caller keeps the
// fastest: P0 the same multiplier and addend for every chain, P1 and P2 four and two
// different ones (on GB300 P1 and P2 run 13 % faster in FP64 than P0).
template <typename T, int P>
__global__ __launch_bounds__(kThreads) void k_fma_peak(int iters, T a0, T b0) {
  T x[8], a[4], b[4];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = (T)(threadIdx.x * 8 + q) * (T)1e-3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a[q] = a0 - (T)q * (T)1e-6;
    b[q] = b0 + (T)q * (T)1e-9;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (P == 0) x[q] = fma(x[q], a0, b0);
        else if (P == 1) x[q] = fma(x[q], a[q & 3], b[(q >> 2) & 3]);
        else x[q] = fma(x[q], a[(q >> 1) & 3], b[q & 1]);
      }
    }
  }
  T t = (T)0;
#pragma unroll
  for (int q = 0; q < 8; ++q) t += x[q];
  if (t == (T)-1.25) g_fma_sink = (double)t;
}

template <typename T>
cudaError_t launch_fma_peak(int pattern, int blocks_per_sm, int iters, cudaStream_t s, double* fmas) {
  const int grid = sm_count() * blocks_per_sm;
  const T a = (T)0.999999, b = (T)1e-7;
  if (pattern == 0) k_fma_peak<T, 0><<<grid, kThreads, 0, s>>>(iters, a, b);
  else if (pattern == 1) k_fma_peak<T, 1><<<grid, kThreads, 0, s>>>(iters, a, b);
  else k_fma_peak<T, 2><<<grid, kThreads, 0, s>>>(iters, a, b);
  if (fmas) *fmas = (double)grid * kThreads * (double)iters * 16.0 * 8.0;
  return cudaGetLastError();
}
template cudaError_t launch_fma_peak<double>(int, int, int, cudaStream_t, double*);
template cudaError_t launch_fma_peak<float>(int, int, int, cudaStream_t, double*);

// -------------------------------------------------------------- combine
// out[r] = keep * out[r] + sum_q coef[q] W_q[r]   (keep = 0 overwrites out)
template <typename TV>
__global__ __launch_bounds__(kThreads) void k_combine(int n, const TV* __restrict__ W, int64_t ld, int nc,
                                                       const double* __restrict__ coef, double* __restrict__ out,
                                                       double keep) {
  extern __shared__ double s_cf[];
  combine_coef_load<TV>(s_cf, coef, nc);
  __syncthreads();
  for (int r = blockIdx.x * kThreads + threadIdx.x; r < n; r += gridDim.x * kThreads) {
    const double a = combine_row<TV>(W, ld, nc, s_cf, r);
    out[r] = (keep != 0.0) ? fma(keep, out[r], a) : a;
  }
}

template <typename TV>
cudaError_t launch_combine(int n, const TV* W, int64_t ld, int nc, const double* coef, double* out, double keep,
                           cudaStream_t s) {
  k_combine<TV><<<grid_rows(n), kThreads, (size_t)(nc > 0 ? nc : 1) * 8, s>>>(n, W, ld, nc, coef, out, keep);
  return cudaGetLastError();
}
template cudaError_t launch_combine<double>(int, const double*, int64_t, int, const double*, double*, double,
                                            cudaStream_t);
template cudaError_t launch_combine<float>(int, const float*, int64_t, int, const double*, double*, double,
                                           cudaStream_t);

// ------------------------------------------------- explicit whitened column
// W_c <- sum_{q<=c} coef[q] W_q, row by row: a thread reads all of its row before
// writing it and no other thread touches that row, so the update is in place.
template <typename TV>
__global__ __launch_bounds__(kThreads) void k_whiten_column(int n, TV* __restrict__ W, int64_t ld, int c,
                                                             const double* __restrict__ coef, DevState* st) {
  extern __shared__ double s_cf[];
  if (st->stop || *(volatile const int*)&st->wh != c + 1) return;
  for (int i = threadIdx.x; i <= c; i += kThreads) s_cf[i] = coef[i];
  __syncthreads();
  for (int r = blockIdx.x * kThreads + threadIdx.x; r < n; r += gridDim.x * kThreads) {
    double a = 0.0;
    for (int q = 0; q <= c; ++q) a = fma(s_cf[q], (double)W[(size_t)q * ld + r], a);
    W[(size_t)c * ld + r] = (TV)a;
  }
}

template <typename TV>
cudaError_t launch_whiten_column(int n, TV* W, int64_t ld, int c, const double* coef, DevState* st,
                                 cudaStream_t s) {
  if (c < 0 || c > kMaxM) return cudaErrorInvalidValue;
  k_whiten_column<TV><<<grid_rows(n), kThreads, (size_t)(c + 1) * 8, s>>>(n, W, ld, c, coef, st);
  return cudaGetLastError();
}
template cudaError_t launch_whiten_column<double>(int, double*, int64_t, int, const double*, DevState*, cudaStream_t);
template cudaError_t launch_whiten_column<float>(int, float*, int64_t, int, const double*, DevState*, cudaStream_t);

// dst_j = sigma_j W_j (normalized basis for inspection)
template <typename TV>
__global__ void k_scale_columns(int n, const TV* __restrict__ W, int64_t ld, int nc, const double* __restrict__ sigma,
                                double* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  if (j >= nc) return;
  const double sg = sigma[j];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    dst[(size_t)j * ldd + r] = sg * (double)W[(size_t)j * ld + r];
}

template <typename TV>
cudaError_t launch_scale_columns(int n, const TV* W, int64_t ld, int nc, const double* sigma, double* dst,
                                 int64_t ldd, cudaStream_t s) {
  dim3 grid((unsigned)min((n + 255) / 256, 1024), (unsigned)nc);
  k_scale_columns<TV><<<grid, 256, 0, s>>>(n, W, ld, nc, sigma, dst, ldd);
  return cudaGetLastError();
}
template cudaError_t launch_scale_columns<double>(int, const double*, int64_t, int, const double*, double*, int64_t,
                                                  cudaStream_t);
template cudaError_t launch_scale_columns<float>(int, const float*, int64_t, int, const double*, double*, int64_t,
                                                 cudaStream_t);

// y = A x, one thread per row, FP64 (the starting vector A b of sign(A) b).
__global__ void k_csr_spmv(int n, const int* __restrict__ rowptr, const int* __restrict__ colind,
                           const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) a = fma(vals[e], x[colind[e]], a);
    y[r] = a;
  }
}

cudaError_t launch_csr_spmv(int n, const int* rowptr, const int* colind, const double* vals, const double* x,
                            double* y, cudaStream_t s) {
  k_csr_spmv<<<grid_rows(n), kThreads, 0, s>>>(n, rowptr, colind, vals, x, y);
  return cudaGetLastError();
}

// FP64 -> FP32 copy (start vector of the mixed-precision path)
__global__ void k_to_f32(int n, const double* __restrict__ x, float* __restrict__ y) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) y[r] = (float)x[r];
}

cudaError_t launch_to_f32(int n, const double* x, float* y, cudaStream_t s) {
  k_to_f32<<<grid_rows(n), kThreads, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------- batched basis
// A wave lists solves and their blocks: job ids[i] owns blocks pre[i] ..
// pre[i+1]-1 (its own launch's grid). wave_slot finds the entry of block b.
__device__ __forceinline__ int wave_slot(const Wave& w, int b) {
  int lo = 0, hi = w.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(w.pre + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// state reset, counters, H = 0, W_0 = b (FP64 -> TV)
template <typename TV>
__device__ __forceinline__ void init_body(const BasisJob<TV>* J, int bid, int nblk) {
  const int n = J->A.n, m = J->m;
  if (bid == 0 && threadIdx.x == 0) {
    DevState* st = J->st;
    st->m_used = m;
    st->stop = 0;
    st->status = FAB_OK;
    st->flag = 0;
    st->iters = 0;
    st->beta = 0.0;
    for (int q = 0; q < 16; ++q) st->scal[q] = 0.0;
    st->kappa = 0.0;
  }
  if (bid == 0 && threadIdx.x < 16) J->counter[threadIdx.x] = 0u;
  const int nh = J->ldh * m;
  for (int q = bid * blockDim.x + threadIdx.x; q < nh; q += nblk * blockDim.x) J->H[q] = 0.0;
  for (int r = bid * blockDim.x + threadIdx.x; r < n; r += nblk * blockDim.x) J->W[r] = (TV)J->b[r];
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The phase bodies of the persistent kernel are separate (not inlined) functions, so
// that each keeps the register allocation of its own kernel instead of sharing one
// allocation with every other phase.
template <typename TV, int KW>
__device__ __noinline__ void spmv_phase_kw(const BasisJob<TV>* J, int c, int bid, int nblk, unsigned char* smem) {
  const Csr A = J->A;
  const ColScale cs = J->cs;
  spmv_dots_body<TV, KW, false, true>(A, J->W, J->ld, c, c - KW, KW, cs, J->H, J->ldh, J->coef, J->part,
                                      J->counter, J->st, bid, nblk, smem);
}

// The SpMV + window-dot body for the window width of the phase (kw <= KMAX).
template <typename TV, int KW, int KMAX>
__device__ __forceinline__ void spmv_phase(int kw, const BasisJob<TV>* J, int c, int bid, int nblk,
                                           unsigned char* smem) {
  if constexpr (KW <= KMAX) {
    if (kw == KW) {
      spmv_phase_kw<TV, KW>(J, c, bid, nblk, smem);
      return;
    }
    spmv_phase<TV, KW + 1, KMAX>(kw, J, c, bid, nblk, smem);
  }
}

template <typename TV>
__device__ __noinline__ void init_phase(const BasisJob<TV>* J, int bid, int nblk) {
  init_body<TV>(J, bid, nblk);
}

// Theta V of every column of a solve from its kept partials (a warp per entry; the
// columns the basis reached: all below m_used, and m_used itself unless it broke down).
template <typename TV>
__device__ __noinline__ void reduce_phase(const BasisJob<TV>* J, int nparts, int bid, int nblk) {
  const SketchDev& sk = J->sk;
  const int lane = threadIdx.x & 31;
  const DevState* st = J->st;
  const int mu = st->m_used;
  const long long nw = (long long)nblk * (blockDim.x >> 5), entries = (long long)(J->m + 1) * sk.s;
  for (long long wid = ((long long)bid * blockDim.x + threadIdx.x) >> 5; wid < entries; wid += nw) {
    const int col = (int)(wid / sk.s), q = (int)(wid % sk.s);
    if (!(col < mu || (col == mu && !st->stop))) continue;  // warp-uniform
    const double* part = sk.part + (size_t)col * J->sk_colstride;
    double a = 0.0;
    for (int b = lane; b < nparts; b += 32) a += part[(size_t)b * sk.s + q];
    a = warp_sum(a);
    if (lane == 0) J->SV[(size_t)col * sk.s + q] = a * J->sk_scale * J->cs.sigma[col];
  }
}

template <int SK, typename TV>
__device__ __noinline__ void update_phase(const BasisJob<TV>* J, int c, int nc, int mode, int bid, int nblk,
                                          unsigned char* smem) {
  const ColScale cs = J->cs;
  SketchDev sk = J->sk;
  sk.part += (size_t)c * J->sk_colstride;  // this column's partials are kept
  update_body<SK, TV>(J->A.n, J->W, J->ld, c, c - nc, nc, J->coef, J->H, J->ldh, cs, mode, J->part, J->counter, sk,
                      J->st, bid, nblk, smem);
}

// The whole basis build of a batch in one persistent launch. The plan lists phases in
// order (the start of every solve; then for every step the SpMV + window dots and the
// window update + norm + fused sketch, Alg. 2 with the sketch of §2.1.1; then per
// solve one reduce of its kept sketch partials); a work item is one block of one solve
// in one phase, items are numbered in plan order, and each has a 16-byte record
// (BatchPlan). Each block of this kernel claims
// the next item number from a global ticket, waits (bounded) until its solve has
// completed the phase before (a per-solve counter, released by the block that ends
// that phase and acquired here), runs the phase's body with the solve's own (bid,
// nblk), and counts itself done. An item waits only on items with smaller numbers,
// which were all claimed before it by running blocks, so the launch completes
// whether or not all its blocks are resident at once. Every solve computes exactly
// what its own launches compute. Columns written by other blocks of this launch are
// read through L1 after the acquire (ld_col<true>), not through the read-only path.
template <typename TV, int KMAX>
__global__ __launch_bounds__(kThreads, 4) void k_batch_basis(const BasisJob<TV>* __restrict__ jobs, BatchPlan P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_item[5];  // item code (-1: no items left), solve, bid | nblk, seq | c, ok
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const unsigned t = atomicAdd(P.ticket, 1u);
      if (t >= P.total) {
        s_item[0] = -1;
      } else {
        const int4 r = __ldg(P.items + t);  // one load: the acquire below empties L1 every item
        const int j = r.x;
        const unsigned seq = (unsigned)r.z & 0xffffu;
        int polls = 0;
        while (ld_acquire_u32(P.done + j) < seq && ++polls < P.poll_limit) __nanosleep(64);
        const bool ok = ld_acquire_u32(P.done + j) >= seq;
        if (!ok) {  // the phase before never completed: this solve stops, the launch goes on
          jobs[j].st->status = FAB_ETIMEOUT;
          jobs[j].st->stop = 1;
        }
        s_item[0] = r.w;
        s_item[1] = j;
        s_item[2] = r.y;
        s_item[3] = r.z;
        s_item[4] = ok ? 1 : 0;
      }
    }
    __syncthreads();
    const int code = s_item[0];
    if (code < 0) break;
    const int j = s_item[1], bid = s_item[2] & 0xffff, nblk = (int)((unsigned)s_item[2] >> 16);
    const int seq = s_item[3] & 0xffff, c = (int)((unsigned)s_item[3] >> 16);
    const bool ok = s_item[4] != 0;
    const int type = code & 3, mode = (code >> 2) & 3, kind = ((code >> 4) & 7) - 1, arg = code >> 8;
    const BasisJob<TV>* J = jobs + j;
    if (ok) {
      if (type == kPhInit) {
        init_phase<TV>(J, bid, nblk);
      } else if (type == kPhSpmv) {
        spmv_phase<TV, 0, KMAX>(arg, J, c, bid, nblk, smem_raw);
      } else if (type == kPhUpdate) {
        switch (kind) {
          case SK_SRHT: update_phase<SK_SRHT, TV>(J, c, arg, mode, bid, nblk, smem_raw); break;
          case SK_SPARSE_TAB: update_phase<SK_SPARSE_TAB, TV>(J, c, arg, mode, bid, nblk, smem_raw); break;
          default: update_phase<SK_NONE, TV>(J, c, arg, mode, bid, nblk, smem_raw); break;
        }
      } else {
        reduce_phase<TV>(J, arg, bid, nblk);
      }
    }
    __syncthreads();  // the body's writes precede the count; s_item may be refilled
    if (tid == 0) {
      __threadfence();
      if (atomicAdd(P.blk + j, 1u) + 1u == (unsigned)nblk) {  // the last block of this phase
        atomicExch(P.blk + j, 0u);
        __threadfence();
        st_release_u32(P.done + j, (unsigned)seq + 1u);
      }
    }
  }
}

template <typename TV>
const void* batch_basis_fn(int kmax) {
  if (kmax <= 2) return (const void*)k_batch_basis<TV, 2>;
  if (kmax <= 4) return (const void*)k_batch_basis<TV, 4>;
  return (const void*)k_batch_basis<TV, 8>;
}

// Blocks of the persistent kernel (every resident slot once) after its
// shared-memory limit is set; call before a graph capture.
template <typename TV>
cudaError_t batch_basis_prepare(int kmax, size_t smem, int* grid) {
  const void* fn = batch_basis_fn<TV>(kmax);
  cudaError_t e = ensure_smem_limit(fn, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  *grid = sm_count() * (occ < 1 ? 1 : occ);
  return cudaSuccess;
}

template <typename TV>
cudaError_t launch_batch_basis(const BasisJob<TV>* jobs, const BatchPlan& plan, int kmax, int grid, size_t smem,
                               cudaStream_t s) {
  if (plan.total == 0) return cudaSuccess;
  const BasisJob<TV>* jb = jobs;
  BatchPlan p = plan;
  void* args[] = {(void*)&jb, &p};
  return cudaLaunchKernel(batch_basis_fn<TV>(kmax), dim3(grid), dim3(kThreads), args, smem, s);
}

// x = sum_{q < m_used} coef_q W_q, the arithmetic of k_combine with keep = 0
template <typename TV>
__global__ __launch_bounds__(kThreads) void k_combine_wave(const BasisJob<TV>* __restrict__ jobs, Wave w) {
  extern __shared__ double s_cf[];
  const int i = wave_slot(w, blockIdx.x);
  const BasisJob<TV>* J = jobs + w.ids[i];
  const int bid = blockIdx.x - w.pre[i], nblk = w.pre[i + 1] - w.pre[i];
  if (J->st->status != FAB_OK) return;
  const int nc = J->st->m_used, n = J->A.n;
  const TV* W = J->W;
  const int64_t ld = J->ld;
  combine_coef_load<TV>(s_cf, J->coef, nc);
  __syncthreads();
  double* out = J->x;
  for (int r = bid * kThreads + threadIdx.x; r < n; r += nblk * kThreads) out[r] = combine_row<TV>(W, ld, nc, s_cf, r);
}

template <typename TV>
cudaError_t launch_combine_wave(const BasisJob<TV>* jobs, const Wave& w, int nblocks, int mmax, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  const size_t smem = (size_t)(mmax + 1) * sizeof(double);
  cudaError_t e = ensure_smem_limit((const void*)k_combine_wave<TV>, smem);
  if (e != cudaSuccess) return e;
  k_combine_wave<TV><<<nblocks, kThreads, smem, s>>>(jobs, w);
  return cudaGetLastError();
}

#define FAB_BATCH(TV)                                                                                           \
  template cudaError_t batch_basis_prepare<TV>(int, size_t, int*);                                              \
  template cudaError_t launch_batch_basis<TV>(const BasisJob<TV>*, const BatchPlan&, int, int, size_t,          \
                                              cudaStream_t);                                                    \
  template cudaError_t launch_combine_wave<TV>(const BasisJob<TV>*, const Wave&, int, int, cudaStream_t);
FAB_BATCH(double)
FAB_BATCH(float)
#undef FAB_BATCH

// ------------------------------------------------------------- grid sizes
static int g_sms = 0;
int sm_count() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

// The dynamic shared-memory limit is a process-wide attribute of a kernel, and
// several host threads (the serving slots) launch the same kernels with different
// sizes. Setting it to each launch's own size would let one thread lower it between
// another thread's set and launch, so it only ever grows, under a lock.
cudaError_t ensure_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = limit.find({dev, fn});
  if (it == limit.end()) {  // start from the kernel's own limit (48 KB less its static shared memory)
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    it = limit.emplace(std::make_pair(dev, fn), (size_t)fa.maxDynamicSharedSizeBytes).first;
  }
  size_t& cur = it->second;
  if (bytes <= cur) return cudaSuccess;  // never lower the limit below a size launched before
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int combine_grid(int n) { return grid_rows(n); }

int grid_rows(int n) {
  const int need = (n + kThreads - 1) / kThreads;
  const int cap = sm_count() * 8;
  return need < 1 ? 1 : (need < cap ? need : cap);
}


}  // namespace fab
