// Internal declarations shared by the libfab translation units (device helpers,
// device-side solve state, kernel launchers). Not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/fab.h"

namespace fab {

constexpr int kThreads = 256;        // threads per block of the streaming kernels
constexpr int kChunkLog2 = 12;       // rows per sketch chunk: 4096 (one int64 transform block)
constexpr int kChunk = 1 << kChunkLog2;
constexpr int kRowsPerThread = kChunk / kThreads;  // 16
constexpr int kMaxWindow = 8;        // k of Alg. 2
constexpr int kMaxM = 1024;          // Krylov dimension limit
constexpr int kMaxS = 4096;          // sketch rows limit
constexpr int kMaxZeta = 16;         // sparse-sign nonzeros per column limit
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

enum SketchKind { SK_NONE = -1, SK_SPARSE = 0, SK_SRHT = 1, SK_GAUSS = 2, SK_SPARSE_TAB = 3 };
// SK_SPARSE_TAB: the sparse sign sketch read from its precomputed pattern table
// (SketchDev::pat) instead of drawing each column's rows again.

// Device-side state of one solve. Written only by kernels (reset by k_state_reset).
struct DevState {
  int m_used;    // basis dimension (m until a breakdown)
  int stop;      // set once the basis loop must not continue (breakdown or error)
  int status;    // FAB_OK or the device-detected error
  int flag;      // iteration-loop flag (LSQR / square-root iteration converged)
  int iters;     // iteration count reported by the loops
  int wh;        // basis columns when it was whitened (FAB_WHITEN), 0: not whitened
  double beta;   // ||b||_2
  double scal[16];  // scalars of the small-stage loops (LSQR recurrence, DB scaling)
  double kappa;  // max |r_ii| / min |r_ii| of the sketch QR (0: no sketch QR in this solve)
};

// Sketch description passed by value to the basis kernels.
struct SketchDev {
  int kind;            // SketchKind
  int s;               // rows of Theta
  int zeta;            // sparse sign: nonzeros per column
  int chunk_log2;      // log2 of the rows per transform chunk (<= kChunkLog2)
  int nchunks;         // ceil(n / chunk)
  int nparts;          // block partials written by the last k_update (its grid)
  uint64_t st_rows;    // SplitMix64 stream states (see fab_rng_state)
  uint64_t st_signs;
  uint64_t st_D;
  const int* P;        // SRHT sampled rows (device, s entries, sorted)
  __nv_bfloat16* Wbf;  // Gaussian: two-term BF16 copy of the basis, hi = bf16(v), lo = bf16(v - hi),
                       // K-blocked (see gauss.cuh: entry ((r/64) 2 cpad + t cpad + c) 64 + r%64)
  int bf_cpad;
  double* part;        // nparts x s block partials (block-major), nparts <= nchunks
  // sparse sign: the pattern transposed per 4096-row chunk (see sparse_rec_bytes): for
  // chunk c at pat + c * sparse_rec_bytes(s, zeta) bytes, uint32 offsets off[0..s] and
  // uint16 entries (bits 0..11 the row in the chunk, bit 15 the sign) with the rows
  // that hit sketch row q at [off[q], off[q+1]); NULL to draw the rows on the fly
  const unsigned short* pat;
};
// Bytes of one chunk's record in the transposed sparse-sign table: the s+1 offsets, then
// zeta entries per row of the chunk, each part padded to 16 bytes.
__host__ __device__ __forceinline__ size_t sparse_off_bytes(int s) { return ((size_t)(s + 1) * 4 + 15) / 16 * 16; }
__host__ __device__ __forceinline__ size_t sparse_rec_bytes(int s, int zeta) {
  return sparse_off_bytes(s) + ((size_t)zeta * 4096 * 2 + 15) / 16 * 16;
}
__host__ __device__ __forceinline__ size_t sparse_table_bytes(int64_t n, int s, int zeta) {
  return (size_t)((n + 4095) / 4096) * sparse_rec_bytes(s, zeta);
}

// ----------------------------------------------------------------- SplitMix64
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Initial state of stream `stream` for `seed`: mix64(seed + stream * gamma).
__host__ __device__ __forceinline__ uint64_t rng_state(uint64_t seed, uint64_t stream) {
  return mix64(seed + stream * kGamma);
}
// idx-th output (0-based) of the generator whose state starts at `state`.
__host__ __device__ __forceinline__ uint64_t rng_u(uint64_t state, uint64_t idx) {
  return mix64(state + (idx + 1) * kGamma);
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV values per thread; result valid in thread 0 (out[0..NV)).
// Fixed combination order (deterministic for a given launch shape).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* >= 32*NV */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[warp * NV + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += sh[w * NV + q];
      v[q] = a;
    }
  }
  __syncthreads();
}

// Warp totals of V values per lane by recursive halving: in each of the first
// log2(P) rounds (P = the power of two >= V, missing values zero) a lane keeps one
// half of its values and adds its partner's copy of that half, then the last
// 5 - log2(P) rounds add single values. P - 1 + 5 - log2(P) additions per lane in
// place of 5 V. Value q's total is returned in lanes [q 32/P, (q+1) 32/P).
// Fixed combination order.
template <int V>
__device__ __forceinline__ double warp_sum_multi(const double (&v)[V]) {
  constexpr int P = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : V <= 16 ? 16 : 32;
  static_assert(V >= 1 && V <= 32, "1..32 values");
  const int lane = threadIdx.x & 31;
  double x[P];
#pragma unroll
  for (int q = 0; q < P; ++q) x[q] = q < V ? v[q] : 0.0;
  int o = 16;
#pragma unroll
  for (int h = P / 2; h >= 1; h /= 2) {
    const bool up = (lane & o) != 0;  // this lane keeps the upper half
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const double keep = up ? x[q + h] : x[q];
      const double send = up ? x[q] : x[q + h];
      x[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    o >>= 1;
  }
  for (; o > 0; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
  return x[0];
}

// Block totals of V values per thread into out[0..V) (shared; valid after the call
// in every thread): warp_sum_multi, then thread q adds the warps' totals of value q
// in warp order.
template <int V>
__device__ __forceinline__ void block_sum_multi(const double (&v)[V], double* sh /* >= 32 V */, double* out) {
  constexpr int P = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : V <= 16 ? 16 : 32;
  constexpr int G = 32 / P;  // lanes that hold each total
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double t = warp_sum_multi<V>(v);
  if (lane % G == 0 && lane / G < V) sh[warp * V + lane / G] = t;
  __syncthreads();
  if (threadIdx.x < V) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += sh[w * V + threadIdx.x];
    out[threadIdx.x] = a;
  }
  __syncthreads();
}

// Totals of the V columns of a row-major nblocks x V partial array, by one block in
// one pass (every column's loads in flight together), into out[0..V) (shared).
template <int V>
__device__ __forceinline__ void sum_partials_multi(const double* part, int nblocks, double* out,
                                                   double* sh /* >= 32 V */) {
  double a[V];
#pragma unroll
  for (int q = 0; q < V; ++q) a[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < V; ++q) a[q] += __ldcg(part + (size_t)b * V + q);
  }
  block_sum_multi<V>(a, sh, out);
}

// Last-block-done: returns true in every thread of the block that finished last.
// Partials written before the call are visible to that block afterwards.
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblk) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}
__device__ __forceinline__ bool last_block(unsigned* counter) { return last_block(counter, gridDim.x); }

// Sum of `nv` columns of a row-major nblocks x nv partial array, by one block,
// in a fixed order. out[q] (shared) receives column q. nv <= 32.
__device__ __forceinline__ void sum_partials(const double* part, int nblocks, int nv, double* out,
                                             double* sh /* blockDim.x doubles */) {
  for (int q = 0; q < nv; ++q) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += __ldcg(part + (size_t)b * nv + q);
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
      out[q] = t;
    }
    __syncthreads();
  }
}

// y * 2^k, exact: integer addition to the exponent field for normal results;
// zeros, subnormals and out-of-range exponents take the FP64 multiply.
static __device__ __noinline__ double scale_pow2_slow(double y, double p2k) { return y * p2k; }
__device__ __forceinline__ double scale_pow2(double y, int k, double p2k) {
  const long long b = __double_as_longlong(y);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e != 0 && e + k > 0 && e + k < 2047) return __longlong_as_double(b + ((long long)k << 52));
  return scale_pow2_slow(y, p2k);  // out of line: keeps the common path free of FP64 work
}
// Unbiased exponent of a positive normal double (floor(log2 x)).
__host__ __device__ __forceinline__ int exponent_of(double x) {
#ifdef __CUDA_ARCH__
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
#else
  long long b;
  memcpy(&b, &x, 8);
  return (int)((b >> 52) & 0x7FF) - 1023;
#endif
}

// 2^e as a double for e in [-1074, 1023], without FP64 arithmetic on the value.
__device__ __forceinline__ double pow2_split(int e, double* second) {
  // returns a and sets *second = b with a*b = 2^e and both normal doubles
  int e1 = e / 2, e2 = e - e1;
  *second = __longlong_as_double((long long)(e2 + 1023) << 52);
  return __longlong_as_double((long long)(e1 + 1023) << 52);
}

// ------------------------------------------------ TMA bulk copy + mbarrier
// One-dimensional bulk copies global -> shared (cp.async.bulk) completing on an
// mbarrier with a transaction count. Source and destination must be 16-byte
// aligned and the size a multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Float-float accumulation for combinations of FP32 basis columns with FP64
// coefficients, on the FP32 pipe: c = hi + lo (two floats), the product hi*w is
// split exactly by an FMA (TwoProd) and added by Knuth's TwoSum, the small parts
// go to lo. The result, hi + lo in FP64, is within about 2^-48 of the sum of
// |terms| (2^24 times below the FP32 basis rounding). The _rn intrinsics are
// never contracted into FMAs, which TwoSum needs.
__device__ __forceinline__ float2 ff_split(double c) {
  const float hi = __double2float_rn(c);
  return make_float2(hi, __double2float_rn(c - (double)hi));
}
__device__ __forceinline__ void ff_madd(float& s_hi, float& s_lo, float2 c, float w) {
  const float p = __fmul_rn(c.x, w);
  const float pe = __fmaf_rn(c.x, w, -p);  // c.x w = p + pe exactly
  const float t = __fadd_rn(s_hi, p);
  const float bp = __fsub_rn(t, s_hi);
  const float e = __fadd_rn(__fsub_rn(s_hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));  // s_hi + p = t + e exactly
  s_hi = t;
  s_lo = __fadd_rn(s_lo, __fadd_rn(e, __fmaf_rn(c.y, w, pe)));
}
// sum_q coef[q] W_q[r] for one row; FP64 columns: FP64 FMAs; FP32 columns: float-float
// with the coefficients pre-split (s_cf holds nc doubles, or nc float2 for FP32).
template <typename TV>
__device__ __forceinline__ double combine_row(const TV* __restrict__ W, int64_t ld, int nc, const void* s_cf, int r) {
  if constexpr (sizeof(TV) == 4) {
    const float2* c = reinterpret_cast<const float2*>(s_cf);
    float hi = 0.0f, lo = 0.0f;
#pragma unroll 8
    for (int q = 0; q < nc; ++q) ff_madd(hi, lo, c[q], (float)W[(size_t)q * ld + r]);
    return (double)hi + (double)lo;
  } else {
    const double* c = reinterpret_cast<const double*>(s_cf);
    double a = 0.0;
#pragma unroll 4
    for (int q = 0; q < nc; ++q) a = fma(c[q], (double)W[(size_t)q * ld + r], a);
    return a;
  }
}
// Fills the shared coefficient table combine_row reads (8 bytes per coefficient).
template <typename TV>
__device__ __forceinline__ void combine_coef_load(void* s_cf, const double* coef, int nc) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    if constexpr (sizeof(TV) == 4)
      reinterpret_cast<float2*>(s_cf)[i] = ff_split(coef[i]);
    else
      reinterpret_cast<double*>(s_cf)[i] = coef[i];
  }
}

// Bulk prefetch of [src, src + bytes) from global memory into L2 (no destination,
// no completion to wait for): src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// The same, skipped unless src and bytes are 16-byte multiples: the library's own
// bases always are (ld a multiple of 32, 256-byte aligned), but a caller's matrix
// (fab_sketch_apply) may have any leading dimension.
__device__ __forceinline__ void bulk_prefetch_l2_aligned(const void* src, uint32_t bytes) {
  if (((uint32_t)reinterpret_cast<uintptr_t>(src) | bytes) & 15u) return;
  if (bytes > 0) bulk_prefetch_l2(src, bytes);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of `bar`: false if the limit expired.
constexpr int kWaitLimit = 1 << 20;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Phase gate of a basis-step kernel of FAB_WHITEN (the launch argument `gate`):
// 0 runs always, 1 only while column c is built by Alg. 2 (not yet whitened),
// 2 only once it is built by Alg. 1 (the basis was whitened with wh <= c
// columns). Every block of a gated-off launch returns before touching memory.
__device__ __forceinline__ bool gate_closed(const DevState* st, int c, int gate) {
  if (gate == 0) return false;
  const int wh = *(volatile const int*)&st->wh;
  const bool bg = wh > 0 && c >= wh;
  return gate == 1 ? bg : !bg;
}

// ----------------------------------------------------------------- launchers
// (defined in basis.cu / small.cu; all take the stream last and return cudaError_t)
struct Csr {
  int n;
  int nnz;
  const int* rowptr;
  const int* colind;
  const void* vals;   // FP64 values (FP64 path) or FP32 values (mixed path)
  const int* tiles;   // SpMV row tiles: tile t is rows tiles[t] .. tiles[t+1]-1 (<= 256 rows)
  int ntiles;
  int staged;         // 1: stage a tile's nonzeros in shared memory by bulk copies when they fit;
                      // 2: the same, and process tiles of many rows by nonzeros
};
constexpr int kSpmvCap = 2048;   // nonzeros per staged SpMV tile (FP64: vals 16 KB + colind 8 KB)
constexpr int kSpmvStages = 2;   // staged tiles in flight per block (ring of shared-memory buffers)

cudaError_t launch_state_reset(DevState* st, int m, cudaStream_t s);
cudaError_t launch_state_set_m(DevState* st, int m, cudaStream_t s);  // basis target dimension
cudaError_t launch_state_clear_flag(DevState* st, cudaStream_t s);   // before an iteration loop
// Column bookkeeping of the raw basis (see basis.cu): sigma[j] = 1/||W_j||,
// shf[j] = floor(log2 sigma[j]) (the exact power of two applied when W_j is the
// SpMV input), scl[c] = sigma[c-1] 2^-shf[c-1] in [1, 2) (A v_{c-1} = scl[c] W_c).
struct ColScale {
  double* sigma;
  int* shf;
  double* scl;
};
template <typename TV>
cudaError_t launch_spmv_dots(const Csr& A, TV* W, int64_t ld, int c, int j0, int kw, ColScale cs,
                             double* H, int ldh, double* coef, double* part, unsigned* counter,
                             DevState* st, cudaStream_t s, int gate = 0);
template <typename TV>
cudaError_t launch_update(int n, TV* W, int64_t ld, int c, int j0, int nc, const double* coef, double* H,
                          int ldh, ColScale cs, int mode, double* part, unsigned* counter,
                          SketchDev& sk, DevState* st, cudaStream_t s, int gate = 0);
// The Alg. 2 window update and norm of column c without a sketch (see k_update_plain).
template <typename TV>
cudaError_t launch_update_plain(int n, TV* W, int64_t ld, int c, int j0, int kw, const double* coef, double* H,
                                int ldh, ColScale cs, int mode, double* part, unsigned* counter,
                                DevState* st, cudaStream_t s);
cudaError_t launch_sketch_reduce(const SketchDev& sk, const double* sigma, int col, double scale, double* out,
                                 DevState* st, cudaStream_t s, int gate = 0);
// The same reduce for ncols columns at once (column c's nparts partials at sk.part +
// c * colstride; Theta v_c to SV + c * s), for a pass whose sketch nothing reads
// before the pass ends.
cudaError_t launch_sketch_reduce_cols(const SketchDev& sk, size_t colstride, int c0, int ncols, int nparts,
                                      const double* sigma, double scale, double* SV, const DevState* st,
                                      cudaStream_t s);
// One-pass basis step of the FP32 path (fused.cu): the update, norm and sketch of column
// c-1 (when upd; window j0u .. j0u+kwu-1, its coefficients in coef) and the SpMV of step c
// with its window dots (j0 .. c-1); w_{c-1} is read from wprev, w_c written to wnext; the
// last block writes H's columns c-2 (norm) and c-1, sigma_{c-1}, scl[c], shf[c] and step
// c's coefficients into coef. Every row of A has at most 8 nonzeros. sk.kind SK_SRHT,
// SK_SPARSE (with its table) or SK_NONE; sk.nparts receives the grid.
// plan: per-chunk flags (zeroed at the start of a solve), the task claim order and the
// chunk ranges the rows of each chunk reference (fused_plan); counter[1] is the task counter.
struct FusePlan {
  int* flags;
  const int* tasks;
  const int* crange;  // int2 per chunk
  const int* ell_col;  // A in ELL form (FP32): slot u of row r at u ell_ld + r
  const float* ell_val;
  int64_t ell_ld;
  int ell_k;           // slots (the longest row, <= 8)
  int stall_pass;      // > 0: in that pass the SpMV tasks wait for a flag no task sets
  int stall_polls;     //      (fab_inject_wait_timeout), giving up after stall_polls polls
};
// The ELL copy of the FP32 CSR matrix for the one-pass steps (k slots, ld >= n).
cudaError_t launch_build_ell(int n, const int* rowptr, const int* colind, const float* vals, int k, int64_t ld,
                             int* ecol, float* eval, cudaStream_t s);
cudaError_t launch_fused_step(const Csr& A, float* W, int64_t ld, int c, int upd, int j0u, int kwu, int j0, int kw,
                              const float* wprev, float* wnext, ColScale cs, double* H, int ldh, double* coef,
                              double* part, unsigned* counter, SketchDev& sk, DevState* st, const FusePlan& plan,
                              cudaStream_t s);
// Blocks of the one-pass step for a matrix of n rows and sketch kind / rows (and its
// dynamic shared memory).
int fused_grid(int kind, int n, int s, size_t* smem);
// The sparse sign pattern of sk, transposed per chunk, into pat (sparse_table_bytes(n, s, zeta) bytes).
cudaError_t launch_sparse_pattern(int n, const SketchDev& sk, unsigned short* pat, cudaStream_t s);

// ------------------------------------------------------------ batched waves
// One solve of a batch as the basis kernels see it (a device-resident table).
template <typename TV>
struct BasisJob {
  Csr A;
  TV* W;  // raw basis, n x (m+1), ld
  int64_t ld;
  ColScale cs;
  double* H;  // (m+1) x m
  int ldh;
  int m, k;
  double *coef, *part;
  unsigned* counter;
  DevState* st;
  SketchDev sk;  // sk.kind SK_NONE for Alg. 5 without a sketch
  size_t sk_colstride;  // sketch partials of column c at sk.part + c * sk_colstride
  double sk_scale;
  double* SV;       // s x (m+1)
  const double* b;  // start vector (FP64, device)
  double* x;        // result (FP64, device)
};
// A wave lists solves and their blocks: job ids[i] owns blocks pre[i] ..
// pre[i+1]-1 (its own launch's grid); aux[i] is a per-job extra (the sketch
// partial count of the update phase before a reduce phase).
struct Wave {
  const int* pre;
  const int* ids;
  const int* aux;
  int count;
};
// Phases of a batch's basis build, run in plan order by one persistent launch.
enum PhaseType { kPhInit = 0, kPhSpmv = 1, kPhUpdate = 2, kPhReduce = 3 };
// One work item of the persistent batch launch, decoded on the host:
//   x = solve, y = bid | nblk << 16, z = phase number of the solve | c << 16,
//   w = type | update mode << 2 | (sketch kind + 1) << 4 | arg << 8
// (arg: SpMV window width, update column count, or the reduce's partials per column).
struct BatchPlan {
  const int4* items;
  unsigned total;   // work items
  unsigned* ticket; // next item to claim
  unsigned* done;   // per solve: phases completed
  unsigned* blk;    // per solve: blocks done in the current phase
  int poll_limit;   // polls of a solve's counter before its solve gives up (FAB_ETIMEOUT)
};
// Grid of the single-solve launch of each basis kernel (a batched solve uses the same).
template <typename TV>
int spmv_grid(int ntiles, int kw, bool seg);
template <typename TV>
int update_grid(int kind, int n, int nc, int s, size_t* smem);
int combine_grid(int n);
// The persistent basis kernel of a batch (window widths up to kmax): its grid, once its
// shared-memory limit (smem bytes) is set, then its launch.
template <typename TV>
cudaError_t batch_basis_prepare(int kmax, size_t smem, int* grid);
template <typename TV>
cudaError_t launch_batch_basis(const BasisJob<TV>* jobs, const BatchPlan& plan, int kmax, int grid, size_t smem,
                               cudaStream_t s);
template <typename TV>
cudaError_t launch_combine_wave(const BasisJob<TV>* jobs, const Wave& w, int nblocks, int mmax, cudaStream_t s);
cudaError_t launch_srht_sample(int64_t npad, int s, uint64_t stP, int* P, cudaStream_t st);
template <typename TV, typename TX>
cudaError_t launch_gemv_t(int n, const TV* W, int64_t ld, int j0, int nc, const TX* x, double* part,
                          int ntiles, DevState* st, cudaStream_t s);
cudaError_t launch_reduce_cols(const double* part, int ntiles, int nc, const double* sigma, int j0,
                               const double* sig_col, double* Hcol, int h_accumulate, double* coef, DevState* st,
                               cudaStream_t s);
template <typename TV>
cudaError_t launch_combine(int n, const TV* W, int64_t ld, int nc, const double* coef, double* out,
                           double keep, cudaStream_t s);
template <typename TV>
cudaError_t launch_scale_columns(int n, const TV* W, int64_t ld, int nc, const double* sigma, double* dst,
                                 int64_t ldd, cudaStream_t s);
// Whitening of FAB_WHITEN: when the basis was whitened at this step (st->wh == c+1),
// column c becomes sum_{q<=c} coef[q] W_q (the explicit whitened vector, unit
// scale), in place; otherwise every block returns at once.
template <typename TV>
cudaError_t launch_whiten_column(int n, TV* W, int64_t ld, int c, const double* coef, DevState* st,
                                 cudaStream_t s);
cudaError_t launch_to_f32(int n, const double* x, float* y, cudaStream_t s);
cudaError_t launch_csr_spmv(int n, const int* rowptr, const int* colind, const double* vals, const double* x,
                            double* y, cudaStream_t s);

// FMA throughput probe (T = double or float; operand pattern 0..2): blocks_per_sm x
// sm_count() blocks of kThreads threads, each thread 128 iters FMAs; *fmas receives the total.
template <typename T>
cudaError_t launch_fma_peak(int pattern, int blocks_per_sm, int iters, cudaStream_t s, double* fmas);
int sm_count();              // multiprocessors of the current device
int grid_rows(int n);        // grid for the thread-per-row kernels
// Raises (never lowers) kernel fn's dynamic shared-memory limit to at least `bytes`; thread-safe.
cudaError_t ensure_smem_limit(const void* fn, size_t bytes);
constexpr int kMaxPartBlocks = 64;  // partial buffers hold sm_count() * kMaxPartBlocks blocks
constexpr int kTileRows = 2048;     // rows per GEMV-T tile

}  // namespace fab
