// Device pieces shared by the basis-loop kernels (basis.cu, fused.cu): the element
// type's floating-point layout, exact power-of-two rescaling, the exact int64 chunk
// sketches (SRHT and sparse sign, paper §2.1.1) and the column bookkeeping after a
// window update (Alg. 2). Internal.
#pragma once

#include <float.h>

#include "fab_internal.cuh"

namespace fab {

// Floating-point layout of the basis element type (FP64 path / FP32 mixed path).
template <typename T>
struct Fp;
template <>
struct Fp<double> {
  static constexpr int kMant = 52, kExpMax = 0x7FF;
  static constexpr int kFixOff = 1071;  // chunk fixed point: x = X * 2^(E - kFixOff)
  __device__ static unsigned long long bits(double x) { return (unsigned long long)__double_as_longlong(x); }
};
template <>
struct Fp<float> {
  static constexpr int kMant = 23, kExpMax = 0xFF;
  static constexpr int kFixOff = 175;
  __device__ static unsigned long long bits(float x) { return (unsigned long long)(unsigned)__float_as_uint(x); }
};

__device__ __forceinline__ float scale_pow2(float y, int k, float p2k) {
  const unsigned b = __float_as_uint(y);
  const int e = (int)((b >> 23) & 0xFF);
  if (e != 0 && e + k > 0 && e + k < 255) return __uint_as_float(b + ((unsigned)k << 23));
  return y * p2k;
}

// tau = sigma_{c-1} 2^-shf[c-1], exactly (power-of-two factors).
__device__ __forceinline__ double column_tau(double sigma_prev, int ksh) {
  double pinv;
  const double pinv_hi = pow2_split(-ksh, &pinv);
  return (sigma_prev * pinv_hi) * pinv;
}

// ---------------------------------------------- exact int64 chunk sketches
// A chunk of 4096 consecutive rows is converted to a common block exponent:
// x = X * 2^(E - 1071) with X an int64 of at most 49 significant bits, E the
// largest biased exponent in the chunk. Sums of up to 4096 such integers are
// exact in int64 (|sum| < 2^61), so the chunk's sketch is exact apart from
// the rounding of x to X (relative 2^-49 of the chunk maximum) and of the
// final int64 -> FP64 conversion, and it does not depend on summation order.

template <typename T>
__device__ __forceinline__ int exp_field(T x) {
  return (int)((Fp<T>::bits(x) >> Fp<T>::kMant) & Fp<T>::kExpMax);
}

// x (FP64 or FP32) as X with x = X 2^(E - kFixOff), |X| < 2^49, rounded to nearest.
template <typename T>
__device__ __forceinline__ long long to_fixed(T x, int E) {
  constexpr int P = Fp<T>::kMant;  // stored mantissa bits
  const unsigned long long bits = Fp<T>::bits(x);
  const int ef = (int)((bits >> P) & Fp<T>::kExpMax);
  const unsigned long long M = ef ? ((bits & ((1ull << P) - 1)) | (1ull << P)) : (bits & ((1ull << P) - 1));
  const int eff = ef ? ef : 1;
  // X = M 2^(eff - E - (P - 48)): a left shift for FP32 (exact), a right shift for FP64
  const int L = eff - E + 48 - P;
  long long X;
  if (L >= 0) {
    X = (long long)(M << L);
  } else {
    int sh = -L;
    if (sh > 63) sh = 63;
    X = (long long)((M + (1ull << (sh - 1))) >> sh);
  }
  return ((bits >> (sizeof(T) * 8 - 1)) & 1ull) ? -X : X;
}

__device__ __forceinline__ int pidx(int j) { return j + (j >> 4); }  // bank-conflict padding


// In-register Walsh-Hadamard butterflies over the 4 index bits held by a thread.
__device__ __forceinline__ void wht16(long long (&X)[16]) {
#pragma unroll
  for (int h = 1; h < 16; h <<= 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if ((i & h) == 0) {
        const long long a = X[i], b = X[i + h];
        X[i] = a + b;
        X[i + h] = a - b;
      }
    }
  }
}

// Block maximum of an int (all threads receive it). reuse_barrier = false leaves out
// the barrier that protects sh from the next call: for callers that pass a block
// barrier of their own before calling again.
__device__ __forceinline__ int block_max_int(int v, int* sh, bool reuse_barrier = true) {
  v = (int)__reduce_max_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  int m = 0;
  for (int w = 0; w < kThreads / 32; ++w) m = max(m, sh[w]);
  if (reuse_barrier) __syncthreads();
  return m;
}

// SRHT chunk: y = H_4096 (D x_chunk); writes y at the sampled in-chunk rows.
// Thread t holds rows i*256 + t (i = 0..15) of the chunk. nrm2 (optional): adds this
// thread's sum of x^2 over its rows, formed exactly in integers from the fixed-point X
// (|X| < 2^49, so 16 squares fit 128 bits) and rounded once, in place of FP64 FMAs.
// kLean: two block barriers fewer per chunk, for a caller that calls it chunk after
// chunk and reads s_acc[q] only from thread q mod 256: s_int is read before the
// barrier that precedes the first write of buf, and buf is not written again before the
// next chunk's first barrier, which every thread reaches only after its reads of buf.
template <typename TV, bool kLean = false>
__device__ void sketch_chunk_srht(const TV (&v)[kRowsPerThread], int chunk, const SketchDev& sk,
                                  long long* buf, const int* s_P, double* s_acc, int* s_int,
                                  double* nrm2 = nullptr) {
  const int t = threadIdx.x;
  int e = 0;
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) e = max(e, exp_field(v[i]));
  const int E = block_max_int(e, s_int, !kLean);
  long long X[16];
  // D's signs: row i*256 + t takes bit (t mod 64) of word chunk*64 + t/64 + 4i. The 32
  // threads of a warp share t/64, so the warp needs 16 words: lane l < 16 draws the word of
  // i = l and every thread reads word i from lane i (one draw per lane instead of 16).
  const unsigned long long word0 = (unsigned long long)chunk * (kChunk / 64) + (t >> 6);
  const unsigned long long mine = rng_u(sk.st_D, word0 + (unsigned long long)(t & 15) * (kThreads / 64));
  unsigned long long sq_lo = 0ull, sq_hi = 0ull;
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) {
    long long x = to_fixed(v[i], E);
    if (nrm2) {
      const unsigned long long ax = (unsigned long long)(x < 0 ? -x : x);
      const unsigned long long lo = ax * ax;
      sq_lo += lo;
      sq_hi += __umul64hi(ax, ax) + (sq_lo < lo ? 1ull : 0ull);
    }
    const unsigned long long dw = __shfl_sync(0xffffffffu, mine, i);
    if ((dw >> (t & 63)) & 1ull) x = -x;
    X[i] = x;
  }
  wht16(X);  // index bits 8..11
#pragma unroll
  for (int i = 0; i < 16; ++i) buf[pidx(i * kThreads + t)] = X[i];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) X[q] = buf[pidx(t * 16 + q)];
  wht16(X);  // index bits 0..3
#pragma unroll
  for (int q = 0; q < 16; ++q) buf[pidx(t * 16 + q)] = X[q];
  __syncthreads();
  const int base3 = (t >> 4) * 256 + (t & 15);
#pragma unroll
  for (int q = 0; q < 16; ++q) X[q] = buf[pidx(base3 + q * 16)];
  wht16(X);  // index bits 4..7
#pragma unroll
  for (int q = 0; q < 16; ++q) buf[pidx(base3 + q * 16)] = X[q];
  __syncthreads();
  double b;
  const double a = pow2_split(E - Fp<TV>::kFixOff, &b);
  if (nrm2) *nrm2 += (((((double)sq_hi * 0x1p64 + (double)sq_lo) * a) * b) * a) * b;  // sum X^2 (2^(E-off))^2
  // cross-chunk Hadamard factor (-1)^popcount(rh_q & chunk), rh_q = P_q >> 12
  for (int q = t; q < sk.s; q += kThreads) {
    const int p = s_P[q];
    const double yq = ((double)buf[pidx(p & (kChunk - 1))] * a) * b;
    s_acc[q] += (__popc((p >> kChunkLog2) & chunk) & 1) ? -yq : yq;
  }
  if (!kLean) __syncthreads();
}

// The zeta distinct sketch rows of column j (R9): candidates floor(h s / 2^32)
// from the 32-bit halves of stream-1 words, in order, repeats rejected; after
// 256 candidates the smallest unused rows fill up (never reached in practice).
__device__ __forceinline__ void sparse_rows(const SketchDev& sk, long long j, int (&rows)[kMaxZeta]) {
  const unsigned s = (unsigned)sk.s;
  int have = 0;
  unsigned long long h = 0;
  for (int cand = 0; cand < 256 && have < sk.zeta; ++cand) {
    if ((cand & 1) == 0) h = rng_u(sk.st_rows, (unsigned long long)j * 128ull + (unsigned long long)(cand >> 1));
    const unsigned half = (cand & 1) ? (unsigned)(h >> 32) : (unsigned)h;
    const int r = (int)(((unsigned long long)half * s) >> 32);
    bool dup = false;
#pragma unroll
    for (int q = 0; q < kMaxZeta; ++q) dup |= (q < have) && (rows[q] == r);
    if (!dup) {
#pragma unroll
      for (int q = 0; q < kMaxZeta; ++q)
        if (q == have) rows[q] = r;
      ++have;
    }
  }
  for (int r = 0; have < sk.zeta; ++r) {  // fallback: smallest unused rows
    bool dup = false;
#pragma unroll
    for (int q = 0; q < kMaxZeta; ++q) dup |= (q < have) && (rows[q] == r);
    if (!dup) {
#pragma unroll
      for (int q = 0; q < kMaxZeta; ++q)
        if (q == have) rows[q] = r;
      ++have;
    }
  }
}

// Sparse-sign chunk: every row j scatters +-X_j into its zeta sketch rows (exact
// int64 sums in shared memory); TAB gathers from the chunk lists of sk.pat instead.
template <typename TV, bool TAB>
__device__ void sketch_chunk_sparse(const TV (&v)[kRowsPerThread], int chunk, int n, const SketchDev& sk,
                                    unsigned long long* acc, double* s_acc, int* s_int) {
  const int t = threadIdx.x;
  int e = 0;
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) e = max(e, exp_field(v[i]));
  const int E = block_max_int(e, s_int);
  if (TAB) {
    // gather instead of scatter: the chunk's X in shared memory, then one warp per
    // sketch row sums the entries of that row's list (no atomics; exact int64 sums)
    long long* xb = reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(acc) + ((size_t)sk.s * 8 + 15) / 16 * 16);
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) {
      const long long j = (long long)chunk * kChunk + i * kThreads + t;
      xb[i * kThreads + t] = (j < n) ? to_fixed(v[i], E) : 0ll;
    }
    __syncthreads();
    const unsigned char* rec = reinterpret_cast<const unsigned char*>(sk.pat) + (size_t)chunk * sparse_rec_bytes(sk.s, sk.zeta);
    const unsigned* off = reinterpret_cast<const unsigned*>(rec);
    const unsigned short* ent = reinterpret_cast<const unsigned short*>(rec + sparse_off_bytes(sk.s));
    const int lane = t & 31;
    for (int q = t >> 5; q < sk.s; q += kThreads / 32) {
      const unsigned lo = __ldg(off + q), hi = __ldg(off + q + 1);
      long long sum = 0;
      for (unsigned e = lo + lane; e < hi; e += 32) {
        const unsigned w = __ldg(ent + e);
        const long long x = xb[w & 0x0FFFu];
        sum += (w >> 15) ? -x : x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) acc[q] += (unsigned long long)sum;
    }
  }
  for (int i = 0; i < kRowsPerThread && !TAB; ++i) {
    const long long j = (long long)chunk * kChunk + i * kThreads + t;
    if (j >= n) break;
    const long long X = to_fixed(v[i], E);
    if (X == 0) continue;
    {
      int rows[kMaxZeta];
      sparse_rows(sk, j, rows);
      const unsigned long long sg = rng_u(sk.st_signs, (unsigned long long)j);
#pragma unroll
      for (int q = 0; q < kMaxZeta; ++q) {
        if (q < sk.zeta) {
          const long long val = ((sg >> q) & 1ull) ? -X : X;
          atomicAdd(acc + rows[q], (unsigned long long)val);
        }
      }
    }
  }
  __syncthreads();
  double b;
  const double a = pow2_split(E - Fp<TV>::kFixOff, &b);
  for (int q = t; q < sk.s; q += kThreads) {
    s_acc[q] += ((double)(long long)acc[q] * a) * b;
    acc[q] = 0ull;
  }
  __syncthreads();
}

// ------------------------------------------ window update + norm + sketch
// W_c <- W_c - sum_q coef_q W_{j0+q}; optionally ||W_c||^2 is reduced over the
// grid (mode & kModeNorm) and the last block writes h_{c,c-1} and sigma_c, or
// ||b|| and sigma_0 for the start vector (mode & kModeInit); optionally the
// chunk sketch partials of the updated column are written.
constexpr int kModeNorm = 1;
constexpr int kModeInit = 2;

// ||w'||^2 over the grid (each block's share nrm, the last block to finish sums the
// shares in block order) and the column's bookkeeping: h_{c,c-1}, the breakdown test,
// sigma_c and its power-of-two shift (kModeInit: the start vector, ||b|| and sigma_0).
// The breakdown test compares h_{c,c-1} with 64 eps ||A v_{c-1}||, and ||A v_{c-1}||^2
// is taken as h_{c,c-1}^2 + sum_{j0 <= j < c} h_{j,c-1}^2, from the column of H that the
// orthogonalization wrote: A v_{c-1} = sum_j h_{j,c-1} v_j + h_{c,c-1} v_c with
// v_{j0..c} orthonormal (Alg. 2: every column is orthogonalized against the k before
// it, and any two columns of a window are fewer than k apart; Arnoldi: all columns).
// The test needs the norm only to a small factor, so no row of the basis pays for it.
__device__ __forceinline__ void column_norm_tail(double nrm, int c, int j0, double* __restrict__ H, int ldh,
                                                 const ColScale& cs, int mode, double* __restrict__ part,
                                                 unsigned* __restrict__ counter, DevState* st, int bid, int nblk,
                                                 double* sh, double* tot) {
  double nv[1] = {nrm};
  block_sum<1>(nv, sh);
  if (threadIdx.x == 0) part[bid] = nv[0];
  if (!last_block(counter, (unsigned)nblk)) return;
  sum_partials(part, nblk, 1, tot, sh);
  if (threadIdx.x == 0) {
    const double h = sqrt(tot[0]);
    if (mode & kModeInit) {
      st->beta = h;
      if (!isfinite(h)) {
        st->status = FAB_ENUMERIC;
        st->stop = 1;
      } else if (h == 0.0) {
        st->m_used = 0;
        st->stop = 1;
        cs.sigma[0] = 0.0;
        cs.shf[0] = 0;
      } else {
        cs.sigma[0] = 1.0 / h;
        cs.shf[0] = exponent_of(cs.sigma[0]);
      }
    } else {
      // the stored column is W_c = w' / scl[c]: h_{c,c-1} = ||w'|| = scl[c] ||W_c||
      const double hc = cs.scl[c] * h;
      H[c + (size_t)ldh * (c - 1)] = hc;
      double av2 = hc * hc;  // ||A v_{c-1}||^2
      for (int j = j0; j < c; ++j) {
        const double hj = H[j + (size_t)ldh * (c - 1)];
        av2 = fma(hj, hj, av2);
      }
      if (!isfinite(hc)) {
        st->status = FAB_ENUMERIC;
        st->stop = 1;
      } else if (!(hc > 64.0 * DBL_EPSILON * sqrt(av2))) {
        st->m_used = c;  // the basis spans an invariant subspace
        st->stop = 1;
        cs.sigma[c] = 0.0;
        cs.shf[c] = 0;
      } else {
        cs.sigma[c] = 1.0 / h;
        cs.shf[c] = exponent_of(cs.sigma[c]);
      }
    }
    *counter = 0;
  }
}


}  // namespace fab
