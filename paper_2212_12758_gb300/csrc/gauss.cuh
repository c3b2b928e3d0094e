// Gaussian sketch on the tensor cores (gauss.cu). Internal.
#pragma once

#include "fab_internal.cuh"

namespace fab {

constexpr int kGaussMaxCols = 256;  // m + 1 columns of the basis per sketch (one UMMA N <= 256)

// K-blocked layouts of the operands (64 reduction indices per block, each block of all
// rows contiguous, so that every tensor-core tile is one contiguous copy):
//   G (s x n):  entry (q, j) at ((j / 64) spad + q) 64 + j % 64, spad = s rounded up to 128;
//   the two-term BF16 copy of the basis: (row r, column c, term t in {0: hi, 1: lo}) at
//   ((r / 64) 2 cpad + t cpad + c) 64 + r % 64, cpad = the columns rounded up to 16.
// Reduction indices past n are zero in G; the copy's rows past n must be finite (zeroed).
__host__ __device__ inline int gauss_spad(int s) { return ((s + 127) / 128) * 128; }
__host__ __device__ inline int gauss_cpad(int ncols) { return ((ncols + 15) / 16) * 16; }
__host__ __device__ inline int64_t gauss_nkb(int64_t n) { return (n + 63) / 64; }
__host__ __device__ inline size_t gauss_bidx(int64_t r, int col, int t, int cpad) {
  return ((size_t)(r >> 6) * 2 * cpad + (size_t)t * cpad + col) * 64 + (size_t)(r & 63);
}
inline size_t gauss_G_bytes(int64_t n, int s) { return (size_t)gauss_nkb(n) * gauss_spad(s) * 64 * 2; }
inline size_t gauss_B_bytes(int64_t n, int ncols) { return (size_t)gauss_nkb(n) * 2 * gauss_cpad(ncols) * 64 * 2; }

// Bytes of the FP32 split-K partial buffer used by launch_gauss_sketch.
size_t gauss_partial_bytes(int n, int s, int ncols);

// G (s x n, K-blocked, gauss_G_bytes): entry (q, j) = bf16(g / sqrt(s)), g the Box-Muller
// normal of the SplitMix64 pair (2 idx, 2 idx + 1), idx = q n + j, of the stream whose
// state is stG; padding (q >= s or j >= n) zero.
cudaError_t launch_gauss_generate(int s, int n, uint64_t stG, __nv_bfloat16* G, cudaStream_t st);

// SV[q, j] = sigma_j sum_r G[q, r] (hi_j[r] + lo_j[r]) for q < s, j < ncols, from the
// two-term copy B (K-blocked with cpad >= gauss_cpad(ncols) columns per term): BF16
// products on the tensor cores (tcgen05, both terms into one FP32 accumulator in tensor
// memory, split over n), FP64 cross-split sum. `part` is scratch of gauss_partial_bytes.
cudaError_t launch_gauss_sketch(const __nv_bfloat16* G, const __nv_bfloat16* B, int cpad, int n, int s, int ncols,
                                const double* sigma, double* part, double* SV, DevState* st, cudaStream_t stream);

// The two-term BF16 copy (hi = bf16(v), lo = bf16(v - hi), round to nearest even) of
// ncols FP64 columns into B (K-blocked, cpad = gauss_cpad(ncols)); rows past n zero.
cudaError_t launch_to_bf16(int n, int ncols, const double* V, int64_t ldv, __nv_bfloat16* B, cudaStream_t st);

}  // namespace fab
