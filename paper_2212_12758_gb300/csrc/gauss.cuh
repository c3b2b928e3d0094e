// Gaussian sketch on the tensor cores (gauss.cu). Internal.
#pragma once

#include "fab_internal.cuh"

namespace fab {

constexpr int kGaussMaxCols = 256;  // m + 1 columns of the basis per sketch (one UMMA N <= 256)

// Bytes of the FP32 split-K partial buffer used by launch_gauss_sketch.
size_t gauss_partial_bytes(int n, int s, int ncols);

// G (s x n, row stride ld elements, BF16): entry (q, j) = bf16(g / sqrt(s)), g the
// Box-Muller normal of the SplitMix64 pair (2 idx, 2 idx + 1), idx = q n + j, of the
// stream whose state is stG; columns n..ld-1 are zero.
cudaError_t launch_gauss_generate(int s, int n, int64_t ld, uint64_t stG, __nv_bfloat16* G, cudaStream_t st);

// SV[q, j] = sigma_j sum_r G[q, r] Wbf_j[r] for q < s, j < ncols: BF16 products on the
// tensor cores (tcgen05, FP32 accumulation in tensor memory, split over n), FP64
// cross-split sum. `part` is scratch of gauss_partial_bytes bytes.
cudaError_t launch_gauss_sketch(const __nv_bfloat16* G, const __nv_bfloat16* Wbf, int64_t ld, int n, int s,
                                int ncols, const double* sigma, double* part, double* SV, DevState* st,
                                cudaStream_t stream);

// BF16 copy (round to nearest even) of ncols FP64 columns.
cudaError_t launch_to_bf16(int n, int ncols, const double* V, int64_t ldv, __nv_bfloat16* B, int64_t ld,
                           cudaStream_t st);

}  // namespace fab
