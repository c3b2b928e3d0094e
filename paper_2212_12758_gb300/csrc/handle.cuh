// The handle behind the C ABI (fab_api.cu) and its device workspace, shared
// with the serving runtime (server.cu). Internal.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <new>
#include <stdexcept>
#include <system_error>
#include <vector>

#include "../../include/fab.h"

namespace fab {

// The C ABI returns error codes and lets no C++ exception out. Called inside a
// catch (...) handler, this maps the exception in flight to a code: a failed host
// allocation, an impossible size or an exhausted system resource (a thread, a lock)
// is FAB_ENOMEM, anything else FAB_EINVAL.
inline int abi_error_code() noexcept {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return FAB_ENOMEM;
  } catch (const std::length_error&) {
    return FAB_ENOMEM;
  } catch (const std::system_error&) {
    return FAB_ENOMEM;
  } catch (...) {
    return FAB_EINVAL;
  }
}

// Grow-only device buffer.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Grow-only device buffer; returns false on allocation failure.
inline bool ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return true;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b.bytes = bytes;
  return true;
}

template <typename T>
T* ptr(Buf& b) {
  return reinterpret_cast<T*>(b.p);
}

}  // namespace fab

struct fab_handle {
  int n = 0, nnz = 0;
  bool owns_matrix = true;     // false for workspace clones (they share the device CSR)
  int* d_rowptr = nullptr;
  int* d_colind = nullptr;
  double* d_vals = nullptr;
  float* d_vals32 = nullptr;  // FP32 copy for the mixed-precision path (made on first use)
  int64_t ld = 0;
  // SpMV row tiles (see build_tiles); shared by workspace clones
  int* d_tiles = nullptr;
  int ntiles = 0;
  int tile_rows = 256, tile_nnz = 2048, tile_staged = 1;
  // one-pass basis steps for the FP32 basis (fused.cu): allowed when every row has at
  // most 8 nonzeros (max_row_nnz, set by fab_create) and fuse = 1 (fab_set_fusion; the
  // default 0 keeps the two-pass loop, measured faster on GB300)
  int max_row_nnz = 0;
  int fuse = 0;
  int* d_ftasks = nullptr;  // the one-pass steps' task claim order (2 chunks ints) and, per
  int* d_fcrange = nullptr; // chunk, the first and last chunk its rows reference (shared by clones)
  int* d_ell_col = nullptr;  // the FP32 matrix in ELL form for the one-pass steps (max_row_nnz
  float* d_ell_val = nullptr;  // slots of ld entries), made with the FP32 copy (shared by clones)
  int* h_rowptr = nullptr;  // host copy of the row pointers (n+1), for re-tiling
  // workspace
  fab::Buf W, H, sigma, shf, scl, coef, part, counter, gpart, skpart, SV, P, qr, tau, y, cvec, dense, piv, scal, lsq, u, xbuf,
      state;
  fab::Buf W32, Wbf, G;  // mixed path: FP32 basis, its BF16 copy, Gaussian sketch (BF16, s x ld)
  fab::Buf wbuf;         // mixed path, one-pass steps: two raw SpMV outputs (2 ld floats)
  fab::Buf fflags;       // one-pass steps: per-chunk flags of the updated column
  int stall_pass = 0, stall_polls = 0;  // fab_inject_wait_timeout (one-shot)
  fab::Buf whm;          // FAB_WHITEN: R, R^{-1}, scratch ((m+1)^2 each), coefficients, norms
  int G_n = -1, G_s = -1;
  uint64_t G_seed = 0;
  // cached sparse sign pattern (zeta x n, see SketchDev::pat)
  fab::Buf spat;
  int spat_n = -1, spat_s = -1, spat_zeta = -1;
  uint64_t spat_seed = 0;
  // cached SRHT sample
  int64_t P_npad = -1;
  int P_s = -1;
  uint64_t P_seed = 0;
  // pinned host scratch for the solve's small readbacks (status word, norms)
  void* h_pinned = nullptr;
  // sign(A) b: the handle of A^2 (built on first use) and device scratch for b, A b
  fab_handle* sq = nullptr;
  fab::Buf sbuf;
  // last solve
  int has_state = 0, last_m = 0, last_s = 0, last_sketched = 0, last_mixed = 0, last_ldh = 0;
};

namespace fab {
// Device bytes the workspace of a solve with these parameters occupies (estimate
// used by admission control), and bytes currently allocated by a handle.
size_t estimate_ws_bytes(const fab_handle* h, const fab_params* p);
size_t handle_ws_bytes(const fab_handle* h);
// A handle that shares h's device matrix and owns a fresh (empty) workspace.
fab_handle* clone_for_workspace(const fab_handle* h);
// Re-point a workspace clone at another matrix (its workspace is kept).
void point_to_matrix(fab_handle* clone, const fab_handle* h);
// FP32 copy of A's values for the mixed-precision path (once per matrix).
int ensure_vals32(fab_handle* h, cudaStream_t s);
// Sets this host thread's fab_last_error() text (carries a serving slot's detail to the poller).
void set_last_error(const char* msg);
// Recut A's SpMV row tiles: consecutive rows, at most rows_max rows and at most
// nnz_cap nonzeros per tile (a longer row is a tile of its own); staged = 1
// stages tiles in shared memory. FAB_OK, FAB_EINVAL or FAB_ENOMEM.
int build_tiles(fab_handle* h, int rows_max, int nnz_cap, int staged);
// The CSR view of h's matrix for the basis kernels (vals: FP64 or FP32 copy).
struct Csr;
// This host thread's solves wait on a blocking-sync event (sleep) instead of spinning.
void use_blocking_waits(bool on);
// Parameter checks of fab_apply (FAB_OK or FAB_EINVAL).
int validate_params(const fab_handle* h, const fab_params* p);
// Pade [13/13] numerator coefficients b_0..b_13 and the threshold theta_13.
const double* pade13_b();
double pade13_theta();
// Host-side allocation fault injection (FAB_FAULT=alloc:N): true for the N-th call.
bool alloc_fault();
// The one-pass steps' plan of a matrix (fused.cu): per 4096-row chunk the first and
// last chunk its rows reference, and the claim order of the update and SpMV tasks.
// lead: extra chunks the updates run ahead of the SpMV tasks.
void fused_plan(int n, const int* rowptr, const int* colind, int lead, std::vector<int>& tasks,
                std::vector<int2>& crange);

}  // namespace fab
