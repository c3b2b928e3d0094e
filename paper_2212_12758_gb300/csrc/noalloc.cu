// fab_sketch_apply_noalloc: the sketch Theta V of fab_sketch_apply, with all of
// its scratch (per-chunk partial sums, the SRHT row sample, the device status
// word) in one fixed, file-scope device array instead of memory allocated per
// call. For callers that must not allocate device memory while they run.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fab_internal.cuh"
#include "handle.cuh"

namespace {

constexpr size_t kStateBytes = 256;                         // DevState, padded
constexpr size_t kPBytes = (size_t)fab::kMaxS * sizeof(int);  // SRHT sampled rows
constexpr size_t kPartDoubles = (size_t)1 << 20;            // chunk partials: 8 MiB
constexpr size_t kScratchBytes = kStateBytes + kPBytes + kPartDoubles * sizeof(double);
// The status word sits in the first kStateBytes; the row sample and the partials
// follow it and must neither overlap it nor lose the 256-byte alignment.
static_assert(sizeof(fab::DevState) <= kStateBytes, "DevState outgrew its slot in the fixed scratch");
static_assert(kStateBytes % 256 == 0 && kPBytes % 256 == 0, "scratch pieces keep 256-byte alignment");

// Shared by every call on a device; kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per
// device). Returns nullptr on failure.
unsigned char* scratch_for_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  return static_cast<unsigned char*>(g_scratch_addr[dev]);
}

int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

}  // namespace

extern "C" int fab_sketch_apply_noalloc(int sketch, int64_t n, int s, int zeta, uint64_t seed, const double* V_dev,
                                        int64_t ldv, int ncols, double* out_dev, void* stream) try {
  using namespace fab;
  if (n < 1 || n >= (int64_t)1 << 31 || s < 1 || s > kMaxS || ncols < 0 || ldv < n || !V_dev || !out_dev)
    return FAB_EINVAL;
  if (sketch == FAB_SK_SPARSE_SIGN) {
    if (zeta < 1 || zeta > kMaxZeta || zeta > s) return FAB_EINVAL;
  } else if (sketch == FAB_SK_SRHT) {
    if (s > next_pow2(n)) return FAB_EINVAL;
  } else {
    return FAB_EINVAL;
  }
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  if ((uint64_t)nchunks * (uint64_t)s > kPartDoubles) return FAB_EINVAL;  // beyond the fixed scratch
  if (ncols == 0) return FAB_OK;
  unsigned char* base = scratch_for_current_device();
  if (!base) return FAB_ECUDA;
  DevState* ds = reinterpret_cast<DevState*>(base);
  int* P = reinterpret_cast<int*>(base + kStateBytes);
  double* part = reinterpret_cast<double*>(base + kStateBytes + kPBytes);
  cudaStream_t st = (cudaStream_t)stream;

  SketchDev sk;
  memset(&sk, 0, sizeof(sk));
  sk.kind = sketch == FAB_SK_SRHT ? SK_SRHT : SK_SPARSE;
  sk.s = s;
  sk.zeta = zeta;
  sk.chunk_log2 = kChunkLog2;
  sk.nchunks = (int)nchunks;
  sk.st_rows = rng_state(seed, 1);
  sk.st_signs = rng_state(seed, 2);
  sk.st_D = rng_state(seed, 3);
  sk.P = P;
  sk.part = part;
  const double scale = sk.kind == SK_SRHT ? 1.0 / sqrt((double)s) : 1.0 / sqrt((double)zeta);
  // The status word is the only scratch that must start cleared; the row sample
  // and every chunk partial read later are rewritten by this call.
  if (launch_state_reset(ds, 0, st) != cudaSuccess) return FAB_ECUDA;
  if (sk.kind == SK_SRHT && launch_srht_sample(next_pow2(n), s, rng_state(seed, 4), P, st) != cudaSuccess)
    return FAB_ECUDA;
  for (int j = 0; j < ncols; ++j) {
    if (launch_update((int)n, const_cast<double*>(V_dev), ldv, j, 0, 0, nullptr, nullptr, 1, ColScale{}, 0,
                      nullptr, nullptr, sk, ds, st) != cudaSuccess ||
        launch_sketch_reduce(sk, nullptr, 0, scale, out_dev + (size_t)j * s, ds, st) != cudaSuccess)
      return FAB_ECUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}
