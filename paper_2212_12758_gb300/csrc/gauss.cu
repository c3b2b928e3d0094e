// Gaussian sketch Theta V on the GB300 tensor cores.
//
// With a dense Gaussian Theta (s x n) the sketch of the basis is a GEMM with a
// short output (s x (m+1)) and a long reduction (n): Theta V = G W with G in
// BF16 (generated once per handle) and the BF16 copy of the basis that the
// update kernel writes as each column is produced, as two BF16 terms (hi = bf16(v),
// lo = bf16(v - hi): hi + lo is v to 2^-16 relative, where hi alone is 2^-8), both
// multiplied into the same FP32 accumulator. The GEMM runs on tcgen05:
// the reduction dimension is split over the CTAs, each CTA owns one 128-row tile
// of G and one K-slice (one CTA per SM, one wave); a TMA producer lane streams 64-wide
// K tiles of G and of both basis terms into a 2- or 3-stage shared-memory ring
// (128-byte swizzle), one lane issues the UMMAs (M = 128, N = m+1 rounded to 16, K = 16,
// two per K step, FP32 accumulation in tensor
// memory), and the four warps read the accumulator back (tcgen05.ld) into an FP32
// split-K partial; a second kernel sums the partials in FP64 in a fixed order and
// applies the column scales sigma_j. Every mbarrier wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>

#include "gauss.cuh"

namespace fab {

namespace {

constexpr int kBM = 128;     // UMMA M (rows of G per CTA)
constexpr int kBK = 64;      // K elements per stage (128 bytes of BF16 = one swizzle row)
constexpr int kMaxStages = 4;  // ring depth: as many stages (4 .. 2) as fit the shared memory
constexpr int kGThreads = 128;
constexpr uint32_t kTmemCols = 256;

// BF16 bits of an FP64 value, rounded to nearest (ties to even) directly from the
// FP64 value (no intermediate FP32 rounding).
__device__ __forceinline__ unsigned short bf16_bits_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = (b >> 48) & 0x8000ull;
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  if (mag == 0) return (unsigned short)sign;
  unsigned long long keep = mag >> 45;  // FP64 exponent (11 bits) and the top 7 mantissa bits
  const unsigned long long rem = mag & ((1ull << 45) - 1);
  const unsigned long long half = 1ull << 44;
  if (rem > half || (rem == half && (keep & 1ull))) keep += 1;  // a carry into the exponent is correct
  const long long e = (long long)(keep >> 7) - 1023 + 127;
  if (e <= 0) return (unsigned short)sign;  // below the BF16 normal range (|x| < 2^-126): 0
  if (e >= 255) return (unsigned short)(sign | 0x7F80ull);
  return (unsigned short)(sign | ((unsigned long long)e << 7) | (keep & 0x7Full));
}

__global__ void k_gauss_generate(int s, int n, int spad, uint64_t stG, unsigned short* __restrict__ G) {
  const int q = blockIdx.y;  // 0 .. spad-1
  const double sq = sqrt((double)s);
  const int64_t nk = gauss_nkb(n) * 64;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x) {
    unsigned short v = 0;
    if (j < n && q < s) {
      const unsigned long long idx = (unsigned long long)q * (unsigned long long)n + (unsigned long long)j;
      const unsigned long long h1 = rng_u(stG, 2ull * idx), h2 = rng_u(stG, 2ull * idx + 1ull);
      const double u1 = ((double)(h1 >> 11) + 1.0) * 0x1p-53;
      const double u2 = (double)(h2 >> 11) * 0x1p-53;
      const double g = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2) / sq;
      v = bf16_bits_rn(g);
    }
    G[((size_t)(j >> 6) * spad + q) * 64 + (size_t)(j & 63)] = v;
  }
}

// ---------------------------------------------------------------- PTX pieces
// One box of a 3D tensor map (x: the 64 reduction indices of a block, always 0; y: the
// first row; z: the K block).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)tm), "r"(smem_addr(bar)), "r"(0), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO), the
// leading-dimension offset unused for this layout, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (16 B; ignored here)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // version
  d |= (uint64_t)2 << 61;                    // swizzle: 128 B
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both
// K-major, N and M as given.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kGThreads, 1)
    k_gauss_mma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int cpad,
                int two, int kStages, int nkb, int kb_per_split, int npad, int mpad, float* __restrict__ part,
                DevState* st) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t bytesA = kBM * kBK * 2;
  const uint32_t bytesB = (uint32_t)npad * kBK * 2;
  unsigned char* sA = base;                       // kStages tiles of 128 x 64 BF16
  unsigned char* sB = base + kStages * bytesA;    // kStages tiles of npad x 64 BF16 (hi term)
  unsigned char* sL = sB + kStages * bytesB;      // kStages tiles of npad x 64 BF16 (lo term, when two)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mtile = blockIdx.x, split = blockIdx.y;
  const int kb0 = split * kb_per_split;
  const int kb1 = min(nkb, kb0 + kb_per_split);
  const int nk = max(0, kb1 - kb0);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    mbar_fence_init();
    s_fail = 0;
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {  // TMA producer
    for (int i = 0; i < nk; ++i) {
      const int stg = i % kStages;
      if (!mbar_wait_bounded(&empty[stg], ((uint32_t)(i / kStages) & 1u) ^ 1u)) {
        s_fail = 1;
        break;
      }
      mbar_arrive_expect_tx(&full[stg], bytesA + (two ? 2u : 1u) * bytesB);
      const int kb = kb0 + i;  // every box is one contiguous block of 128 (G) or npad (basis) rows
      tma_load_3d(sA + stg * bytesA, &tmA, mtile * kBM, kb, &full[stg]);
      tma_load_3d(sB + stg * bytesB, &tmB, 0, kb, &full[stg]);
      if (two) tma_load_3d(sL + stg * bytesB, &tmB, cpad, kb, &full[stg]);
    }
  } else if (warp == 1 && lane == 0) {  // UMMA issuer
    const uint32_t idesc = idesc_bf16(kBM, npad);
    for (int i = 0; i < nk; ++i) {
      const int stg = i % kStages;
      if (!mbar_wait_bounded(&full[stg], (uint32_t)(i / kStages) & 1u)) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint64_t da = sdesc_sw128(smem_addr(sA + stg * bytesA));
      const uint64_t db = sdesc_sw128(smem_addr(sB + stg * bytesB));
      const uint64_t dl = sdesc_sw128(smem_addr(sL + stg * bytesB));
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {  // 16 BF16 = 32 bytes per UMMA K step
        umma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        if (two) umma_bf16(tmem, da + 2 * kk, dl + 2 * kk, idesc, 1u);  // G lo into the same accumulator
      }
      umma_commit(&empty[stg]);  // the stage is free once these UMMAs have read it
    }
    umma_commit(&done);
  }
  __syncwarp();
  // epilogue: warp w reads accumulator rows 32w..32w+31 (tensor-memory lanes)
  const bool ok = mbar_wait_bounded(&done, 0u);
  tc_fence_after();
  const int row = warp * 32 + lane;
  float* out = part + ((size_t)split * mpad + (size_t)mtile * kBM + row) * npad;
  const bool have = ok && nk > 0 && !s_fail;
  for (int c0 = 0; c0 < npad; c0 += 16) {
    uint32_t r[16];
    if (have) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) r[j] = 0u;
    }
#pragma unroll
    for (int j = 0; j < 16; j += 4)
      *reinterpret_cast<float4*>(out + c0 + j) =
          make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                      __uint_as_float(r[j + 3]));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
  if (threadIdx.x == 0 && (!ok || s_fail)) {
    st->status = FAB_ETIMEOUT;
    st->stop = 1;
  }
}

// SV[q + s j] = sigma_j * sum_split part[split][q][j] (FP64, fixed order)
__global__ void k_gauss_reduce(const float* __restrict__ part, int splits, int mpad, int npad, int s, int ncols,
                               const double* __restrict__ sigma, double* __restrict__ SV) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (j >= ncols || q >= s) return;
  double a = 0.0;
  for (int sp = 0; sp < splits; ++sp) a += (double)part[((size_t)sp * mpad + q) * npad + j];
  SV[q + (size_t)s * j] = sigma[j] * a;
}

struct Split {
  int mtiles, mpad, npad, nkb, kb_per_split, splits;
};

Split plan(int n, int s, int ncols) {
  Split p;
  p.mtiles = (s + kBM - 1) / kBM;
  p.mpad = p.mtiles * kBM;
  p.npad = ((ncols + 15) / 16) * 16;
  if (p.npad < 16) p.npad = 16;
  p.nkb = (n + kBK - 1) / kBK;
  // one CTA per SM and one wave: mtiles x splits <= SMs (a 156th CTA on 152 SMs would
  // run alone after the first wave and double the kernel's time)
  int want = sm_count() / p.mtiles;
  if (want < 1) want = 1;
  if (want > p.nkb) want = p.nkb;
  p.kb_per_split = (p.nkb + want - 1) / want;
  p.splits = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;
  return p;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// 3D BF16 tensor map over a K-blocked operand: x the 64 reduction indices of a block
// (128 bytes, contiguous), y the rows (rows_total, 128 bytes apart), z the K blocks
// (rows_total x 128 bytes apart); box 64 x box_rows x 1, 128-byte swizzle.
bool make_map(CUtensorMap* tm, const void* base, int rows_total, int64_t nkb, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kBK, (cuuint64_t)rows_total, (cuuint64_t)nkb};
  cuuint64_t strides[2] = {(cuuint64_t)kBK * 2, (cuuint64_t)rows_total * kBK * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The two-term BF16 copy of ncols FP64 columns (stride ldv) in the K-blocked layout
// (cpad = gauss_cpad(ncols)): hi = bf16(v), lo = bf16(v - hi), both rounded to nearest
// even from FP64 (v - hi is exact); rows past n (to the end of the last block) zero.
__device__ __forceinline__ double bf16_bits_to_double(unsigned short h) {
  return (double)__uint_as_float((unsigned)h << 16);
}
__global__ void k_to_bf16(int n, int ncols, const double* __restrict__ V, int64_t ldv, unsigned short* __restrict__ B) {
  const int j = blockIdx.y;
  const int cpad = gauss_cpad(ncols);
  const int64_t nk = gauss_nkb(n) * 64;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nk; r += (int64_t)gridDim.x * blockDim.x) {
    const double v = r < n ? V[(size_t)j * ldv + r] : 0.0;
    const unsigned short h = bf16_bits_rn(v);
    B[gauss_bidx(r, j, 0, cpad)] = h;
    B[gauss_bidx(r, j, 1, cpad)] = bf16_bits_rn(v - bf16_bits_to_double(h));
  }
}

}  // namespace

cudaError_t launch_to_bf16(int n, int ncols, const double* V, int64_t ldv, __nv_bfloat16* B, cudaStream_t st) {
  const int64_t nk = gauss_nkb(n) * 64;
  const int gx = (int)((nk + 255) / 256 < 1024 ? (nk + 255) / 256 : 1024);
  k_to_bf16<<<dim3(gx < 1 ? 1 : gx, ncols), 256, 0, st>>>(n, ncols, V, ldv, reinterpret_cast<unsigned short*>(B));
  return cudaGetLastError();
}

size_t gauss_partial_bytes(int n, int s, int ncols) {
  if (ncols < 1 || s < 1) return 0;
  const Split p = plan(n, s, ncols);
  return (size_t)p.splits * p.mpad * p.npad * sizeof(float);
}

cudaError_t launch_gauss_generate(int s, int n, uint64_t stG, __nv_bfloat16* G, cudaStream_t st) {
  const int64_t per = (gauss_nkb(n) * 64 + 255) / 256;
  const int gx = (int)(per < 1024 ? per : 1024);
  k_gauss_generate<<<dim3(gx, gauss_spad(s)), 256, 0, st>>>(s, n, gauss_spad(s), stG,
                                                             reinterpret_cast<unsigned short*>(G));
  return cudaGetLastError();
}

cudaError_t launch_gauss_sketch(const __nv_bfloat16* G, const __nv_bfloat16* B, int cpad, int n, int s, int ncols,
                                const double* sigma, double* part, double* SV, DevState* st, cudaStream_t stream) {
  if (ncols < 1 || ncols > kGaussMaxCols || cpad < gauss_cpad(ncols)) return cudaErrorInvalidValue;
  const Split p = plan(n, s, ncols);
  const int two = 1;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, G, gauss_spad(s), gauss_nkb(n), kBM) || !make_map(&tmB, B, 2 * cpad, gauss_nkb(n), p.npad))
    return cudaErrorInvalidValue;
  const size_t stage = kBM * kBK * 2 + (size_t)(1 + two) * p.npad * kBK * 2;
  const size_t cap = 227 * 1024 - 2048;  // dynamic shared memory a CTA may take, less the static part
  int nst = kMaxStages;
  while (nst > 2 && (size_t)nst * stage + 1024 > cap) --nst;
  const size_t smem = (size_t)nst * stage + 1024;
  cudaError_t e = ensure_smem_limit((const void*)k_gauss_mma, smem);
  if (e != cudaSuccess) return e;
  float* fpart = reinterpret_cast<float*>(part);
  k_gauss_mma<<<dim3(p.mtiles, p.splits), kGThreads, smem, stream>>>(tmA, tmB, cpad, two, nst, p.nkb,
                                                                      p.kb_per_split, p.npad, p.mpad, fpart, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gauss_reduce<<<dim3((ncols + 127) / 128, s), 128, 0, stream>>>(fpart, p.splits, p.mpad, p.npad, s, ncols, sigma,
                                                                   SV);
  return cudaGetLastError();
}

}  // namespace fab
