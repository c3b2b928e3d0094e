// Batched solves of libfab: many f(A)b solves of uneven size (different
// matrices, n, m, window k, sketch and f) captured into one CUDA graph.
//
// The plan lists phases: for every basis step c, per (window, sketch kind) group,
// the SpMV + window dots, then the window update + norm + fused sketch, then the
// sketch reduce (Alg. 2 with the sketch of §2.1.1), each over every solve still
// building its basis. A solve's blocks in a phase run the bodies of its own
// launches on the same tiles and chunks (with at least kMinTiles SpMV tiles per
// block), so its results equal fab_apply's up to the grouping of partial sums. The
// whole basis build is one persistent launch (k_batch_basis: blocks claim the
// plan's work items in order and wait only for their own solve's previous phase),
// then one launch runs every solve's small stage as one CTA (QR of the sketch, the
// sketch-and-solve projection of eq. sFOM or none for Alg. 5, f(H)e_1) and one
// the combines x = ||b|| V_m c. The graph holds these three kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <tuple>
#include <vector>

#include "handle.cuh"
#include "small.cuh"

namespace {

using namespace fab;

constexpr int kReduceEntries = 8 * 32;  // sketch entries per block of the reduce phase (a warp per entry, 32 rounds)

// Bump allocator over one device allocation (sizing pass when base is NULL).
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

enum WaveType { W_INIT, W_SPMV, W_UPDATE, W_REDUCE, W_SMALL, W_COMBINE };

struct HostWave {
  int type;
  int c = 0, arg = 0, mode = 0, kind = SK_NONE;  // arg: window / update column count
  size_t smem = 0;
  int nblocks = 0;
  size_t pre = 0, ids = 0, aux = 0, seq = 0;  // offsets into the table
  int count = 0;
  int mmax = 0;
};

int sk_kind_of(const fab_params& p) {
  if (p.method != FAB_SKETCHED_FAST) return SK_NONE;
  return p.sketch == FAB_SK_SRHT ? SK_SRHT : SK_SPARSE_TAB;  // sparse sign: pattern drawn once, at creation
}

// A batched solve's blocks: its own launch's grid, but at least kMinTiles SpMV
// tiles and kMinChunks update chunks per block (a solve shares the GPU with the
// rest of the batch, so fewer, longer blocks amortise each block's start-up and
// its partial-sum reduction).
constexpr int kMinTiles = 32;
constexpr int kMinChunks = 4;
// Polls (each a 64 ns sleep and an L2 round trip) of a solve's phase counter before
// the waiting block gives up: seconds, far beyond any phase's duration.
constexpr int kPhasePolls = 1 << 22;

}  // namespace

struct fab_batch {
  int count = 0;
  bool mixed = false;
  void* mem = nullptr;
  size_t bytes = 0;
  std::vector<int> n;
  std::vector<double*> bdev, xdev;
  DevState* states = nullptr;
  std::vector<DevState> hst;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  int kernels = 0;
};

namespace {

template <typename TV>
int build(fab_batch* bt, fab_handle* const* hs, const fab_params* ps, cudaStream_t user) {
  const int count = bt->count;
  // ------------------------------------------------------------ plan
  std::vector<int> kind(count);
  int mmax = 1;
  for (int j = 0; j < count; ++j) {
    kind[j] = sk_kind_of(ps[j]);
    mmax = std::max(mmax, ps[j].m);
  }
  // groups: distinct (k, sketch kind); waves of a group share the kernel template
  std::vector<std::pair<int, int>> groups;
  std::vector<int> group_of(count);
  for (int j = 0; j < count; ++j) {
    const std::pair<int, int> g{ps[j].k, kind[j]};
    auto it = std::find(groups.begin(), groups.end(), g);
    if (it == groups.end()) {
      groups.push_back(g);
      it = groups.end() - 1;
    }
    group_of[j] = (int)(it - groups.begin());
  }
  std::vector<int> tab;  // wave tables (prefix, ids, aux, phase numbers), uploaded once
  std::vector<HostWave> waves;  // the basis phases, in plan order
  std::vector<int> phases(count, 0);  // per solve: phases planned so far
  auto add_table = [&](HostWave& w, const std::vector<int>& ids, const std::vector<int>& nblk,
                       const std::vector<int>& aux) {
    w.count = (int)ids.size();
    w.pre = tab.size();
    int acc = 0;
    tab.push_back(0);
    for (int b : nblk) tab.push_back(acc += b);
    w.nblocks = acc;
    w.ids = tab.size();
    tab.insert(tab.end(), ids.begin(), ids.end());
    w.aux = tab.size();
    if (aux.empty()) tab.insert(tab.end(), ids.size(), 0);
    else tab.insert(tab.end(), aux.begin(), aux.end());
    w.seq = tab.size();
    for (int j : ids) tab.push_back(phases[j]++);
  };
  auto add_wave = [&](HostWave w, const std::vector<int>& ids, const std::vector<int>& nblk,
                      const std::vector<int>& aux) {
    if (ids.empty()) return;
    add_table(w, ids, nblk, aux);
    waves.push_back(w);
  };
  {  // start: state, counters, H = 0, W_0 = b
    std::vector<int> ids, nb;
    for (int j = 0; j < count; ++j) {
      ids.push_back(j);
      nb.push_back(std::max(1, std::min((bt->n[j] + 2047) / 2048, 128)));
    }
    add_wave(HostWave{W_INIT}, ids, nb, {});
  }
  std::vector<size_t> part_need(count, 1);  // per-solve partial counts
  std::vector<int> upd_blocks(count, 1);     // per solve: the largest update grid (sketch partials per column)
  for (int c = 0; c <= mmax; ++c) {
    for (int g = 0; g < (int)groups.size(); ++g) {
      const int k = groups[g].first, kd = groups[g].second;
      std::vector<int> ids;
      for (int j = 0; j < count; ++j)
        if (group_of[j] == g && ps[j].m >= c) ids.push_back(j);
      if (ids.empty()) continue;
      const int kw = c == 0 ? 0 : std::min(c, k);
      if (c > 0) {
        std::vector<int> nb;
        for (int j : ids) {
          nb.push_back(std::min(spmv_grid<TV>(hs[j]->ntiles, kw, false), (hs[j]->ntiles + kMinTiles - 1) / kMinTiles));
          part_need[j] = std::max(part_need[j], (size_t)nb.back() * (kMaxWindow + 1));
        }
        HostWave w{W_SPMV};
        w.c = c;
        w.arg = kw;
        add_wave(w, ids, nb, {});
      }
      std::vector<int> nb;
      size_t smem = 0;
      for (int j : ids) {
        size_t sm = 0;
        const int s = kd == SK_NONE ? 0 : ps[j].s;
        int grid = update_grid<TV>(kd, bt->n[j], kw, s, &sm);
        if (grid < 1) return FAB_ECUDA;
        grid = std::min(grid, ((bt->n[j] + kChunk - 1) / kChunk + kMinChunks - 1) / kMinChunks);
        nb.push_back(grid);
        smem = std::max(smem, sm);
        part_need[j] = std::max(part_need[j], (size_t)grid);
        upd_blocks[j] = std::max(upd_blocks[j], grid);
      }
      HostWave w{W_UPDATE};
      w.c = c;
      w.arg = kw;
      w.mode = c == 0 ? 3 : 1;
      w.kind = kd;
      w.smem = smem;
      add_wave(w, ids, nb, {});
    }
  }
  // The sketch partials of every column stay (column c at c * colstride), so one
  // reduce phase per sketched solve, after its basis, forms all of Theta V (a warp
  // per sketch entry) instead of a reduce phase per step.
  {
    std::vector<int> ids, nr, np;
    for (int j = 0; j < count; ++j)
      if (kind[j] != SK_NONE) {
        ids.push_back(j);
        nr.push_back((int)(((size_t)(ps[j].m + 1) * ps[j].s + kReduceEntries - 1) / kReduceEntries));
        np.push_back(upd_blocks[j]);  // partials per column: the largest update grid
      }
    HostWave r{W_REDUCE};
    add_wave(r, ids, nr, np);
  }
  // after the basis: every solve's small stage (one CTA each), then every combine
  std::vector<int> all(count), ones(count, 1), ncomb(count);
  for (int j = 0; j < count; ++j) {
    all[j] = j;
    ncomb[j] = combine_grid(bt->n[j]);
  }
  HostWave small_w{W_SMALL};
  small_w.mmax = mmax;
  add_table(small_w, all, ones, {});
  HostWave comb_w{W_COMBINE};
  comb_w.mmax = mmax;
  add_table(comb_w, all, ncomb, {});
  int kmax = 1;
  for (int j = 0; j < count; ++j) kmax = std::max(kmax, ps[j].k);

  // ------------------------------------------------------------ work items
  // every block of every phase, in plan order, decoded once here (see BatchPlan)
  std::vector<int4> items;
  size_t upd_smem = 0;
  for (const HostWave& w : waves) {
    const int type = w.type == W_INIT ? kPhInit : w.type == W_SPMV ? kPhSpmv : w.type == W_UPDATE ? kPhUpdate : kPhReduce;
    if (w.type == W_UPDATE) upd_smem = std::max(upd_smem, w.smem);
    for (int i = 0; i < w.count; ++i) {
      const int j = tab[w.ids + i], nb = tab[w.pre + i + 1] - tab[w.pre + i], seq = tab[w.seq + i];
      const int arg = type == kPhReduce ? tab[w.aux + i] : w.arg;
      if (nb >= 65536 || seq >= 65536 || w.c >= 65536 || arg >= (1 << 23) || w.kind + 1 > 7) return FAB_EINVAL;
      const int code = type | (w.mode << 2) | ((w.kind + 1) << 4) | (arg << 8);
      for (int b = 0; b < nb; ++b) items.push_back(make_int4(j, b | (nb << 16), seq | (w.c << 16), code));
    }
  }
  const size_t n_items = items.size();

  // ------------------------------------------------------------ layout
  std::vector<BasisJob<TV>> jobs(count);
  std::vector<SmallJob> small(count);
  auto layout = [&](Arena& ar) {
    BasisJob<TV>* jobs_dev = ar.take<BasisJob<TV>>(count);
    SmallJob* small_dev = ar.take<SmallJob>(count);
    int* tab_dev = ar.take<int>(tab.size());
    DevState* states = ar.take<DevState>(count);
    int4* items_dev = ar.take<int4>(n_items);
    unsigned* ctr_dev = ar.take<unsigned>(1 + 2 * (size_t)count);  // ticket, done[count], blk[count]
    for (int j = 0; j < count; ++j) {
      fab_handle* h = hs[j];
      const fab_params& p = ps[j];
      const int n = h->n, m = p.m, s = kind[j] == SK_NONE ? 1 : p.s;
      BasisJob<TV>& J = jobs[j];
      memset(&J, 0, sizeof(J));
      J.A = Csr{h->n,
                h->nnz,
                h->d_rowptr,
                h->d_colind,
                bt->mixed ? (const void*)h->d_vals32 : (const void*)h->d_vals,
                h->d_tiles,
                h->ntiles,
                h->tile_staged};
      J.ld = h->ld;
      J.W = ar.take<TV>((size_t)h->ld * (m + 1));
      J.cs.sigma = ar.take<double>(m + 1);
      J.cs.shf = ar.take<int>(m + 1);
      J.cs.scl = ar.take<double>(m + 1);
      J.H = ar.take<double>((size_t)(m + 1) * m);
      J.ldh = m + 1;
      J.m = m;
      J.k = p.k;
      J.coef = ar.take<double>(m + 1);
      J.part = ar.take<double>(part_need[j]);
      J.counter = ar.take<unsigned>(16);
      J.st = states ? states + j : nullptr;
      J.SV = ar.take<double>((size_t)s * (m + 1));
      SketchDev& sk = J.sk;
      sk.kind = kind[j];
      sk.s = kind[j] == SK_NONE ? 0 : p.s;
      sk.zeta = p.zeta;
      sk.chunk_log2 = kChunkLog2;
      sk.nchunks = (n + kChunk - 1) / kChunk;
      sk.st_rows = rng_state(p.seed, 1);
      sk.st_signs = rng_state(p.seed, 2);
      sk.st_D = rng_state(p.seed, 3);
      sk.P = ar.take<int>(s);
      J.sk_colstride = (size_t)upd_blocks[j] * (size_t)std::max(s, 1);
      sk.part = ar.take<double>((size_t)(m + 1) * J.sk_colstride);
      sk.pat = kind[j] == SK_SPARSE_TAB ? ar.take<unsigned short>(sparse_table_bytes(n, p.s, p.zeta) / 2) : nullptr;
      J.sk_scale = kind[j] == SK_SRHT ? 1.0 / sqrt((double)p.s) : (kind[j] == SK_SPARSE_TAB ? 1.0 / sqrt((double)p.zeta) : 1.0);
      double* bst = ar.take<double>(n);
      double* xst = ar.take<double>(n);
      J.b = bst;
      J.x = xst;
      if (ar.base) {
        bt->bdev[j] = bst;
        bt->xdev[j] = xst;
      }
      SmallJob& S = small[j];
      memset(&S, 0, sizeof(S));
      S.method = p.method;
      S.f = p.f;
      S.m = m;
      S.s = s;
      S.t = p.t;
      S.H = J.H;
      S.ldh = J.ldh;
      S.SV = J.SV;
      S.sigma = J.cs.sigma;
      S.st = J.st;
      S.qr = ar.take<double>((size_t)s * (m + 1));
      S.tau = ar.take<double>(m + 1);
      S.y = ar.take<double>(m + 1);
      S.mats = ar.take<double>((size_t)9 * m * m);
      S.piv = ar.take<int>(m + 1);
      S.cvec = ar.take<double>(m + 1);
      S.scal = ar.take<double>(16);
      S.coef = J.coef;
    }
    return std::make_tuple(jobs_dev, small_dev, tab_dev, states, items_dev, ctr_dev);
  };
  Arena sizing;
  layout(sizing);
  const size_t bytes = sizing.off + 256;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  if (bytes > free_b || alloc_fault()) return FAB_ENOMEM;
  if (cudaMalloc(&bt->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    bt->mem = nullptr;
    return FAB_ENOMEM;
  }
  bt->bytes = bytes;
  Arena ar;
  ar.base = reinterpret_cast<char*>(bt->mem);
  BasisJob<TV>* jobs_dev;
  SmallJob* small_dev;
  int* tab_dev;
  int4* items_dev;
  unsigned* ctr_dev;
  std::tie(jobs_dev, small_dev, tab_dev, bt->states, items_dev, ctr_dev) = layout(ar);
  BatchPlan plan;
  plan.items = items_dev;
  plan.total = (unsigned)items.size();
  plan.ticket = ctr_dev;
  plan.done = ctr_dev + 1;
  plan.blk = ctr_dev + 1 + count;
  plan.poll_limit = kPhasePolls;
  const size_t basis_smem = std::max(upd_smem, (size_t)kSpmvStages * kSpmvCap * (sizeof(TV) + sizeof(int)));

  cudaStream_t cap = nullptr;
  auto cleanup = [&]() {
    if (cap) cudaStreamDestroy(cap);
  };
#define BK(call)              \
  do {                        \
    if ((call) != cudaSuccess) { \
      cudaGetLastError();     \
      cleanup();              \
      return FAB_ECUDA;       \
    }                         \
  } while (0)
  BK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  BK(cudaMemcpyAsync(jobs_dev, jobs.data(), sizeof(BasisJob<TV>) * count, cudaMemcpyHostToDevice, cap));
  BK(cudaMemcpyAsync(small_dev, small.data(), sizeof(SmallJob) * count, cudaMemcpyHostToDevice, cap));
  BK(cudaMemcpyAsync(tab_dev, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, cap));
  BK(cudaMemcpyAsync(items_dev, items.data(), sizeof(int4) * n_items, cudaMemcpyHostToDevice, cap));
  for (int j = 0; j < count; ++j) {  // SRHT samples and sparse sign patterns are fixed: drawn once here
    if (kind[j] == SK_SRHT) {
      int64_t npad = 1;
      while (npad < bt->n[j]) npad <<= 1;
      BK(launch_srht_sample(npad, ps[j].s, rng_state(ps[j].seed, 4), const_cast<int*>(jobs[j].sk.P), cap));
    }
    if (kind[j] == SK_SPARSE_TAB)
      BK(launch_sparse_pattern(bt->n[j], jobs[j].sk, const_cast<unsigned short*>(jobs[j].sk.pat), cap));
  }
  for (int j = 0; j < count; ++j)  // partial slots a column's update grid leaves unwritten read as zero
    if (kind[j] != SK_NONE)
      BK(cudaMemsetAsync(jobs[j].sk.part, 0, (size_t)(ps[j].m + 1) * jobs[j].sk_colstride * sizeof(double), cap));
  BK(cudaStreamSynchronize(cap));
  PadeCoef pd;
  memcpy(pd.b, pade13_b(), sizeof(pd.b));
  pd.theta = pade13_theta();
  // every kernel gets its shared-memory limit before the capture
  BK(small_fused_prepare(mmax));
  int basis_grid = 0;
  BK(batch_basis_prepare<TV>(kmax, basis_smem, &basis_grid));

  // ------------------------------------------------------------ capture
  BK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(ctr_dev, 0, (1 + 2 * (size_t)count) * sizeof(unsigned), cap);
  if (e == cudaSuccess) e = launch_batch_basis<TV>(jobs_dev, plan, kmax, basis_grid, basis_smem, cap);
  if (e == cudaSuccess) e = launch_small_fused(small_dev, tab_dev + small_w.ids, count, mmax, pd, cap);
  if (e == cudaSuccess) {
    const Wave cw{tab_dev + comb_w.pre, tab_dev + comb_w.ids, tab_dev + comb_w.aux, comb_w.count};
    e = launch_combine_wave<TV>(jobs_dev, cw, comb_w.nblocks, mmax, cap);
  }
  const int kernels = 3;
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    cleanup();
    return FAB_ECUDA;
  }
  e = cudaGraphInstantiate(&bt->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) e = cudaGraphUpload(bt->exec, user);
  if (e == cudaSuccess) e = cudaStreamSynchronize(user);
  cleanup();
#undef BK
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FAB_ECUDA;
  }
  bt->kernels = kernels;
  return FAB_OK;
}

}  // namespace

extern "C" int fab_batch_create(fab_batch** out, fab_handle* const* hs, const fab_params* ps, int count) try {
  if (!out) return FAB_EINVAL;
  *out = nullptr;
  if (!hs || !ps || count < 1) return FAB_EINVAL;
  const int prec = ps[0].precision;
  for (int j = 0; j < count; ++j) {
    const fab_params& p = ps[j];
    if (!hs[j] || validate_params(hs[j], &p) != FAB_OK) return FAB_EINVAL;
    if (p.precision != prec || p.target_rel_err != 0.0 || p.f == FAB_F_SIGN) return FAB_EINVAL;
    if (p.method != FAB_SKETCHED_FAST && p.method != FAB_NOPROJ) return FAB_EINVAL;
    if (p.method == FAB_SKETCHED_FAST && p.sketch != FAB_SK_SRHT && p.sketch != FAB_SK_SPARSE_SIGN)
      return FAB_EINVAL;
  }
  cudaStream_t user = (cudaStream_t)ps[0].stream;
  if (prec == FAB_MIXED)
    for (int j = 0; j < count; ++j) {
      const int rc = ensure_vals32(hs[j], user);
      if (rc != FAB_OK) return rc;
    }
  fab_batch* bt = new fab_batch();
  // Releases a partly built batch on every early return and on an exception.
  struct Owner {
    fab_batch* bt;
    ~Owner() {
      if (bt) fab_batch_destroy(bt);
    }
  } owner{bt};
  bt->count = count;
  bt->mixed = prec == FAB_MIXED;
  bt->n.resize(count);
  bt->bdev.resize(count);
  bt->xdev.resize(count);
  bt->hst.resize(count);
  for (int j = 0; j < count; ++j) bt->n[j] = hs[j]->n;
  int rc = bt->mixed ? build<float>(bt, hs, ps, user) : build<double>(bt, hs, ps, user);
  if (rc == FAB_OK && (cudaEventCreate(&bt->t0) != cudaSuccess || cudaEventCreate(&bt->t1) != cudaSuccess)) {
    cudaGetLastError();
    rc = FAB_ECUDA;
  }
  if (rc != FAB_OK) return rc;
  owner.bt = nullptr;
  *out = bt;
  return FAB_OK;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" int fab_batch_exec(fab_batch* bt, const double* const* bs, double* const* xs, fab_stats* sts,
                              void* stream) try {
  if (!bt || !bt->exec) return FAB_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int count = bt->count;
  if (bs)
    for (int j = 0; j < count; ++j) {
      if (!bs[j]) return FAB_EINVAL;
      if (cudaMemcpyAsync(bt->bdev[j], bs[j], (size_t)bt->n[j] * sizeof(double), cudaMemcpyDefault, s) !=
          cudaSuccess)
        goto cuda_fail;
    }
  if (cudaEventRecord(bt->t0, s) != cudaSuccess || cudaGraphLaunch(bt->exec, s) != cudaSuccess ||
      cudaEventRecord(bt->t1, s) != cudaSuccess)
    goto cuda_fail;
  if (cudaMemcpyAsync(bt->hst.data(), bt->states, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    goto cuda_fail;
  if (xs)
    for (int j = 0; j < count; ++j) {
      if (!xs[j]) continue;
      if (cudaMemcpyAsync(xs[j], bt->xdev[j], (size_t)bt->n[j] * sizeof(double), cudaMemcpyDefault, s) !=
          cudaSuccess)
        goto cuda_fail;
    }
  if (cudaStreamSynchronize(s) != cudaSuccess) goto cuda_fail;
  {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, bt->t0, bt->t1);
    int rc = FAB_OK;
    for (int j = 0; j < count; ++j) {
      const DevState& d = bt->hst[j];
      if (d.status != FAB_OK && rc == FAB_OK) rc = d.status;
      if (sts) {
        fab_stats& st = sts[j];
        memset(&st, 0, sizeof(st));
        st.m_used = d.m_used;
        st.fh_iters = d.iters;
        st.launches = bt->kernels;
        st.beta = d.beta;
        st.h_last = d.scal[15];
        st.ms_total = ms;
      }
    }
    return rc;
  }
cuda_fail:
  cudaGetLastError();
  return FAB_ECUDA;
} catch (...) {
  return fab::abi_error_code();
}

extern "C" double* fab_batch_input(fab_batch* bt, int i) {
  return (bt && i >= 0 && i < bt->count) ? bt->bdev[i] : nullptr;
}

extern "C" double* fab_batch_output(fab_batch* bt, int i) {
  return (bt && i >= 0 && i < bt->count) ? bt->xdev[i] : nullptr;
}

extern "C" int fab_batch_kernels(const fab_batch* bt) { return bt ? bt->kernels : 0; }

extern "C" void fab_batch_destroy(fab_batch* bt) try {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->t0) cudaEventDestroy(bt->t0);
  if (bt->t1) cudaEventDestroy(bt->t1);
  if (bt->mem) cudaFree(bt->mem);
  cudaGetLastError();
  delete bt;
} catch (...) {
}

extern "C" int fab_batch_run(fab_handle* const* hs, const fab_params* ps, const double* const* bs, double* const* xs,
                             int count, fab_stats* sts) try {
  if (!bs || !xs) return FAB_EINVAL;
  fab_batch* bt = nullptr;
  int rc = fab_batch_create(&bt, hs, ps, count);
  if (rc != FAB_OK) return rc;
  rc = fab_batch_exec(bt, bs, xs, sts, ps[0].stream);
  fab_batch_destroy(bt);
  return rc;
} catch (...) {
  return fab::abi_error_code();
}
