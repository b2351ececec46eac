// Batched form: many independent CSR matrices processed by one persistent
// kernel (warps walk the concatenated tile directory of all matrices) and
// one fix-up kernel; the partition counts and tile sizes per size bucket
// come from a tuning table that msrep_autotune measures.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "spmv_core.cuh"
#include "batch.cuh"

namespace msrep {

msrep_status check_matrix(const msrep_matrix *A);
int32_t effective_tile(int32_t tile);
int *kernel_err_ptr();


// Thread-block shapes of the batched kernel (warps per block) and the
// resident blocks asked of the register allocator for each: the same budget
// of about 80 registers a thread as the single-matrix CSR kernel for 4 and
// 8 warps (24 warps per SM); 16-warp blocks get one block per SM and more
// registers.  The autotuner picks one shape per batch.
template <int W>
struct BShape {
  static constexpr int kThreads = 32 * W;
  static constexpr int kMinBlocks = W == 4 ? 6 : W == 8 ? 3 : 1;
};

// matrix that owns global tile g: last j with toff[j] <= g
__device__ __forceinline__ int owner_item(const int64_t *toff, int count, int64_t g) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(toff + mid) <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// W warps per block; dynamic shared memory: per warp the row pointers of
// its tile, rp_cap = largest tile + 8 entries.
template <class Pol, int W>
__global__ void __launch_bounds__(BShape<W>::kThreads, BShape<W>::kMinBlocks)
    batched_csr(const BatchItem *items, const int64_t *toff, int count, const void *const *xs,
                void *const *ys, double *head, double *tail, double alpha, double beta,
                int finish, unsigned comp_mode, int *err, int rp_cap) {
  extern __shared__ __align__(16) int32_t s_rp_all[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *s_rp = s_rp_all + wid * rp_cap;
  const int64_t total = __ldg(toff + count);
  int j = 0;
  for (int64_t g = int64_t(blockIdx.x) * W + wid; g < total; g += int64_t(gridDim.x) * W) {
    // a warp's tiles increase: step forward from the previous owner, and
    // search only when the tile is more than a few matrices ahead
    int step = 0;
    while (step < 4 && j + 1 < count && __ldg(toff + j + 1) <= g) {
      ++j;
      ++step;
    }
    if (step == 4) j = owner_item(toff, count, g);
    const BatchItem it = items[j];
    const int64_t base = __ldg(toff + j);
    const int b = static_cast<int>(g - base);
    CsrArgs<Pol> a;
    a.part_toff = nullptr;
    a.row_ptr = it.row_ptr;
    a.col_idx = it.col_idx;
    a.val = static_cast<const typename Pol::V *>(it.val);
    a.x = static_cast<const typename Pol::X *>(xs[j]);
    a.y = static_cast<typename Pol::X *>(ys[j]);
    a.alpha = alpha;
    a.beta = beta;
    a.finish = finish;
    a.tile_row = it.tile_row;
    a.tile_k = it.tile_k;
    a.head = head + base;
    a.tail = tail + base;
    a.m = it.m;
    a.comp_mode = comp_mode;
    a.err = err;
    const int32_t r0 = __ldg(a.tile_row + b), k0 = __ldg(a.tile_k + b);
    const int32_t r1 = __ldg(a.tile_row + b + 1), k1 = __ldg(a.tile_k + b + 1);
    const int32_t rend = min(r1 + 2, a.m + 1);
    for (int32_t r = r0 + lane; r < rend; r += 32) s_rp[r - r0] = __ldg(a.row_ptr + r);
    __syncwarp();
    csr_tile_compute<Pol>(a, b, r0, k0, r1, k1, s_rp, Seg<int32_t>{a.col_idx, 0},
                          Seg<typename Pol::V>{a.val, 0}, it.nnz, GlobalSrc{});
    __syncwarp();
  }
}

template <class X>
__global__ void batched_fixup(const BatchItem *items, const int64_t *toff, int count,
                              void *const *ys, const double *head, const double *tail,
                              double alpha, double beta) {
  grid_dependency_wait();
  const int64_t total = __ldg(toff + count);
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < total;
       g += int64_t(gridDim.x) * blockDim.x) {
    const int j = owner_item(toff, count, g);
    const int64_t base = __ldg(toff + j);
    const int T = static_cast<int>(__ldg(toff + j + 1) - base);
    const BatchItem it = items[j];
    struct View {
      const int32_t *tile_row, *tile_k, *row_ptr;
      __device__ void row_flag(int b, int32_t &r, bool &f) const {
        r = __ldg(tile_row + b);
        f = __ldg(row_ptr + r) < __ldg(tile_k + b);
      }
    } v{it.tile_row, it.tile_k, it.row_ptr};
    fixup_tile(v, T, static_cast<int>(g - base), head + base, tail + base,
               static_cast<X *>(ys[j]), alpha, beta);
  }
}

static int bucket_of(int64_t nnz) {
  int b = 0;
  while (b + 1 < MSREP_TUNE_BUCKETS && (int64_t(1) << (b + 1)) <= nnz) ++b;
  return b;
}

static void tuned(const msrep_tune_table *t, int64_t nnz, int32_t *tile, int32_t *np) {
  const int b = bucket_of(nnz);
  *tile = effective_tile(t ? t->tile[b] : 0);
  const int64_t pn = t ? t->part_nnz[b] : 0;
  *np = pn > 0 ? static_cast<int32_t>(std::max<int64_t>(1, ceil_div(nnz, pn))) : 1;
}

// layout of one matrix's partition + plan inside the batch buffer
struct ItemLayout {
  int32_t np, tile;
  size_t off_meta, off_flag, off_plan, plan_bytes, end;
};

static ItemLayout item_layout(const msrep_matrix *A, const msrep_tune_table *t, size_t at) {
  ItemLayout L;
  tuned(t, A->nnz, &L.tile, &L.np);
  L.off_meta = at;
  size_t o = align256(at + 4 * sizeof(int32_t) * size_t(L.np));
  L.off_flag = o;
  o = align256(o + size_t(L.np));
  L.off_plan = o;
  L.plan_bytes = plan_layout(A->m, A->nnz, L.np, L.tile).bytes;
  L.end = align256(o + L.plan_bytes);
  return L;
}

static msrep_status check_batch_inputs(int32_t count, const msrep_matrix *As) {
  if (count < 1 || !As) return fail(MSREP_ERR_INVALID_ARG, "empty batch");
  for (int32_t j = 0; j < count; ++j) {
    MSREP_TRY(check_matrix(As + j));
    if (As[j].fmt != MSREP_CSR) return fail(MSREP_ERR_INVALID_ARG, "batch matrix %d is not CSR", j);
    if (As[j].val_dtype != As[0].val_dtype)
      return fail(MSREP_ERR_INVALID_ARG, "batch matrices must share one value type");
  }
  return MSREP_OK;
}

static size_t batch_bytes(int32_t count, const msrep_matrix *As, const msrep_tune_table *t,
                          std::vector<ItemLayout> *lay, size_t *items_off, size_t *toff_off) {
  size_t at = 0;
  for (int32_t j = 0; j < count; ++j) {
    ItemLayout L = item_layout(As + j, t, at);
    at = L.end;
    if (lay) lay->push_back(L);
  }
  *items_off = at;
  at = align256(at + sizeof(BatchItem) * size_t(count));
  *toff_off = at;
  at = align256(at + sizeof(int64_t) * size_t(count + 1));
  return at;
}

msrep_status launch_batched(const BatchItem *items, const int64_t *toff, int count,
                            int64_t total_tiles, int32_t val_dtype, const void *const *xs,
                            void *const *ys, double *head, double *tail, double alpha,
                            double beta, unsigned flags, cudaStream_t st, int cta_threads,
                            int max_tile) {
  int *err = kernel_err_ptr();
  if (!err) return fail(MSREP_ERR_CUDA, "cannot resolve the device error word");
  if (cta_threads != 128 && cta_threads != 256 && cta_threads != 512)
    return fail(MSREP_ERR_INVALID_ARG, "cta_threads must be 128, 256 or 512 (got %d)",
                cta_threads);
  if (!tile_supported(max_tile))
    return fail(MSREP_ERR_INVALID_ARG, "unsupported largest tile %d", max_tile);
  const int finish = finish_mode(alpha, beta);
  const unsigned comp = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  const int64_t T = total_tiles;
  if (T == 0) return MSREP_OK;
  const int sms = sm_count();
  const int rp_cap = max_tile + 8;
  auto launch = [&](auto kern, auto fix, int warps, int min_blocks) -> msrep_status {
    const int threads = 32 * warps;
    const size_t smem = sizeof(int32_t) * size_t(warps) * rp_cap;
    // The kernel's attributes are set once per device for its largest
    // buffer (tile 1024): the dynamic shared-memory limit, and the smallest
    // carveout that holds the blocks it asks for.  (Setting the limit to a
    // launch's own size would lower it for later launches with larger
    // tiles.)  Resident blocks are then known per shared-memory size.
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> prepared;
    static std::map<std::tuple<int, const void *, size_t>, int> blocks;
    int dev = 0, nb = 1;
    MSREP_CUDA_TRY(cudaGetDevice(&dev));
    {
      std::lock_guard<std::mutex> lk(mu);
      const void *kp = reinterpret_cast<const void *>(kern);
      if (!prepared[std::make_pair(dev, kp)]) {
        const size_t most = sizeof(int32_t) * size_t(warps) * (1024 + 8);
        MSREP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(most)));
        MSREP_TRY(set_min_carveout(kp, most, min_blocks));
        prepared[std::make_pair(dev, kp)] = true;
      }
      const auto key = std::make_tuple(dev, kp, smem);
      auto it = blocks.find(key);
      if (it == blocks.end()) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) !=
                cudaSuccess ||
            nb < 1)
          nb = 1;
        blocks[key] = nb;
      } else {
        nb = it->second;
      }
    }
    const int64_t grid =
        std::max<int64_t>(1, std::min<int64_t>(ceil_div(T, warps), int64_t(nb) * sms));
    kern<<<static_cast<int>(grid), threads, smem, st>>>(items, toff, count, xs, ys, head, tail,
                                                        alpha, beta, finish, comp, err, rp_cap);
    MSREP_CUDA_TRY(cudaGetLastError());
    const int64_t fg = std::max<int64_t>(1, std::min<int64_t>(ceil_div(T, 256), 4 * sms));
    MSREP_TRY(launch_dependent(fix, fg, 256, st, 0, items, toff, count, ys, head, tail, alpha,
                               beta));
    return MSREP_OK;
  };
  auto shaped = [&](auto pol, auto fix) -> msrep_status {
    using Pol = decltype(pol);
    if (cta_threads == 128) return launch(batched_csr<Pol, 4>, fix, 4, BShape<4>::kMinBlocks);
    if (cta_threads == 512) return launch(batched_csr<Pol, 16>, fix, 16, BShape<16>::kMinBlocks);
    return launch(batched_csr<Pol, 8>, fix, 8, BShape<8>::kMinBlocks);
  };
  switch (val_dtype) {
    case MSREP_F64: return shaped(PolF64{}, batched_fixup<double>);
    case MSREP_F32: return shaped(PolF32<float>{}, batched_fixup<float>);
    default: return shaped(PolF32<bf16_t>{}, batched_fixup<float>);
  }
}

}  // namespace msrep

using namespace msrep;

extern "C" {

msrep_status msrep_tune_default(msrep_tune_table *t) {
  if (!t) return fail(MSREP_ERR_INVALID_ARG, "table is NULL");
  for (int b = 0; b < MSREP_TUNE_BUCKETS; ++b) {
    t->tile[b] = kDefaultTile;
    t->part_nnz[b] = 0;
  }
  t->cta_threads = 256;
  t->reserved = 0;
  return ok();
}

msrep_status msrep_batch_plan_size(int32_t count, const msrep_matrix *As,
                                   const msrep_tune_table *tune, int64_t *dev_bytes) {
  MSREP_TRY(check_batch_inputs(count, As));
  if (!dev_bytes) return fail(MSREP_ERR_INVALID_ARG, "dev_bytes is NULL");
  size_t io, to;
  *dev_bytes = static_cast<int64_t>(batch_bytes(count, As, tune, nullptr, &io, &to));
  return ok();
}

msrep_status msrep_partition_csr(const msrep_matrix *A, msrep_partition *part, unsigned flags,
                                 void *stream);

msrep_status msrep_batch_prepare(int32_t count, const msrep_matrix *As,
                                 const msrep_tune_table *tune, void *dev, int64_t dev_bytes,
                                 msrep_batch *out, void *stream) {
  MSREP_TRY(check_batch_inputs(count, As));
  if (!dev || !out) return fail(MSREP_ERR_INVALID_ARG, "dev or out is NULL");
  if (tune && tune->cta_threads != 0 && tune->cta_threads != 128 && tune->cta_threads != 256 &&
      tune->cta_threads != 512)
    return fail(MSREP_ERR_INVALID_ARG, "cta_threads must be 0, 128, 256 or 512");
  if (reinterpret_cast<uintptr_t>(dev) & 255)
    return fail(MSREP_ERR_INVALID_ARG, "dev must be 256-byte aligned");
  std::vector<ItemLayout> lay;
  size_t items_off, toff_off;
  const size_t need = batch_bytes(count, As, tune, &lay, &items_off, &toff_off);
  if (dev_bytes < static_cast<int64_t>(need))
    return fail(MSREP_ERR_WORKSPACE, "batch buffer has %lld bytes, needs %zu",
                (long long)dev_bytes, need);
  cudaStream_t st = as_stream(stream);
  char *base = static_cast<char *>(dev);
  std::vector<const int32_t *> ntile_ptr(count);
  std::vector<BatchItem> items(count);
  for (int32_t j = 0; j < count; ++j) {
    const ItemLayout &L = lay[j];
    msrep_partition p{};
    p.np = L.np;
    p.tile = L.tile;
    int32_t *meta = reinterpret_cast<int32_t *>(base + L.off_meta);
    p.start_idx = meta;
    p.end_idx = meta + L.np;
    p.start_major = meta + 2 * L.np;
    p.end_major = meta + 3 * L.np;
    p.start_flag = reinterpret_cast<uint8_t *>(base + L.off_flag);
    p.plan = base + L.off_plan;
    p.plan_bytes = static_cast<int64_t>(L.plan_bytes);
    MSREP_TRY(msrep_partition_csr(As + j, &p, 0, stream));
    const PlanLayout PL = plan_layout(As[j].m, As[j].nnz, L.np, L.tile);
    const char *plan = base + L.off_plan;
    ntile_ptr[j] = reinterpret_cast<const int32_t *>(plan + PL.off_toff) + L.np;
    items[j] = BatchItem{As[j].ptr, As[j].idx, As[j].val,
                         reinterpret_cast<const int32_t *>(plan + PL.off_row),
                         reinterpret_cast<const int32_t *>(plan + PL.off_k), As[j].m, As[j].n,
                         As[j].nnz, 1, 0};
  }
  std::vector<int32_t> nt(count);
  for (int32_t j = 0; j < count; ++j)
    MSREP_CUDA_TRY(cudaMemcpyAsync(&nt[j], ntile_ptr[j], sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MSREP_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int64_t> toff(count + 1, 0);
  for (int32_t j = 0; j < count; ++j) toff[j + 1] = toff[j] + nt[j];
  MSREP_CUDA_TRY(cudaMemcpyAsync(base + items_off, items.data(), sizeof(BatchItem) * count,
                                 cudaMemcpyHostToDevice, st));
  MSREP_CUDA_TRY(cudaMemcpyAsync(base + toff_off, toff.data(), sizeof(int64_t) * (count + 1),
                                 cudaMemcpyHostToDevice, st));
  MSREP_CUDA_TRY(cudaStreamSynchronize(st));
  out->count = count;
  out->val_dtype = As[0].val_dtype;
  out->total_tiles = toff[count];
  out->ws_bytes = static_cast<int64_t>(2 * align256(sizeof(double) * std::max<int64_t>(toff[count], 1)));
  out->dev = dev;
  out->dev_bytes = dev_bytes;
  out->items_off = static_cast<int64_t>(items_off);
  out->toff_off = static_cast<int64_t>(toff_off);
  out->cta_threads = tune && tune->cta_threads ? tune->cta_threads : 256;
  int32_t mt = 0;
  for (const ItemLayout &L : lay) mt = std::max(mt, L.tile);
  out->max_tile = mt;
  return ok();
}

msrep_status msrep_spmv_batched(const msrep_batch *B, const void *const *xs, void *const *ys,
                                double alpha, double beta, unsigned flags, void *workspace,
                                void *stream) {
  if (!B || !B->dev || B->count < 1) return fail(MSREP_ERR_INVALID_ARG, "batch not prepared");
  if (!xs || !ys || !workspace) return fail(MSREP_ERR_INVALID_ARG, "xs, ys or workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) & 15)
    return fail(MSREP_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  const char *base = static_cast<const char *>(B->dev);
  double *head = static_cast<double *>(workspace);
  double *tail = reinterpret_cast<double *>(static_cast<char *>(workspace) +
                                            align256(sizeof(double) * std::max<int64_t>(B->total_tiles, 1)));
  MSREP_TRY(launch_batched(reinterpret_cast<const BatchItem *>(base + B->items_off),
                           reinterpret_cast<const int64_t *>(base + B->toff_off), B->count,
                           B->total_tiles, B->val_dtype, xs, ys, head, tail, alpha, beta, flags,
                           as_stream(stream), B->cta_threads ? B->cta_threads : 256,
                           B->max_tile ? B->max_tile : 1024));
  return ok();
}

msrep_status msrep_spmv_workspace_size(const msrep_matrix *A, const msrep_partition *part,
                                       size_t *bytes);
msrep_status msrep_spmv(const msrep_matrix *A, const msrep_partition *part, double alpha,
                        const void *x, double beta, void *y, int32_t xy_dtype, unsigned flags,
                        void *workspace, void *stream);

static const int32_t kTuneTiles[] = {256, 512, 1024};
static const int64_t kTuneParts[] = {0, int64_t(1) << 14, int64_t(1) << 18};

// scratch for one candidate trial: partition + plan + workspace of the
// largest matrix under the smallest tile / most partitions
static size_t trial_bytes(const msrep_matrix *A) {
  size_t worst = 0;
  for (int32_t tile : kTuneTiles)
    for (int64_t pn : kTuneParts) {
      const int32_t np = pn > 0 ? static_cast<int32_t>(std::max<int64_t>(1, ceil_div(A->nnz, pn))) : 1;
      size_t b = align256(4 * sizeof(int32_t) * np) + align256(np) +
                 align256(plan_layout(A->m, A->nnz, np, tile).bytes);
      msrep_partition p{};
      p.np = np;
      p.tile = tile;
      size_t ws = 0;
      msrep_spmv_workspace_size(A, &p, &ws);
      worst = std::max(worst, b + align256(ws));
    }
  return worst;
}

// The table that makes a batch's plan and workspace largest: the smallest
// tile and the most partitions of the autotuner's candidates.
static msrep_tune_table largest_table() {
  msrep_tune_table t;
  for (int b = 0; b < MSREP_TUNE_BUCKETS; ++b) {
    t.tile[b] = kTuneTiles[0];
    t.part_nnz[b] = kTuneParts[1];
  }
  t.cta_threads = 256;
  t.reserved = 0;
  return t;
}

// Scratch of the autotuner's thread-block phase: the prepared batch (at a
// 256-byte boundary), the device arrays of x and y pointers and the
// batched workspace, under the largest table.
static size_t cta_phase_bytes(int32_t count, const msrep_matrix *As) {
  const msrep_tune_table t = largest_table();
  size_t io, to;
  const size_t bb = batch_bytes(count, As, &t, nullptr, &io, &to);
  int64_t tiles = 0;
  for (int32_t j = 0; j < count; ++j) {
    int32_t tile, np;
    tuned(&t, As[j].nnz, &tile, &np);
    tiles += plan_layout(As[j].m, As[j].nnz, np, tile).tmax;
  }
  return 256 + align256(bb) + 2 * align256(sizeof(void *) * size_t(count)) +
         2 * align256(sizeof(double) * size_t(std::max<int64_t>(tiles, 1)));
}

msrep_status msrep_autotune_scratch_size(int32_t count, const msrep_matrix *As, int64_t *bytes) {
  MSREP_TRY(check_batch_inputs(count, As));
  if (!bytes) return fail(MSREP_ERR_INVALID_ARG, "bytes is NULL");
  size_t w = 0;
  for (int32_t j = 0; j < count; ++j) w = std::max(w, trial_bytes(As + j));
  w = std::max(w, cta_phase_bytes(count, As));
  *bytes = static_cast<int64_t>(w);
  return ok();
}

msrep_status msrep_autotune(int32_t count, const msrep_matrix *As, const void *const *xs,
                            void *const *ys, void *scratch, int64_t scratch_bytes,
                            msrep_tune_table *out, void *stream) {
  MSREP_TRY(check_batch_inputs(count, As));
  if (!xs || !ys || !scratch || !out) return fail(MSREP_ERR_INVALID_ARG, "NULL argument");
  int64_t need = 0;
  MSREP_TRY(msrep_autotune_scratch_size(count, As, &need));
  if (scratch_bytes < need) return fail(MSREP_ERR_WORKSPACE, "autotune scratch too small");
  MSREP_TRY(msrep_tune_default(out));
  cudaStream_t st = as_stream(stream);
  const int32_t xy = As[0].val_dtype == MSREP_F64 ? MSREP_F64 : MSREP_F32;
  // matrices of each bucket, largest first
  std::vector<std::vector<int32_t>> by_bucket(MSREP_TUNE_BUCKETS);
  for (int32_t j = 0; j < count; ++j) by_bucket[bucket_of(As[j].nnz)].push_back(j);
  cudaEvent_t e0, e1;
  MSREP_CUDA_TRY(cudaEventCreate(&e0));
  MSREP_CUDA_TRY(cudaEventCreate(&e1));
  char *base = static_cast<char *>(scratch);
  msrep_status status = MSREP_OK;
  for (int bkt = 0; bkt < MSREP_TUNE_BUCKETS && status == MSREP_OK; ++bkt) {
    auto &v = by_bucket[bkt];
    if (v.empty()) continue;
    std::sort(v.begin(), v.end(), [&](int32_t a, int32_t b) { return As[a].nnz > As[b].nnz; });
    const size_t reps = std::min<size_t>(3, v.size());
    float best = INFINITY;
    for (int32_t tile : kTuneTiles)
      for (int64_t pn : kTuneParts) {
        float total = 0.f;
        for (size_t q = 0; q < reps && status == MSREP_OK; ++q) {
          const msrep_matrix *A = As + v[q];
          const int32_t np =
              pn > 0 ? static_cast<int32_t>(std::max<int64_t>(1, ceil_div(A->nnz, pn))) : 1;
          msrep_partition p{};
          p.np = np;
          p.tile = tile;
          int32_t *meta = reinterpret_cast<int32_t *>(base);
          p.start_idx = meta;
          p.end_idx = meta + np;
          p.start_major = meta + 2 * np;
          p.end_major = meta + 3 * np;
          size_t o = align256(4 * sizeof(int32_t) * np);
          p.start_flag = reinterpret_cast<uint8_t *>(base + o);
          o = align256(o + np);
          p.plan = base + o;
          p.plan_bytes = static_cast<int64_t>(plan_layout(A->m, A->nnz, np, tile).bytes);
          o = align256(o + p.plan_bytes);
          status = msrep_partition_csr(A, &p, 0, stream);
          if (status != MSREP_OK) break;
          for (int rep = 0; rep < 4 && status == MSREP_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            status = msrep_spmv(A, &p, 1.0, xs[v[q]], 0.0, ys[v[q]], xy, 0, base + o, stream);
          }
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            status = fail(MSREP_ERR_CUDA, "autotune timing failed");
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          total += ms;
        }
        if (status == MSREP_OK && total < best) {
          best = total;
          out->tile[bkt] = tile;
          out->part_nnz[bkt] = pn;
        }
      }
  }
  // Thread-block shape: one per batch, since one launch runs every matrix.
  // The whole batch is prepared with the table chosen above and the
  // batched launch timed with each shape.
  if (status == MSREP_OK) {
    char *b0 = reinterpret_cast<char *>(align256(reinterpret_cast<uintptr_t>(base)));
    size_t io, to;
    const size_t bb = batch_bytes(count, As, out, nullptr, &io, &to);
    msrep_batch B{};
    status = msrep_batch_prepare(count, As, out, b0, static_cast<int64_t>(bb), &B, stream);
    char *p = b0 + align256(bb);
    void **dxs = reinterpret_cast<void **>(p);
    p += align256(sizeof(void *) * size_t(count));
    void **dys = reinterpret_cast<void **>(p);
    p += align256(sizeof(void *) * size_t(count));
    if (status == MSREP_OK &&
        (cudaMemcpyAsync(dxs, xs, sizeof(void *) * count, cudaMemcpyHostToDevice, st) !=
             cudaSuccess ||
         cudaMemcpyAsync(dys, ys, sizeof(void *) * count, cudaMemcpyHostToDevice, st) !=
             cudaSuccess))
      status = fail(MSREP_ERR_CUDA, "autotune: copying the vector pointers failed");
    float best_ms = INFINITY;
    for (int cta : {128, 256, 512}) {
      if (status != MSREP_OK) break;
      B.cta_threads = cta;
      for (int rep = 0; rep < 4 && status == MSREP_OK; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        status = msrep_spmv_batched(&B, dxs, dys, 1.0, 0.0, 0, p, stream);
      }
      if (status != MSREP_OK) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        status = fail(MSREP_ERR_CUDA, "autotune timing failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        out->cta_threads = cta;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != MSREP_OK) return status;
  return ok();
}

}  // extern "C"
