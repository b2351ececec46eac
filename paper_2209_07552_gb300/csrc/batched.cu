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
#include <vector>

#include "common.cuh"
#include "spmv_core.cuh"
#include "batch.cuh"

namespace msrep {

msrep_status check_matrix(const msrep_matrix *A);
int32_t effective_tile(int32_t tile);
int *kernel_err_ptr();


constexpr int kBWarps = 8;
constexpr int kBThreads = 32 * kBWarps;
constexpr int kBMaxIPT = 32;  // the largest tile (1024) fits the warp buffers

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

// Three resident blocks per SM (80 registers a thread), as for the
// single-matrix CSR kernel.
template <class Pol>
__global__ void __launch_bounds__(kBThreads, 3) batched_csr(const BatchItem *items,
                                                         const int64_t *toff, int count,
                                                         const void *const *xs, void *const *ys,
                                                         double *head, double *tail, double alpha,
                                                         double beta, int finish,
                                                         unsigned comp_mode, int *err) {
  __shared__ int32_t s_rp[kBWarps][32 * kBMaxIPT + 8];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = __ldg(toff + count);
  int j = 0;
  for (int64_t g = int64_t(blockIdx.x) * kBWarps + wid; g < total;
       g += int64_t(gridDim.x) * kBWarps) {
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
    for (int32_t r = r0 + lane; r < rend; r += 32) s_rp[wid][r - r0] = __ldg(a.row_ptr + r);
    __syncwarp();
    csr_tile_compute<Pol>(a, b, r0, k0, r1, k1, s_rp[wid], Seg<int32_t>{a.col_idx, 0},
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
                            double beta, unsigned flags, cudaStream_t st) {
  int *err = kernel_err_ptr();
  if (!err) return fail(MSREP_ERR_CUDA, "cannot resolve the device error word");
  const int finish = finish_mode(alpha, beta);
  const unsigned comp = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  const int64_t T = total_tiles;
  if (T == 0) return MSREP_OK;
  const int sms = sm_count();
  auto launch = [&](auto kern, auto fix) -> msrep_status {
    // resident blocks per device, after the smallest carveout for 3 blocks
    static std::mutex mu;
    static std::map<int, int> blocks;
    int dev = 0, nb = 1;
    MSREP_CUDA_TRY(cudaGetDevice(&dev));
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = blocks.find(dev);
      if (it == blocks.end()) {
        MSREP_TRY(set_min_carveout(reinterpret_cast<const void *>(kern), 0, 3));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBThreads, 0) != cudaSuccess || nb < 1)
          nb = 1;
        blocks[dev] = nb;
      } else {
        nb = it->second;
      }
    }
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(T, kBWarps), int64_t(nb) * sms));
    kern<<<static_cast<int>(grid), kBThreads, 0, st>>>(items, toff, count, xs, ys, head, tail,
                                                       alpha, beta, finish, comp, err);
    MSREP_CUDA_TRY(cudaGetLastError());
    const int64_t fg = std::max<int64_t>(1, std::min<int64_t>(ceil_div(T, 256), 4 * sms));
    MSREP_TRY(launch_dependent(fix, fg, 256, st, 0, items, toff, count, ys, head, tail, alpha,
                               beta));
    return MSREP_OK;
  };
  switch (val_dtype) {
    case MSREP_F64: return launch(batched_csr<PolF64>, batched_fixup<double>);
    case MSREP_F32: return launch(batched_csr<PolF32<float>>, batched_fixup<float>);
    default: return launch(batched_csr<PolF32<bf16_t>>, batched_fixup<float>);
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
                           as_stream(stream)));
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

msrep_status msrep_autotune_scratch_size(int32_t count, const msrep_matrix *As, int64_t *bytes) {
  MSREP_TRY(check_batch_inputs(count, As));
  if (!bytes) return fail(MSREP_ERR_INVALID_ARG, "bytes is NULL");
  size_t w = 0;
  for (int32_t j = 0; j < count; ++j) w = std::max(w, trial_bytes(As + j));
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
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != MSREP_OK) return status;
  return ok();
}

}  // extern "C"
