// k right-hand sides (msrep_spmm, CSR): Y = alpha * A * X + beta * Y for
// up to eight vectors at once, and its batched form used by the server for
// requests that carry several x vectors.  The tile kernels are in
// spmm_core.cuh.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "batch.cuh"
#include "common.cuh"
#include "spmm_core.cuh"

namespace msrep {

msrep_status check_matrix(const msrep_matrix *A);
int32_t effective_tile(int32_t tile);

// xt[c * KP + j] = x[j * ldx + c] for j < k, 0 for k <= j < KP; a thread
// per column: coalesced reads of each vector, one KP-wide write
template <class X, int KP>
__device__ __forceinline__ void interleave_column(const X *x, int64_t ldx, int k, int64_t c,
                                                  X *xt) {
  X r[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) r[j] = j < k ? x[j * ldx + c] : X(0);
#pragma unroll
  for (int j = 0; j < KP; ++j) xt[c * KP + j] = r[j];
}

template <class X, int KP>
__global__ void interleave_x(const X *x, int64_t ldx, int k, int64_t n, X *xt) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < n;
       c += int64_t(gridDim.x) * blockDim.x)
    interleave_column<X, KP>(x, ldx, k, c, xt);
}

template <class Pol, int KP>
__global__ void __launch_bounds__(kKvThreads) csr_spmm_direct(SpmmArgs<Pol, KP> a,
                                                              const int32_t *n_tiles,
                                                              int64_t nnz) {
  using Sh = KvShape<typename Pol::X, KP>;
  __shared__ KvSmem<typename Pol::Acc, Sh::G> sm;
  grid_dependency_wait();
  const int T = *n_tiles, ts = threadIdx.x / Sh::GT;
  // alpha = 1, beta = 0 finishes rows by a copy, chosen at compile time
  if (a.finish == kFinishCopy) {
    for (int b = blockIdx.x * Sh::G + ts; b < T; b += gridDim.x * Sh::G)
      kv_tile<Pol, KP, Sh::G, true>(a, b, nnz, sm, ts);
  } else {
    for (int b = blockIdx.x * Sh::G + ts; b < T; b += gridDim.x * Sh::G)
      kv_tile<Pol, KP, Sh::G>(a, b, nnz, sm, ts);
  }
}

template <class X, int KP>
__global__ void fixup_spmm(CsrTileView v, const double *head, const double *tail, X *y,
                           int64_t ldy, int k, double alpha, double beta) {
  grid_dependency_wait();
  const int T = v.count();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < T; b += gridDim.x * blockDim.x)
    fixup_tile_k<X, KP>(v, T, b, head, tail, y, ldy, k, alpha, beta);
}

// resident blocks of a kernel per device (after the dynamic shared-memory
// opt-in and the smallest carveout for `want` blocks)
template <class K>
static msrep_status blocks_of(K kern, size_t dyn, int want, int *nb) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> cache;
  int dev = 0;
  MSREP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, reinterpret_cast<const void *>(kern));
  auto it = cache.find(key);
  if (it != cache.end()) {
    *nb = it->second;
    return MSREP_OK;
  }
  MSREP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(dyn)));
  MSREP_TRY(set_min_carveout(reinterpret_cast<const void *>(kern), dyn, want));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, kKvThreads, dyn) != cudaSuccess ||
      *nb < 1)
    *nb = 1;
  cache[key] = *nb;
  return MSREP_OK;
}

// workspace: head and tail partials (tiles x KP doubles each), then the
// interleaved X (n x KP values of the x type)
static size_t spmm_ws_layout(int64_t tiles, int kp, int64_t n, size_t xsize, double **head,
                             double **tail, void **xt, void *base) {
  size_t o = 0;
  const size_t oh = o;
  o = align256(o + sizeof(double) * tiles * kp);
  const size_t ot = o;
  o = align256(o + sizeof(double) * tiles * kp);
  const size_t ox = o;
  o = align256(o + xsize * n * kp);
  if (base) {
    char *p = static_cast<char *>(base);
    *head = reinterpret_cast<double *>(p + oh);
    *tail = reinterpret_cast<double *>(p + ot);
    *xt = p + ox;
  }
  return o + 256;
}

template <class Pol, int KP>
static msrep_status run_spmm(const msrep_matrix *A, const msrep_partition *p, int k,
                             double alpha, const void *x, int64_t ldx, double beta, void *y,
                             int64_t ldy, unsigned flags, void *ws, cudaStream_t st) {
  using X = typename Pol::X;
  const int32_t tile = effective_tile(p->tile);
  const PlanLayout L = plan_layout(A->m, A->nnz, p->np, tile);
  const char *plan = static_cast<const char *>(p->plan);
  double *head = nullptr, *tail = nullptr;
  void *xt = nullptr;
  spmm_ws_layout(L.tmax, KP, A->n, sizeof(X), &head, &tail, &xt, ws);
  const int sg = 4 * sm_count();
  if (A->n > 0) {
    interleave_x<X, KP><<<sg, 256, 0, st>>>(static_cast<const X *>(x), ldx, k, A->n,
                                            static_cast<X *>(xt));
    MSREP_CUDA_TRY(cudaGetLastError());
  }
  SpmmArgs<Pol, KP> a;
  a.row_ptr = A->ptr;
  a.col_idx = A->idx;
  a.val = static_cast<const typename Pol::V *>(A->val);
  a.xt = static_cast<const X *>(xt);
  a.y = static_cast<X *>(y);
  a.ldy = ldy;
  a.k = k;
  a.alpha = alpha;
  a.beta = beta;
  a.finish = finish_mode(alpha, beta);
  a.tile_row = reinterpret_cast<const int32_t *>(plan + L.off_row);
  a.tile_k = reinterpret_cast<const int32_t *>(plan + L.off_k);
  a.head = head;
  a.tail = tail;
  a.hs = KP;
  a.m = A->m;
  a.comp_mode = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  const int32_t *n_tiles = reinterpret_cast<const int32_t *>(plan + L.off_toff) + p->np;
  int nb = 1;
  // a tile's walk is a chain of dependent loads, so tiles in flight set the
  // rate: the 1- and 2-vector layouts fit three blocks an SM in registers
  // (R-MAT FP32, 2 vectors: 207 -> 174 us); the wider ones fit two
  MSREP_TRY(blocks_of(csr_spmm_direct<Pol, KP>, 0, KP <= 2 ? 3 : 2, &nb));
  constexpr int G = KvShape<X, KP>::G;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.tmax, G),
                                                             int64_t(nb) * sm_count()));
  MSREP_TRY(launch_dependent(csr_spmm_direct<Pol, KP>, grid, kKvThreads, st, 0, a, n_tiles,
                             A->nnz));
  CsrTileView v{a.tile_row, a.tile_k, A->ptr, n_tiles};
  const int64_t fg = std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.tmax, 256), 4 * sm_count()));
  MSREP_TRY(launch_dependent(fixup_spmm<X, KP>, fg, 256, st, 0, v,
                             static_cast<const double *>(head), static_cast<const double *>(tail),
                             a.y, ldy, k, alpha, beta));
  return MSREP_OK;
}

template <class Pol>
static msrep_status dispatch_k(const msrep_matrix *A, const msrep_partition *p, int k,
                               double alpha, const void *x, int64_t ldx, double beta, void *y,
                               int64_t ldy, unsigned flags, void *ws, cudaStream_t st) {
  switch (spmm_width(k)) {
    case 1: return run_spmm<Pol, 1>(A, p, k, alpha, x, ldx, beta, y, ldy, flags, ws, st);
    case 2: return run_spmm<Pol, 2>(A, p, k, alpha, x, ldx, beta, y, ldy, flags, ws, st);
    case 4: return run_spmm<Pol, 4>(A, p, k, alpha, x, ldx, beta, y, ldy, flags, ws, st);
    default: return run_spmm<Pol, 8>(A, p, k, alpha, x, ldx, beta, y, ldy, flags, ws, st);
  }
}

// ---------------------------------------------------------------------------
// batched form (the server): every item is one request, k <= 8 vectors,
// x interleaved with width 8, y as k vectors of m values
// ---------------------------------------------------------------------------

__device__ __forceinline__ int owner_item_k(const int64_t *toff, int count, int64_t g) {
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

// one block work unit of an item: tile u * G + ts by tile group ts
template <class Pol, int KP>
__device__ __forceinline__ void batched_unit(const BatchItem &it, int64_t base, int T, int u,
                                             const void *xt, void *y, double *head,
                                             double *tail, unsigned comp_mode,
                                             KvSmem<typename Pol::Acc, 8> &sm) {
  using Sh = KvShape<typename Pol::X, KP>;
  const int ts = threadIdx.x / Sh::GT, b = u * Sh::G + ts;
  if (b >= T) return;  // uniform over the tile group
  SpmmArgs<Pol, KP> a;
  a.row_ptr = it.row_ptr;
  a.col_idx = it.col_idx;
  a.val = static_cast<const typename Pol::V *>(it.val);
  a.xt = static_cast<const typename Pol::X *>(xt);
  a.y = static_cast<typename Pol::X *>(y);
  a.ldy = it.m;
  a.k = it.k;
  a.alpha = 1.0;
  a.beta = 0.0;
  a.finish = kFinishCopy;
  a.tile_row = it.tile_row;
  a.tile_k = it.tile_k;
  a.head = head + base * kBatchWidth;
  a.tail = tail + base * kBatchWidth;
  a.hs = kBatchWidth;
  a.m = it.m;
  a.comp_mode = comp_mode;
  kv_tile<Pol, KP, 8>(a, b, it.nnz, sm, ts);
}

// Items of 2..8 vectors; item j's x interleaved with width KP_j =
// spmm_width(k_j) and its tiles cut into uoff[j+1] - uoff[j] block work
// units of KvShape<float, KP_j>::G tiles, one unit per block at a time.
// Tile groups run ahead of each other within a layout; where the layout
// (KP) changes from one unit to the next the block synchronises, because
// the two layouts share shared-memory slots differently.
template <class Pol>
__global__ void __launch_bounds__(kKvThreads) batched_spmm(const BatchItem *items,
                                                           const int64_t *toff,
                                                           const int64_t *uoff, int count,
                                                           const void *const *xs,
                                                           void *const *ys, double *head,
                                                           double *tail, unsigned comp_mode) {
  __shared__ KvSmem<typename Pol::Acc, 8> sm;
  grid_dependency_wait();
  const int64_t total = __ldg(uoff + count);
  int j = 0, prev_kp = 0;
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    int step = 0;
    while (step < 4 && j + 1 < count && __ldg(uoff + j + 1) <= g) {
      ++j;
      ++step;
    }
    if (step == 4) j = owner_item_k(uoff, count, g);
    const BatchItem it = items[j];
    const int64_t base = __ldg(toff + j);
    const int T = static_cast<int>(__ldg(toff + j + 1) - base);
    const int u = static_cast<int>(g - __ldg(uoff + j));
    const int kp = spmm_width(it.k);
    if (kp != prev_kp) {
      __syncthreads();
      prev_kp = kp;
    }
    if (kp == 2)
      batched_unit<Pol, 2>(it, base, T, u, xs[j], ys[j], head, tail, comp_mode, sm);
    else if (kp == 4)
      batched_unit<Pol, 4>(it, base, T, u, xs[j], ys[j], head, tail, comp_mode, sm);
    else
      batched_unit<Pol, 8>(it, base, T, u, xs[j], ys[j], head, tail, comp_mode, sm);
  }
}

template <class X>
__global__ void batched_fixup_k(const BatchItem *items, const int64_t *toff, int count,
                                void *const *ys, const double *head, const double *tail) {
  grid_dependency_wait();
  constexpr int KP = kBatchWidth;
  const int64_t total = __ldg(toff + count);
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < total;
       g += int64_t(gridDim.x) * blockDim.x) {
    const int j = owner_item_k(toff, count, g);
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
    fixup_tile_k<X, KP>(v, T, static_cast<int>(g - base), head + base * KP, tail + base * KP,
                        static_cast<X *>(ys[j]), it.m, it.k, 1.0, 0.0);
  }
}

// blockIdx.y = item (grid-stride), blocks along x share the item's
// columns; item j is interleaved with width spmm_width(k_j)
template <class X>
__global__ void interleave_batch(const BatchItem *items, int count, const void *const *xin,
                                 void *const *xt) {
  for (int j = blockIdx.y; j < count; j += gridDim.y) {
    const BatchItem it = items[j];
    const X *x = static_cast<const X *>(xin[j]);
    X *o = static_cast<X *>(xt[j]);
    const int kp = spmm_width(it.k);
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < it.n;
         c += int64_t(gridDim.x) * blockDim.x) {
      if (kp == 2)
        interleave_column<X, 2>(x, it.n, it.k, c, o);
      else if (kp == 4)
        interleave_column<X, 4>(x, it.n, it.k, c, o);
      else
        interleave_column<X, 8>(x, it.n, it.k, c, o);
    }
  }
}

int64_t batched_k_units(int64_t tiles, int k) {
  const int kp = spmm_width(k);
  const int g = kp == 2 ? KvShape<float, 2>::G : kp == 4 ? KvShape<float, 4>::G
                                                         : KvShape<float, 8>::G;
  return (tiles + g - 1) / g;
}

msrep_status launch_batched_k(const BatchItem *items, const int64_t *toff, const int64_t *uoff,
                              int count, int64_t total_tiles, int64_t total_units,
                              const void *const *xin, void *const *xt, void *const *ys,
                              double *head, double *tail, unsigned flags, cudaStream_t st) {
  if (count == 0) return MSREP_OK;
  const int sms = sm_count();
  interleave_batch<float><<<dim3(64, std::min(count, 1024)), 256, 0, st>>>(items, count, xin, xt);
  MSREP_CUDA_TRY(cudaGetLastError());
  if (total_tiles == 0) return MSREP_OK;
  const unsigned comp = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  int nb = 1;
  MSREP_TRY(blocks_of(batched_spmm<PolF32<float>>, 0, 2, &nb));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(total_units, int64_t(nb) * sms));
  MSREP_TRY(launch_dependent(batched_spmm<PolF32<float>>, grid, kKvThreads, st, 0, items, toff,
                             uoff, count, static_cast<const void *const *>(xt), ys, head, tail,
                             comp));
  const int64_t fg = std::max<int64_t>(1, std::min<int64_t>(ceil_div(total_tiles, 256), 4 * sms));
  MSREP_TRY(launch_dependent(batched_fixup_k<float>, fg, 256, st, 0, items, toff, count, ys,
                             static_cast<const double *>(head), static_cast<const double *>(tail)));
  return MSREP_OK;
}

}  // namespace msrep

using namespace msrep;

extern "C" {

msrep_status msrep_spmm_workspace_size(const msrep_matrix *A, const msrep_partition *part,
                                       int32_t k, size_t *bytes) {
  MSREP_TRY(check_matrix(A));
  if (!part || part->np < 1 || !bytes || k < 1)
    return fail(MSREP_ERR_INVALID_ARG, "bad partition, k or bytes pointer");
  if (A->fmt != MSREP_CSR) return fail(MSREP_ERR_INVALID_ARG, "msrep_spmm takes CSR");
  const int32_t tile = effective_tile(part->tile);
  if (!tile_supported(tile)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", part->tile);
  const int64_t tiles = plan_layout(A->m, A->nnz, part->np, tile).tmax;
  const size_t xs = A->val_dtype == MSREP_F64 ? sizeof(double) : sizeof(float);
  // one pass of at most MSREP_SPMM_MAX_K vectors at a time
  *bytes = spmm_ws_layout(tiles, spmm_width(std::min(k, MSREP_SPMM_MAX_K)), A->n, xs, nullptr,
                          nullptr, nullptr, nullptr);
  return ok();
}

msrep_status msrep_spmm(const msrep_matrix *A, const msrep_partition *part, int32_t k,
                        double alpha, const void *x, int64_t ldx, double beta, void *y,
                        int64_t ldy, int32_t xy_dtype, unsigned flags, void *workspace,
                        void *stream) {
  MSREP_TRY(check_matrix(A));
  if (A->fmt != MSREP_CSR) return fail(MSREP_ERR_INVALID_ARG, "msrep_spmm takes CSR");
  if (!part || part->np < 1 || !part->start_idx)
    return fail(MSREP_ERR_INVALID_ARG, "bad partition");
  if (k < 1) return fail(MSREP_ERR_INVALID_ARG, "k = %d < 1", k);
  if (ldx < A->n || ldy < A->m) return fail(MSREP_ERR_INVALID_ARG, "ldx < n or ldy < m");
  const int32_t tile = effective_tile(part->tile);
  if (!tile_supported(tile)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", part->tile);
  const bool f64 = A->val_dtype == MSREP_F64;
  if (f64 != (xy_dtype == MSREP_F64) || (xy_dtype != MSREP_F64 && xy_dtype != MSREP_F32))
    return fail(MSREP_ERR_INVALID_ARG,
                "unsupported types: val %d with x/y %d (F64/F64, F32/F32 or BF16/F32)",
                A->val_dtype, xy_dtype);
  if ((A->m > 0 && !y) || (A->n > 0 && !x)) return fail(MSREP_ERR_INVALID_ARG, "x or y is NULL");
  const int64_t need = static_cast<int64_t>(plan_layout(A->m, A->nnz, part->np, tile).bytes);
  if (!part->plan || part->plan_bytes < need)
    return fail(MSREP_ERR_WORKSPACE, "msrep_spmm needs the partition's tile plan (%lld bytes)",
                (long long)need);
  {
    const uintptr_t mis = reinterpret_cast<uintptr_t>(A->idx) | reinterpret_cast<uintptr_t>(A->val);
    if ((mis & (A->val_dtype == MSREP_BF16 ? 15 : 31)) || (reinterpret_cast<uintptr_t>(A->ptr) & 15))
      return fail(MSREP_ERR_INVALID_ARG,
                  "idx and val must be 32-byte aligned (16-byte for bf16 val), ptr 16-byte");
  }
  if (!workspace) return fail(MSREP_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) & 15)
    return fail(MSREP_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  if (A->m == 0) return ok();
  cudaStream_t st = as_stream(stream);
  // passes of at most MSREP_SPMM_MAX_K vectors, in stream order on the same
  // workspace; each pass reads A once
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  for (int32_t j = 0; j < k; j += MSREP_SPMM_MAX_K) {
    const int32_t kc = std::min(MSREP_SPMM_MAX_K, k - j);
    const void *xj = static_cast<const char *>(x) + size_t(j) * size_t(ldx) * es;
    void *yj = static_cast<char *>(y) + size_t(j) * size_t(ldy) * es;
    switch (A->val_dtype) {
      case MSREP_F64:
        MSREP_TRY(dispatch_k<PolF64>(A, part, kc, alpha, xj, ldx, beta, yj, ldy, flags,
                                     workspace, st));
        break;
      case MSREP_F32:
        MSREP_TRY(dispatch_k<PolF32<float>>(A, part, kc, alpha, xj, ldx, beta, yj, ldy, flags,
                                            workspace, st));
        break;
      default:
        MSREP_TRY(dispatch_k<PolF32<bf16_t>>(A, part, kc, alpha, xj, ldx, beta, yj, ldy, flags,
                                             workspace, st));
        break;
    }
  }
  return ok();
}

}  // extern "C"
