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

constexpr int kKWarps = 8;
constexpr int kKThreads = 32 * kKWarps;
constexpr int kKMaxIPT = 32;  // row-pointer stage sized for the largest tile (1024)

int spmm_width(int k) { return k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : 8; }

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
__global__ void __launch_bounds__(kKThreads, 2) csr_spmm_direct(SpmmArgs<Pol, KP> a,
                                                                const int32_t *n_tiles,
                                                                int64_t nnz) {
  __shared__ int32_t s_rp[kKWarps][32 * kKMaxIPT + 8];
  extern __shared__ __align__(16) unsigned char s_stage[];
  grid_dependency_wait();
  const int T = *n_tiles, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *stage = s_stage + threadIdx.x * SpmmStage<Pol, KP>::LANE;
  for (int b = blockIdx.x * kKWarps + wid; b < T; b += gridDim.x * kKWarps) {
    const int32_t r0 = __ldg(a.tile_row + b), k0 = __ldg(a.tile_k + b);
    const int32_t r1 = __ldg(a.tile_row + b + 1), k1 = __ldg(a.tile_k + b + 1);
    const int32_t rend = min(r1 + 2, a.m + 1);
    for (int32_t r = r0 + lane; r < rend; r += 32) s_rp[wid][r - r0] = __ldg(a.row_ptr + r);
    __syncwarp();
    csr_tile_compute_k<Pol, KP>(a, b, r0, k0, r1, k1, s_rp[wid], nnz, stage);
    __syncwarp();
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
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, kKThreads, dyn) != cudaSuccess ||
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
  a.m = A->m;
  a.comp_mode = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  const int32_t *n_tiles = reinterpret_cast<const int32_t *>(plan + L.off_toff) + p->np;
  int nb = 1;
  constexpr size_t dyn = size_t(kKWarps) * SpmmStage<Pol, KP>::WARP;
  MSREP_TRY(blocks_of(csr_spmm_direct<Pol, KP>, dyn, 2, &nb));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.tmax, kKWarps),
                                                             int64_t(nb) * sm_count()));
  MSREP_TRY(launch_dependent(csr_spmm_direct<Pol, KP>, grid, kKThreads, st, dyn, a, n_tiles,
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

template <class Pol>
__global__ void __launch_bounds__(kKThreads, 2) batched_spmm(const BatchItem *items,
                                                             const int64_t *toff, int count,
                                                             const void *const *xs,
                                                             void *const *ys, double *head,
                                                             double *tail, unsigned comp_mode) {
  constexpr int KP = kBatchWidth;
  __shared__ int32_t s_rp[kKWarps][32 * kKMaxIPT + 8];
  extern __shared__ __align__(16) unsigned char s_stage[];
  grid_dependency_wait();
  unsigned char *stage = s_stage + threadIdx.x * SpmmStage<Pol, KP>::LANE;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = __ldg(toff + count);
  int j = 0;
  for (int64_t g = int64_t(blockIdx.x) * kKWarps + wid; g < total;
       g += int64_t(gridDim.x) * kKWarps) {
    int step = 0;
    while (step < 4 && j + 1 < count && __ldg(toff + j + 1) <= g) {
      ++j;
      ++step;
    }
    if (step == 4) j = owner_item_k(toff, count, g);
    const BatchItem it = items[j];
    const int64_t base = __ldg(toff + j);
    const int b = static_cast<int>(g - base);
    SpmmArgs<Pol, KP> a;
    a.row_ptr = it.row_ptr;
    a.col_idx = it.col_idx;
    a.val = static_cast<const typename Pol::V *>(it.val);
    a.xt = static_cast<const typename Pol::X *>(xs[j]);
    a.y = static_cast<typename Pol::X *>(ys[j]);
    a.ldy = it.m;
    a.k = it.k;
    a.alpha = 1.0;
    a.beta = 0.0;
    a.finish = kFinishCopy;
    a.tile_row = it.tile_row;
    a.tile_k = it.tile_k;
    a.head = head + base * KP;
    a.tail = tail + base * KP;
    a.m = it.m;
    a.comp_mode = comp_mode;
    const int32_t r0 = __ldg(a.tile_row + b), k0 = __ldg(a.tile_k + b);
    const int32_t r1 = __ldg(a.tile_row + b + 1), k1 = __ldg(a.tile_k + b + 1);
    const int32_t rend = min(r1 + 2, a.m + 1);
    for (int32_t r = r0 + lane; r < rend; r += 32) s_rp[wid][r - r0] = __ldg(a.row_ptr + r);
    __syncwarp();
    csr_tile_compute_k<Pol, KP>(a, b, r0, k0, r1, k1, s_rp[wid], it.nnz, stage);
    __syncwarp();
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

// blockIdx.y = item (grid-stride), blocks along x share the item's columns
template <class X>
__global__ void interleave_batch(const BatchItem *items, int count, const void *const *xin,
                                 void *const *xt) {
  for (int j = blockIdx.y; j < count; j += gridDim.y) {
    const BatchItem it = items[j];
    const X *x = static_cast<const X *>(xin[j]);
    X *o = static_cast<X *>(xt[j]);
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < it.n;
         c += int64_t(gridDim.x) * blockDim.x)
      interleave_column<X, kBatchWidth>(x, it.n, it.k, c, o);
  }
}

msrep_status launch_batched_k(const BatchItem *items, const int64_t *toff, int count,
                              int64_t total_tiles, const void *const *xin, void *const *xt,
                              void *const *ys, double *head, double *tail, unsigned flags,
                              cudaStream_t st) {
  if (count == 0) return MSREP_OK;
  const int sms = sm_count();
  interleave_batch<float><<<dim3(64, std::min(count, 1024)), 256, 0, st>>>(items, count, xin, xt);
  MSREP_CUDA_TRY(cudaGetLastError());
  if (total_tiles == 0) return MSREP_OK;
  const unsigned comp = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  int nb = 1;
  constexpr size_t dyn = size_t(kKWarps) * SpmmStage<PolF32<float>, kBatchWidth>::WARP;
  MSREP_TRY(blocks_of(batched_spmm<PolF32<float>>, dyn, 2, &nb));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(total_tiles, kKWarps),
                                                             int64_t(nb) * sms));
  MSREP_TRY(launch_dependent(batched_spmm<PolF32<float>>, grid, kKThreads, st, dyn, items, toff,
                             count, static_cast<const void *const *>(xt), ys, head, tail, comp));
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
