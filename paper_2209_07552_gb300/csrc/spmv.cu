// SpMV over pCSR / pCSC / pCOO partitions on one GPU.
//
// The paper runs one SpMV kernel per partition, each on its own GPU, and
// merges the partial results of rows that partition boundaries split
// (Alg. 3, 5, 7; Sec. 4.3).  Here each partition is cut further into
// thread-block tiles (the two-level split of Sec. 4.2, with thread blocks in
// place of GPUs); tiles never straddle a partition boundary.
//
//  CSR  merge-path tiles (rows + nonzeros per tile bounded), per-thread
//       sequential reduction, block-wide segmented scan, then an
//       atomic-free fix-up kernel that merges split rows in tile order.
//  COO  nonzero tiles (Alg. 2's split inside each partition), the same
//       segmented reduction keyed by row_idx, the same fix-up.
//  CSC  merge-path tiles over col_ptr; each nonzero is scattered into y with
//       an atomic add (the column merge of Alg. 5 done in place).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "spmv_core.cuh"

namespace msrep {

msrep_status check_matrix(const msrep_matrix *A);
int32_t effective_tile(int32_t tile);

// ---------------------------------------------------------------------------
// single-matrix kernels: a grid of (resident blocks x SMs) walks the tiles
// ---------------------------------------------------------------------------

constexpr int kWarps = 8;  // warps per block; each warp owns whole tiles
constexpr int kThreads = 32 * kWarps;

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads, 4) csr_tiles(CsrArgs<Pol> a, const int32_t *n_tiles,
                                                          int64_t nnz) {
  __shared__ int32_t s_end[kWarps][32 * IPT];
  const int T = *n_tiles, wid = threadIdx.x >> 5;
  for (int b = blockIdx.x * kWarps + wid; b < T; b += gridDim.x * kWarps)
    csr_tile<Pol, IPT>(a, b, s_end[wid], nnz);
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads, 4) coo_tiles(CooArgs<Pol> a) {
  const int T = a.np * a.G, wid = threadIdx.x >> 5;
  for (int b = blockIdx.x * kWarps + wid; b < T; b += gridDim.x * kWarps)
    coo_tile<Pol, IPT>(a, b);
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads, 4) csc_tiles(CscArgs<Pol> a, const int32_t *n_tiles,
                                                          int64_t nnz) {
  __shared__ int32_t s_end[kWarps][32 * IPT];
  const int T = *n_tiles, wid = threadIdx.x >> 5;
  for (int b = blockIdx.x * kWarps + wid; b < T; b += gridDim.x * kWarps)
    csc_tile<Pol, IPT>(a, b, s_end[wid], nnz);
}

// ---------------------------------------------------------------------------
// fix-up: rows split between tiles, merged in tile (= partition) order
// ---------------------------------------------------------------------------

struct CsrTileView {
  const int32_t *tile_row, *tile_k, *row_ptr, *n_tiles;
  __device__ int count() const { return *n_tiles; }
  __device__ void row_flag(int b, int32_t &r, bool &f) const {
    r = __ldg(tile_row + b);
    f = __ldg(row_ptr + r) < __ldg(tile_k + b);
  }
};

struct CooTileView {
  const int32_t *row_idx, *start_idx, *end_idx;
  int64_t nnz;
  int32_t G, np, m;
  __device__ int count() const { return np * G; }
  __device__ int32_t k0(int b) const {
    int i = b / G, g = b % G;
    int64_t s = start_idx[i], L = int64_t(end_idx[i]) - s + 1;
    return static_cast<int32_t>(s + (int64_t(g) * L) / G);
  }
  __device__ void row_flag(int b, int32_t &r, bool &f) const {
    int32_t k = k0(b);
    if (k >= nnz) {
      r = m;
      f = false;
      return;
    }
    r = __ldg(row_idx + k);
    f = k > 0 && __ldg(row_idx + k - 1) == r;
  }
};

template <class X, class View>
__global__ void fixup_split_rows(View v, const double *head, const double *tail,
                                 X *y, double alpha, double beta) {
  const int T = v.count();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < T;
       b += gridDim.x * blockDim.x) {
    int32_t r;
    bool f;
    v.row_flag(b, r, f);
    if (!f || b == 0) continue;
    int32_t rp;
    bool fp;
    v.row_flag(b - 1, rp, fp);
    if (fp && rp == r) continue;  // not the first flagged tile of the run
    double s = tail[b - 1];
    for (int j = b; j < T; ++j) {
      int32_t rj;
      bool fj;
      v.row_flag(j, rj, fj);
      if (!fj || rj != r) break;
      s += head[j];
    }
    double yo = beta == 0.0 ? 0.0 : double(y[r]);
    y[r] = static_cast<X>(beta == 0.0 ? alpha * s : alpha * s + beta * yo);
  }
}

__global__ void scale_f64(double *y, int64_t m, double beta) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < m;
       r += int64_t(gridDim.x) * blockDim.x)
    y[r] = beta * y[r];
}

__global__ void finish_csc_f32(const double *yacc, float *y, int64_t m,
                               double alpha, double beta) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < m;
       r += int64_t(gridDim.x) * blockDim.x) {
    double v = alpha * yacc[r];
    if (beta != 0.0) v += beta * double(y[r]);
    y[r] = float(v);
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

// msrep_profile_events: events recorded around the main kernel
static thread_local cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

static inline void prof_begin(cudaStream_t st) {
  if (g_prof_start) cudaEventRecord(g_prof_start, st);
}
static inline void prof_end(cudaStream_t st) {
  if (g_prof_stop) cudaEventRecord(g_prof_stop, st);
}

template <class K>
static int resident_blocks(K kernel, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, smem) !=
          cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

struct Workspace {
  double *head, *tail, *yacc;
};

static size_t ws_layout(int64_t tiles, int64_t m_acc, Workspace *w, void *base) {
  size_t o = 0;
  size_t oh = o;
  o = align256(o + sizeof(double) * tiles);
  size_t ot = o;
  o = align256(o + sizeof(double) * tiles);
  size_t oy = o;
  o = align256(o + sizeof(double) * m_acc);
  if (w && base) {
    char *p = static_cast<char *>(base);
    w->head = reinterpret_cast<double *>(p + oh);
    w->tail = reinterpret_cast<double *>(p + ot);
    w->yacc = reinterpret_cast<double *>(p + oy);
  }
  return o + 256;
}

static int64_t tiles_for(const msrep_matrix *A, const msrep_partition *p, int32_t tile) {
  if (A->fmt == MSREP_COO) return p->np * coo_tiles_per_part(A->nnz, p->np, tile);
  const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
  return plan_layout(n_major, A->nnz, p->np, tile).tmax;
}

template <class Pol, int IPT>
static msrep_status run_csr(const msrep_matrix *A, const msrep_partition *p,
                            double alpha, const void *x, double beta, void *y,
                            unsigned flags, const Workspace &w, cudaStream_t st) {
  const int32_t tile = effective_tile(p->tile);
  PlanLayout L = plan_layout(A->m, A->nnz, p->np, tile);
  const char *plan = static_cast<const char *>(p->plan);
  CsrArgs<Pol> a;
  a.row_ptr = A->ptr;
  a.col_idx = A->idx;
  a.val = static_cast<const typename Pol::V *>(A->val);
  a.x = static_cast<const typename Pol::X *>(x);
  a.y = static_cast<typename Pol::X *>(y);
  a.alpha = alpha;
  a.beta = beta;
  a.finish = finish_mode(alpha, beta);
  a.tile_row = reinterpret_cast<const int32_t *>(plan + L.off_row);
  a.tile_k = reinterpret_cast<const int32_t *>(plan + L.off_k);
  const int32_t *n_tiles = reinterpret_cast<const int32_t *>(plan + L.off_toff) + p->np;
  a.head = w.head;
  a.tail = w.tail;
  a.m = A->m;
  a.comp_mode = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  auto kern = csr_tiles<Pol, IPT>;
  static int nb = -1;
  if (nb < 0) nb = resident_blocks(kern, 0);
  int64_t grid = std::min<int64_t>(ceil_div(L.tmax, kWarps), int64_t(nb) * sm_count());
  if (grid < 1) grid = 1;
  prof_begin(st);
  kern<<<static_cast<int>(grid), kThreads, 0, st>>>(a, n_tiles, A->nnz);
  prof_end(st);
  MSREP_CUDA_TRY(cudaGetLastError());
  CsrTileView v{a.tile_row, a.tile_k, A->ptr, n_tiles};
  int64_t fg = std::min<int64_t>(ceil_div(L.tmax, 256), 4 * sm_count());
  fixup_split_rows<typename Pol::X, CsrTileView>
      <<<static_cast<int>(std::max<int64_t>(fg, 1)), 256, 0, st>>>(
          v, w.head, w.tail, a.y, alpha, beta);
  MSREP_CUDA_TRY(cudaGetLastError());
  return MSREP_OK;
}

template <class Pol, int IPT>
static msrep_status run_coo(const msrep_matrix *A, const msrep_partition *p,
                            double alpha, const void *x, double beta, void *y,
                            unsigned flags, const Workspace &w, cudaStream_t st) {
  const int32_t tile = effective_tile(p->tile);
  CooArgs<Pol> a;
  a.row_idx = A->idx2;
  a.col_idx = A->idx;
  a.val = static_cast<const typename Pol::V *>(A->val);
  a.x = static_cast<const typename Pol::X *>(x);
  a.y = static_cast<typename Pol::X *>(y);
  a.alpha = alpha;
  a.beta = beta;
  a.finish = finish_mode(alpha, beta);
  a.start_idx = p->start_idx;
  a.end_idx = p->end_idx;
  a.np = p->np;
  a.G = static_cast<int32_t>(coo_tiles_per_part(A->nnz, p->np, tile));
  a.m = A->m;
  a.nnz = A->nnz;
  a.head = w.head;
  a.tail = w.tail;
  a.comp_mode = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  auto kern = coo_tiles<Pol, IPT>;
  static int nb = -1;
  if (nb < 0) nb = resident_blocks(kern, 0);
  const int64_t T = int64_t(a.np) * a.G;
  int64_t grid = std::min<int64_t>(ceil_div(T, kWarps), int64_t(nb) * sm_count());
  prof_begin(st);
  kern<<<static_cast<int>(std::max<int64_t>(grid, 1)), kThreads, 0, st>>>(a);
  prof_end(st);
  MSREP_CUDA_TRY(cudaGetLastError());
  CooTileView v{A->idx2, p->start_idx, p->end_idx, A->nnz, a.G, a.np, A->m};
  int64_t fg = std::min<int64_t>(ceil_div(T, 256), 4 * sm_count());
  fixup_split_rows<typename Pol::X, CooTileView>
      <<<static_cast<int>(std::max<int64_t>(fg, 1)), 256, 0, st>>>(
          v, w.head, w.tail, a.y, alpha, beta);
  MSREP_CUDA_TRY(cudaGetLastError());
  return MSREP_OK;
}

template <class Pol, int IPT>
static msrep_status run_csc(const msrep_matrix *A, const msrep_partition *p,
                            double alpha, const void *x, double beta, void *y,
                            const Workspace &w, cudaStream_t st) {
  const int32_t tile = effective_tile(p->tile);
  PlanLayout L = plan_layout(A->n, A->nnz, p->np, tile);
  const char *plan = static_cast<const char *>(p->plan);
  constexpr bool kF64 = sizeof(typename Pol::X) == 8;
  CscArgs<Pol> a;
  a.col_ptr = A->ptr;
  a.row_idx = A->idx;
  a.val = static_cast<const typename Pol::V *>(A->val);
  a.x = static_cast<const typename Pol::X *>(x);
  a.tile_row = reinterpret_cast<const int32_t *>(plan + L.off_row);
  a.tile_k = reinterpret_cast<const int32_t *>(plan + L.off_k);
  const int32_t *n_tiles = reinterpret_cast<const int32_t *>(plan + L.off_toff) + p->np;
  a.n = A->n;
  const int64_t m = A->m;
  const int sg = 4 * sm_count();
  if (kF64) {
    a.yacc = static_cast<double *>(y);
    a.scale = alpha;
    a.scaled = alpha != 1.0;
    if (m > 0) {
      if (beta == 0.0)
        MSREP_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * m, st));
      else if (beta != 1.0)
        scale_f64<<<sg, 256, 0, st>>>(a.yacc, m, beta);
    }
  } else {
    a.yacc = w.yacc;
    a.scale = 1.0;
    a.scaled = false;
    if (m > 0) MSREP_CUDA_TRY(cudaMemsetAsync(w.yacc, 0, sizeof(double) * m, st));
  }
  MSREP_CUDA_TRY(cudaGetLastError());
  auto kern = csc_tiles<Pol, IPT>;
  static int nb = -1;
  if (nb < 0) nb = resident_blocks(kern, 0);
  int64_t grid = std::min<int64_t>(ceil_div(L.tmax, kWarps), int64_t(nb) * sm_count());
  prof_begin(st);
  kern<<<static_cast<int>(std::max<int64_t>(grid, 1)), kThreads, 0, st>>>(a, n_tiles, A->nnz);
  prof_end(st);
  MSREP_CUDA_TRY(cudaGetLastError());
  if (!kF64 && m > 0) {
    finish_csc_f32<<<sg, 256, 0, st>>>(w.yacc, static_cast<float *>(y), m, alpha, beta);
    MSREP_CUDA_TRY(cudaGetLastError());
  }
  return MSREP_OK;
}

template <class Pol>
static msrep_status dispatch_tile(const msrep_matrix *A, const msrep_partition *p,
                                  double alpha, const void *x, double beta,
                                  void *y, unsigned flags, const Workspace &w,
                                  cudaStream_t st) {
  const int32_t tile = effective_tile(p->tile);
#define MSREP_FMT_CASE(IPT)                                                   \
  switch (A->fmt) {                                                           \
    case MSREP_CSR: return run_csr<Pol, IPT>(A, p, alpha, x, beta, y, flags, w, st); \
    case MSREP_COO: return run_coo<Pol, IPT>(A, p, alpha, x, beta, y, flags, w, st); \
    default: return run_csc<Pol, IPT>(A, p, alpha, x, beta, y, w, st);        \
  }
  switch (tile) {
    case 128: MSREP_FMT_CASE(4)
    case 256: MSREP_FMT_CASE(8)
    case 512: MSREP_FMT_CASE(16)
    case 1024: MSREP_FMT_CASE(32)
  }
#undef MSREP_FMT_CASE
  return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", tile);
}

__global__ void scale_any(void *y, int64_t m, double beta, int is_f64) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < m;
       r += int64_t(gridDim.x) * blockDim.x) {
    if (is_f64) {
      double *yy = static_cast<double *>(y);
      yy[r] = beta * yy[r];
    } else {
      float *yy = static_cast<float *>(y);
      yy[r] = float(beta * double(yy[r]));
    }
  }
}

}  // namespace msrep

using namespace msrep;

extern "C" {

msrep_status msrep_profile_events(void *start, void *stop) {
  g_prof_start = reinterpret_cast<cudaEvent_t>(start);
  g_prof_stop = reinterpret_cast<cudaEvent_t>(stop);
  return ok();
}

msrep_status msrep_spmv_workspace_size(const msrep_matrix *A,
                                       const msrep_partition *part,
                                       size_t *bytes) {
  MSREP_TRY(check_matrix(A));
  if (!part || part->np < 1 || !bytes)
    return fail(MSREP_ERR_INVALID_ARG, "bad partition or bytes pointer");
  const int32_t tile = effective_tile(part->tile);
  if (!tile_supported(tile)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", part->tile);
  const int64_t tiles = tiles_for(A, part, tile);
  const int64_t m_acc = (A->fmt == MSREP_CSC && A->val_dtype != MSREP_F64) ? A->m : 0;
  *bytes = ws_layout(tiles, m_acc, nullptr, nullptr);
  return ok();
}

msrep_status msrep_spmv(const msrep_matrix *A, const msrep_partition *part,
                        double alpha, const void *x, double beta, void *y,
                        int32_t xy_dtype, unsigned flags, void *workspace,
                        void *stream) {
  MSREP_TRY(check_matrix(A));
  if (!part || part->np < 1 || !part->start_idx || !part->end_idx)
    return fail(MSREP_ERR_INVALID_ARG, "bad partition");
  const int32_t tile = effective_tile(part->tile);
  if (!tile_supported(tile)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", part->tile);
  if ((A->m > 0 && !y) || (A->n > 0 && !x && A->nnz > 0))
    return fail(MSREP_ERR_INVALID_ARG, "x or y is NULL");
  const bool f64 = A->val_dtype == MSREP_F64;
  if (f64 != (xy_dtype == MSREP_F64) || (xy_dtype != MSREP_F64 && xy_dtype != MSREP_F32))
    return fail(MSREP_ERR_INVALID_ARG,
                "unsupported types: val %d with x/y %d (F64/F64, F32/F32 or BF16/F32)",
                A->val_dtype, xy_dtype);
  cudaStream_t st = as_stream(stream);
  if (A->m == 0) return ok();
  if (A->fmt != MSREP_COO) {
    const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
    const int64_t need = static_cast<int64_t>(plan_layout(n_major, A->nnz, part->np, tile).bytes);
    if (!part->plan || part->plan_bytes < need)
      return fail(MSREP_ERR_WORKSPACE, "CSR/CSC SpMV needs the partition's tile plan (%lld bytes)",
                  (long long)need);
  }
  if (A->nnz == 0) {
    // y = beta * y
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    if (beta == 0.0) {
      MSREP_CUDA_TRY(cudaMemsetAsync(y, 0, es * size_t(A->m), st));
    } else if (beta != 1.0) {
      scale_any<<<4 * sm_count(), 256, 0, st>>>(y, A->m, beta, f64 ? 1 : 0);
      MSREP_CUDA_TRY(cudaGetLastError());
    }
    return ok();
  }
  {
    // the kernels read the nonzero arrays in aligned groups of 8 elements
    const uintptr_t mis = reinterpret_cast<uintptr_t>(A->idx) | reinterpret_cast<uintptr_t>(A->idx2) |
                          reinterpret_cast<uintptr_t>(A->val);
    if (mis & (A->val_dtype == MSREP_BF16 ? 15 : 31))
      return fail(MSREP_ERR_INVALID_ARG,
                  "idx, idx2 and val must be 32-byte aligned (16-byte for bf16-only val)");
  }
  if (!workspace) return fail(MSREP_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) & 15)
    return fail(MSREP_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  const int64_t tiles = tiles_for(A, part, tile);
  const int64_t m_acc = (A->fmt == MSREP_CSC && !f64) ? A->m : 0;
  Workspace w;
  ws_layout(tiles, m_acc, &w, workspace);
  msrep_status s;
  switch (A->val_dtype) {
    case MSREP_F64:
      s = dispatch_tile<PolF64>(A, part, alpha, x, beta, y, flags, w, st);
      break;
    case MSREP_F32:
      s = dispatch_tile<PolF32<float>>(A, part, alpha, x, beta, y, flags, w, st);
      break;
    default:
      s = dispatch_tile<PolF32<bf16_t>>(A, part, alpha, x, beta, y, flags, w, st);
      break;
  }
  if (s != MSREP_OK) return s;
  return ok();
}

}  // extern "C"
