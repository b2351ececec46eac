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

namespace msrep {

msrep_status check_matrix(const msrep_matrix *A);
int32_t effective_tile(int32_t tile);

// ---------------------------------------------------------------------------
// arithmetic policies
// ---------------------------------------------------------------------------

// Plain FP64: products and sums rounded in binary64.
struct PolF64 {
  using V = double;
  using X = double;
  using Prod = double;
  using Acc = double;
  __device__ static Prod prod(double v, double x) { return __dmul_rn(v, x); }
  __device__ static Acc zero() { return 0.0; }
  __device__ static Acc add(Acc a, Prod p, bool) { return __dadd_rn(a, p); }
  __device__ static Acc combine(Acc a, Acc b) { return __dadd_rn(a, b); }
  __device__ static double to_f64(Acc a) { return a; }
  __device__ static X finish(Acc a, double alpha, double beta, X yold) {
    return beta == 0.0 ? alpha * a : alpha * a + beta * yold;
  }
  __device__ static Acc shfl_up(Acc a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
};

// Low precision: values FP32 or BF16, x and y FP32, binary32 accumulation.
// A product is kept with its rounding error (TwoProduct by FMA); rows that
// are compensated accumulate (s, c) by TwoSum, i.e. Ogita-Rump-Oishi Dot2.
struct F32Pair {
  float s, c;
};

template <typename VT>
struct PolF32 {
  using V = VT;
  using X = float;
  using Prod = float2;  // (product, its rounding error)
  using Acc = F32Pair;
  __device__ static Prod prod(float v, float x) {
    float p, e;
    two_prod(v, x, p, e);
    return make_float2(p, e);
  }
  __device__ static Acc zero() { return F32Pair{0.f, 0.f}; }
  __device__ static Acc add(Acc a, Prod p, bool comp) {
    if (comp) {
      float s, e;
      two_sum(a.s, p.x, s, e);
      return F32Pair{s, __fadd_rn(a.c, __fadd_rn(e, p.y))};
    }
    return F32Pair{__fadd_rn(a.s, p.x), a.c};
  }
  __device__ static Acc combine(Acc a, Acc b) {
    float s, e;
    two_sum(a.s, b.s, s, e);
    return F32Pair{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
  }
  __device__ static double to_f64(Acc a) { return double(a.s) + double(a.c); }
  __device__ static X finish(Acc a, double alpha, double beta, X yold) {
    float t = __fadd_rn(a.s, a.c);
    float r = __fmul_rn(float(alpha), t);
    return beta == 0.0 ? r : __fadd_rn(r, __fmul_rn(float(beta), yold));
  }
  __device__ static Acc shfl_up(Acc a, int o) {
    return F32Pair{__shfl_up_sync(0xffffffffu, a.s, o),
                   __shfl_up_sync(0xffffffffu, a.c, o)};
  }
};

__device__ __forceinline__ double load_x(const double *x, int32_t c) { return __ldg(x + c); }
__device__ __forceinline__ float load_x(const float *x, int32_t c) { return __ldg(x + c); }

// ---------------------------------------------------------------------------
// block-wide segmented scan of (flag, value): a set flag restarts the sum.
// Returns the exclusive prefix; `last` receives the block-inclusive value
// of the last thread.
// ---------------------------------------------------------------------------

template <class Pol, int THREADS>
struct SegScan {
  using Acc = typename Pol::Acc;
  struct Storage {
    Acc wv[THREADS / 32];
    int wf[THREADS / 32];
    Acc last;
  };
  __device__ static Acc run(Storage &sm, bool flag, Acc v, Acc &last) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int f = flag;
    Acc inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Acc u = Pol::shfl_up(inc, o);
      int fu = __shfl_up_sync(0xffffffffu, f, o);
      if (lane >= o) {
        if (!f) inc = Pol::combine(u, inc);
        f |= fu;
      }
    }
    if (lane == 31) {
      sm.wv[wid] = inc;
      sm.wf[wid] = f;
    }
    __syncthreads();
    if (wid == 0) {
      constexpr int NW = THREADS / 32;
      int wf = lane < NW ? sm.wf[lane] : 0;
      Acc wv = lane < NW ? sm.wv[lane] : Pol::zero();
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        Acc u = Pol::shfl_up(wv, o);
        int fu = __shfl_up_sync(0xffffffffu, wf, o);
        if (lane >= o) {
          if (!wf) wv = Pol::combine(u, wv);
          wf |= fu;
        }
      }
      // exclusive prefix over warps, stored back
      Acc ev = Pol::shfl_up(wv, 1);
      int ef = __shfl_up_sync(0xffffffffu, wf, 1);
      if (lane == 0) {
        ev = Pol::zero();
        ef = 0;
      }
      if (lane < NW) {
        sm.wv[lane] = ev;
        sm.wf[lane] = ef;
      }
    }
    __syncthreads();
    // block-inclusive value of this thread
    Acc wpre = sm.wv[wid];
    Acc binc = f ? inc : Pol::combine(wpre, inc);
    // exclusive = block-inclusive of the previous thread
    Acc ex = Pol::shfl_up(binc, 1);
    if (lane == 0) ex = wpre;
    if (threadIdx.x == THREADS - 1) sm.last = binc;
    __syncthreads();
    last = sm.last;
    return ex;
  }
};

// ---------------------------------------------------------------------------
// CSR: merge-path tiles
// ---------------------------------------------------------------------------

template <class Pol>
struct CsrArgs {
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  typename Pol::X *y;
  double alpha, beta;
  const int32_t *tile_row;  // [T+1]
  const int32_t *tile_k;    // [T+1]
  const int32_t *n_tiles;   // device scalar T
  double *head, *tail;      // [T] FP64 partials of split rows
  int32_t m;
  unsigned comp_mode;       // 0 selective, MSREP_COMP_ALL, MSREP_COMP_NONE
};

template <class Pol>
__device__ __forceinline__ bool want_comp(unsigned mode, int64_t len, bool split) {
  if (mode & MSREP_COMP_ALL) return true;
  if (mode & MSREP_COMP_NONE) return false;
  return split || len > 256;
}

template <class Pol, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS) csr_tiles(CsrArgs<Pol> a) {
  using Acc = typename Pol::Acc;
  using Prod = typename Pol::Prod;
  constexpr int TILE = THREADS * IPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Prod *s_prod = reinterpret_cast<Prod *>(smem_raw);
  int32_t *s_end = reinterpret_cast<int32_t *>(smem_raw + sizeof(Prod) * TILE);
  __shared__ typename SegScan<Pol, THREADS>::Storage scan_sm;

  const int T = *a.n_tiles;
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < T; b += gridDim.x) {
    const int32_t r0 = __ldg(a.tile_row + b), k0 = __ldg(a.tile_k + b);
    const int32_t r1 = __ldg(a.tile_row + b + 1), k1 = __ldg(a.tile_k + b + 1);
    const int32_t nrows = r1 - r0, nnzt = k1 - k0;
    const int32_t rs0 = __ldg(a.row_ptr + r0);
    const bool flag = rs0 < k0;  // first row started in an earlier tile
    // end of the last (partial) row, for the compensation predicate
    const int32_t re_last = (r1 < a.m) ? __ldg(a.row_ptr + r1 + 1) : k1;

    for (int i = tid; i < nrows; i += THREADS) s_end[i] = __ldg(a.row_ptr + r0 + 1 + i) - k0;
    {
      int32_t cj[IPT];
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        int j = tid + u * THREADS;
        cj[u] = j < nnzt ? ld_stream(a.col_idx + k0 + j) : 0;
      }
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        int j = tid + u * THREADS;
        if (j < nnzt) s_prod[j] = Pol::prod(ld_stream(a.val + k0 + j), load_x(a.x, cj[u]));
      }
    }
    __syncthreads();

    // this thread's stretch of the tile's merge path
    const int items = nrows + nnzt;
    const int d = min(tid * IPT, items);
    const int dend = min(d + IPT, items);
    int lo = max(0, d - nnzt), hi = min(d, nrows);
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (s_end[mid] <= d - mid - 1)
        lo = mid + 1;
      else
        hi = mid;
    }
    int r = lo, k = d - lo;

    auto row_comp = [&](int rr) -> bool {
      int64_t st = rr == 0 ? int64_t(rs0) : int64_t(k0) + s_end[rr - 1];
      int64_t en = rr < nrows ? int64_t(k0) + s_end[rr] : int64_t(re_last);
      bool split = (rr == 0 && flag) || rr == nrows;
      return want_comp<Pol>(a.comp_mode, en - st, split);
    };

    Acc acc = Pol::zero(), first_acc = Pol::zero();
    bool emitted = false;
    int first_r = 0;
    bool comp = (d < dend) ? row_comp(r) : false;
    for (int it = d; it < dend; ++it) {
      if (r < nrows && s_end[r] <= k) {
        if (!emitted) {
          emitted = true;
          first_r = r;
          first_acc = acc;
        } else {
          const int32_t row = r0 + r;
          a.y[row] = Pol::finish(acc, a.alpha, a.beta, a.beta == 0.0 ? 0 : a.y[row]);
        }
        acc = Pol::zero();
        ++r;
        comp = row_comp(r);
      } else {
        acc = Pol::add(acc, s_prod[k], comp);
        ++k;
      }
    }

    Acc last;
    Acc carry = SegScan<Pol, THREADS>::run(scan_sm, emitted, acc, last);
    if (emitted) {
      Acc tot = Pol::combine(carry, first_acc);
      if (first_r == 0 && flag) {
        a.head[b] = Pol::to_f64(tot);
      } else {
        const int32_t row = r0 + first_r;
        a.y[row] = Pol::finish(tot, a.alpha, a.beta, a.beta == 0.0 ? 0 : a.y[row]);
      }
    }
    if (tid == THREADS - 1) {
      if (nrows == 0) {
        if (flag)
          a.head[b] = Pol::to_f64(last);
        else if (nnzt > 0)
          a.tail[b] = Pol::to_f64(last);
      } else if (k1 > __ldg(a.row_ptr + r1)) {
        a.tail[b] = Pol::to_f64(last);
      }
    }
    __syncthreads();
  }
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

// ---------------------------------------------------------------------------
// COO: nonzero tiles inside each partition
// ---------------------------------------------------------------------------

template <class Pol>
struct CooArgs {
  const int32_t *row_idx;
  const int32_t *col_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  typename Pol::X *y;
  double alpha, beta;
  const int32_t *start_idx, *end_idx;  // partition metadata
  int32_t np, G, m;
  int64_t nnz;
  double *head, *tail;
  unsigned comp_mode;
};

template <class X>
__device__ __forceinline__ void write_beta(X *y, int32_t row, double beta) {
  y[row] = beta == 0.0 ? X(0) : static_cast<X>(beta * double(y[row]));
}

template <class Pol, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS) coo_tiles(CooArgs<Pol> a) {
  using Acc = typename Pol::Acc;
  using Prod = typename Pol::Prod;
  constexpr int TILE = THREADS * IPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Prod *s_prod = reinterpret_cast<Prod *>(smem_raw);
  int32_t *s_row = reinterpret_cast<int32_t *>(smem_raw + sizeof(Prod) * TILE);
  __shared__ typename SegScan<Pol, THREADS>::Storage scan_sm;

  const int T = a.np * a.G;
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < T; b += gridDim.x) {
    const int i = b / a.G, g = b % a.G;
    const int64_t s = a.start_idx[i], L = int64_t(a.end_idx[i]) - s + 1;
    const int32_t k0 = static_cast<int32_t>(s + (int64_t(g) * L) / a.G);
    const int32_t k1 = static_cast<int32_t>(s + (int64_t(g + 1) * L) / a.G);
    const int32_t nnzt = k1 - k0;
    if (tid == 0) {
      a.head[b] = 0.0;
      a.tail[b] = 0.0;
    }
    if (nnzt == 0) continue;  // uniform across the block
    const int32_t prev_row = k0 > 0 ? __ldg(a.row_idx + k0 - 1) : -1;
    const int32_t next_row = k1 < a.nnz ? __ldg(a.row_idx + k1) : a.m;
    {
      int32_t cj[IPT];
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        int j = tid + u * THREADS;
        if (j < nnzt) {
          cj[u] = ld_stream(a.col_idx + k0 + j);
          s_row[j] = ld_stream(a.row_idx + k0 + j);
        }
      }
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        int j = tid + u * THREADS;
        if (j < nnzt) s_prod[j] = Pol::prod(ld_stream(a.val + k0 + j), load_x(a.x, cj[u]));
      }
    }
    __syncthreads();
    const int32_t first_row = s_row[0], last_row = s_row[nnzt - 1];
    const bool flag = prev_row == first_row;
    const bool cont = next_row == last_row;

    // leading empty rows (only the tile that holds nonzero 0)
    if (k0 == 0)
      for (int32_t rr = tid; rr < first_row; rr += THREADS) write_beta(a.y, rr, a.beta);

    // compensation predicate of the run that starts at j: its length inside
    // the tile (found by bisection in shared memory) and whether it is split
    auto run_comp = [&](int j) -> bool {
      if (a.comp_mode & (MSREP_COMP_ALL | MSREP_COMP_NONE))
        return want_comp<Pol>(a.comp_mode, 0, false);
      const int32_t rv = s_row[j];
      int lo = 0, hi = j;  // first index with row == rv
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (s_row[mid] < rv) lo = mid + 1; else hi = mid;
      }
      int st = lo;
      lo = j;
      hi = nnzt;  // first index with row > rv
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (s_row[mid] <= rv) lo = mid + 1; else hi = mid;
      }
      bool split = (st == 0 && flag) || (lo == nnzt && cont);
      return want_comp<Pol>(a.comp_mode, lo - st, split);
    };

    const int j0 = min(tid * IPT, nnzt), j1 = min(j0 + IPT, nnzt);
    Acc acc = Pol::zero(), first_acc = Pol::zero();
    bool emitted = false;
    int32_t first_r = 0;
    int32_t cur = j0 < nnzt ? (tid == 0 ? first_row : s_row[j0 - 1]) : 0;
    bool comp = j0 < j1 ? run_comp(j0) : false;
    for (int j = j0; j < j1; ++j) {
      const int32_t rj = s_row[j];
      if (rj != cur) {
        if (!emitted) {
          emitted = true;
          first_r = cur;
          first_acc = acc;
        } else {
          a.y[cur] = Pol::finish(acc, a.alpha, a.beta, a.beta == 0.0 ? 0 : a.y[cur]);
        }
        for (int32_t rr = cur + 1; rr < rj; ++rr) write_beta(a.y, rr, a.beta);
        cur = rj;
        acc = Pol::zero();
        comp = run_comp(j);
      }
      acc = Pol::add(acc, s_prod[j], comp);
    }

    Acc last;
    Acc carry = SegScan<Pol, THREADS>::run(scan_sm, emitted, acc, last);
    if (emitted) {
      Acc tot = Pol::combine(carry, first_acc);
      if (first_r == first_row && flag)
        a.head[b] = Pol::to_f64(tot);
      else
        a.y[first_r] = Pol::finish(tot, a.alpha, a.beta, a.beta == 0.0 ? 0 : a.y[first_r]);
    }
    if (tid == THREADS - 1) {
      if (last_row == first_row && flag)
        a.head[b] = Pol::to_f64(last);
      else if (cont)
        a.tail[b] = Pol::to_f64(last);
      else
        a.y[last_row] = Pol::finish(last, a.alpha, a.beta, a.beta == 0.0 ? 0 : a.y[last_row]);
    }
    // empty rows between this tile's last row and the next tile's first row
    if (!cont)
      for (int32_t rr = last_row + 1 + tid; rr < next_row; rr += THREADS)
        write_beta(a.y, rr, a.beta);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// CSC: merge-path tiles over col_ptr, scatter-add into y
// ---------------------------------------------------------------------------

template <class Pol>
struct CscArgs {
  const int32_t *col_ptr;
  const int32_t *row_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  double *yacc;  // FP64 accumulation target (y itself on the FP64 path)
  double scale;  // alpha on the FP64 path, 1 when a finishing pass follows
  const int32_t *tile_row, *tile_k, *n_tiles;
  int32_t n;
};

template <class Pol, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS) csc_tiles(CscArgs<Pol> a) {
  constexpr int TILE = THREADS * IPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *s_val = reinterpret_cast<double *>(smem_raw);
  int32_t *s_row = reinterpret_cast<int32_t *>(smem_raw + sizeof(double) * TILE);
  int32_t *s_end = s_row + TILE;

  const int T = *a.n_tiles;
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < T; b += gridDim.x) {
    const int32_t c0 = __ldg(a.tile_row + b), k0 = __ldg(a.tile_k + b);
    const int32_t c1 = __ldg(a.tile_row + b + 1), k1 = __ldg(a.tile_k + b + 1);
    const int32_t ncols = c1 - c0, nnzt = k1 - k0;
    for (int i = tid; i < ncols; i += THREADS) s_end[i] = __ldg(a.col_ptr + c0 + 1 + i) - k0;
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      int j = tid + u * THREADS;
      if (j < nnzt) {
        s_row[j] = ld_stream(a.row_idx + k0 + j);
        s_val[j] = double(ld_stream(a.val + k0 + j));
      }
    }
    __syncthreads();
    const int items = ncols + nnzt;
    const int d = min(tid * IPT, items);
    const int dend = min(d + IPT, items);
    int lo = max(0, d - nnzt), hi = min(d, ncols);
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (s_end[mid] <= d - mid - 1)
        lo = mid + 1;
      else
        hi = mid;
    }
    int c = lo, k = d - lo;
    double xc = (d < dend && c0 + c < a.n) ? double(load_x(a.x, c0 + c)) * a.scale : 0.0;
    for (int it = d; it < dend; ++it) {
      if (c < ncols && s_end[c] <= k) {
        ++c;
        xc = (c0 + c < a.n) ? double(load_x(a.x, c0 + c)) * a.scale : 0.0;
      } else {
        atomicAdd(a.yacc + s_row[k], s_val[k] * xc);
        ++k;
      }
    }
    __syncthreads();
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

constexpr int kThreads = 256;

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

template <class K>
static msrep_status prep_kernel(K kernel, size_t smem) {
  MSREP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
  return MSREP_OK;
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
  a.tile_row = reinterpret_cast<const int32_t *>(plan + L.off_row);
  a.tile_k = reinterpret_cast<const int32_t *>(plan + L.off_k);
  a.n_tiles = reinterpret_cast<const int32_t *>(plan + L.off_toff) + p->np;
  a.head = w.head;
  a.tail = w.tail;
  a.m = A->m;
  a.comp_mode = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  constexpr int TILE = kThreads * IPT;
  const size_t smem = (sizeof(typename Pol::Prod) + sizeof(int32_t)) * TILE;
  auto kern = csr_tiles<Pol, kThreads, IPT>;
  static int nb = -1;
  if (nb < 0) {
    MSREP_TRY(prep_kernel(kern, smem));
    nb = resident_blocks(kern, smem);
  }
  int64_t grid = std::min<int64_t>(L.tmax, int64_t(nb) * sm_count());
  if (grid < 1) grid = 1;
  prof_begin(st);
  kern<<<static_cast<int>(grid), kThreads, smem, st>>>(a);
  prof_end(st);
  MSREP_CUDA_TRY(cudaGetLastError());
  CsrTileView v{a.tile_row, a.tile_k, A->ptr, a.n_tiles};
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
  a.start_idx = p->start_idx;
  a.end_idx = p->end_idx;
  a.np = p->np;
  a.G = static_cast<int32_t>(coo_tiles_per_part(A->nnz, p->np, tile));
  a.m = A->m;
  a.nnz = A->nnz;
  a.head = w.head;
  a.tail = w.tail;
  a.comp_mode = flags & (MSREP_COMP_ALL | MSREP_COMP_NONE);
  constexpr int TILE = kThreads * IPT;
  const size_t smem = (sizeof(typename Pol::Prod) + sizeof(int32_t)) * TILE;
  auto kern = coo_tiles<Pol, kThreads, IPT>;
  static int nb = -1;
  if (nb < 0) {
    MSREP_TRY(prep_kernel(kern, smem));
    nb = resident_blocks(kern, smem);
  }
  const int64_t T = int64_t(a.np) * a.G;
  int64_t grid = std::min<int64_t>(T, int64_t(nb) * sm_count());
  prof_begin(st);
  kern<<<static_cast<int>(std::max<int64_t>(grid, 1)), kThreads, smem, st>>>(a);
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
  a.n_tiles = reinterpret_cast<const int32_t *>(plan + L.off_toff) + p->np;
  a.n = A->n;
  const int64_t m = A->m;
  const int sg = 4 * sm_count();
  if (kF64) {
    a.yacc = static_cast<double *>(y);
    a.scale = alpha;
    if (m > 0) {
      if (beta == 0.0)
        MSREP_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * m, st));
      else if (beta != 1.0)
        scale_f64<<<sg, 256, 0, st>>>(a.yacc, m, beta);
    }
  } else {
    a.yacc = w.yacc;
    a.scale = 1.0;
    if (m > 0) MSREP_CUDA_TRY(cudaMemsetAsync(w.yacc, 0, sizeof(double) * m, st));
  }
  MSREP_CUDA_TRY(cudaGetLastError());
  constexpr int TILE = kThreads * IPT;
  const size_t smem = (sizeof(double) + 2 * sizeof(int32_t)) * TILE;
  auto kern = csc_tiles<Pol, kThreads, IPT>;
  static int nb = -1;
  if (nb < 0) {
    MSREP_TRY(prep_kernel(kern, smem));
    nb = resident_blocks(kern, smem);
  }
  int64_t grid = std::min<int64_t>(L.tmax, int64_t(nb) * sm_count());
  prof_begin(st);
  kern<<<static_cast<int>(std::max<int64_t>(grid, 1)), kThreads, smem, st>>>(a);
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
    case 512: MSREP_FMT_CASE(2)
    case 1024: MSREP_FMT_CASE(4)
    case 2048: MSREP_FMT_CASE(8)
    case 4096: MSREP_FMT_CASE(16)
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
