// Tile processors of the partitioned SpMV, shared by the single-matrix
// kernels (spmv.cu) and the persistent batched kernel (batched.cu), so that
// a matrix gives bit-identical results in both.
//
// Work decomposition (two levels, as in the two-level split of Sec. 4.2 with
// thread blocks in place of GPUs):
//  * a partition of Alg. 2/4/6 is cut into warp tiles; CSR/CSC tiles are
//    equal stretches of the merge path of (row ends, nonzeros), so both rows
//    and nonzeros per tile are bounded; COO tiles are equal nonzero ranges
//    (Alg. 2's split applied inside the partition).  A warp owns a tile
//    alone: no block-wide barrier, so the warps of a block overlap their
//    memory latencies freely;
//  * inside a tile the nonzeros are split evenly over the 32 lanes (the same
//    floor(i*nnz/P) rule), and each lane sums its contiguous run with one
//    fused multiply-add per nonzero.  On GB300 the FP64 pipe sustains about
//    two lane operations per clock per SM, so one DFMA per nonzero, equal
//    nonzero counts per lane (no idle lanes in the DFMA warp instructions)
//    and no FP64 work for row finishing when alpha = 1, beta = 0 keep the
//    plain FP64 path from being FP64-bound; the x gathers (one L1 line
//    lookup each) bound it instead.
//  * rows split between lanes are merged by a warp segmented scan (skipped
//    when every lane finished a row), rows split between tiles by the fix-up
//    kernel in tile order, with beta applied once (Sec. 3.2.1, Sec. 4.3).
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "tma.cuh"

namespace msrep {

// ---------------------------------------------------------------------------
// arithmetic policies
// ---------------------------------------------------------------------------

// y-update modes, chosen on the host so the device never compares doubles
enum : int { kFinishCopy = 0, kFinishScale = 1, kFinishAxpby = 2 };

inline int finish_mode(double alpha, double beta) {
  if (beta == 0.0) return alpha == 1.0 ? kFinishCopy : kFinishScale;
  return kFinishAxpby;
}

// Plain FP64.  One fused multiply-add per nonzero.
struct PolF64 {
  using V = double;
  using X = double;
  using Acc = double;
  static constexpr bool kLow = false;
  __device__ static Acc zero() { return 0.0; }
  __device__ static Acc fma(Acc a, double v, double x, bool) { return __fma_rn(v, x, a); }
  __device__ static Acc combine(Acc a, Acc b) { return __dadd_rn(a, b); }
  __device__ static double to_f64(Acc a) { return a; }
  __device__ static X finish(Acc a, int mode, double alpha, double beta, const X *y) {
    if (mode == kFinishCopy) return a;
    if (mode == kFinishScale) return __dmul_rn(alpha, a);
    return __fma_rn(alpha, a, __dmul_rn(beta, *y));
  }
  __device__ static Acc shfl_up(Acc a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
  __device__ static Acc shfl(Acc a, int l) { return __shfl_sync(0xffffffffu, a, l); }
};

// Low precision: values FP32 or BF16, x and y FP32, binary32 accumulation.
// A compensated row accumulates (s, c) by Ogita-Rump-Oishi Dot2: every
// product keeps its rounding error (TwoProduct by FMA) and every addition
// its error (TwoSum); a plain row uses one FP32 FMA per nonzero.
struct F32Pair {
  float s, c;
};

template <typename VT>
struct PolF32 {
  using V = VT;
  using X = float;
  using Acc = F32Pair;
  static constexpr bool kLow = true;
  __device__ static Acc zero() { return F32Pair{0.f, 0.f}; }
  __device__ static Acc fma(Acc a, float v, float x, bool comp) {
    if (comp) {
      float p, ep, s, es;
      two_prod(v, x, p, ep);
      two_sum(a.s, p, s, es);
      return F32Pair{s, __fadd_rn(a.c, __fadd_rn(ep, es))};
    }
    return F32Pair{__fmaf_rn(v, x, a.s), a.c};
  }
  __device__ static Acc combine(Acc a, Acc b) {
    float s, e;
    two_sum(a.s, b.s, s, e);
    return F32Pair{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
  }
  __device__ static double to_f64(Acc a) { return double(a.s) + double(a.c); }
  __device__ static X finish(Acc a, int mode, double alpha, double beta, const X *y) {
    float t = __fadd_rn(a.s, a.c);
    if (mode == kFinishCopy) return t;
    float r = __fmul_rn(float(alpha), t);
    if (mode == kFinishScale) return r;
    return __fmaf_rn(float(beta), *y, r);
  }
  __device__ static Acc shfl_up(Acc a, int o) {
    return F32Pair{__shfl_up_sync(0xffffffffu, a.s, o), __shfl_up_sync(0xffffffffu, a.c, o)};
  }
  __device__ static Acc shfl(Acc a, int l) {
    return F32Pair{__shfl_sync(0xffffffffu, a.s, l), __shfl_sync(0xffffffffu, a.c, l)};
  }
};

__device__ __forceinline__ double load_x(const double *x, int32_t c) { return __ldg(x + c); }
__device__ __forceinline__ float load_x(const float *x, int32_t c) { return __ldg(x + c); }

// Compensation predicate of the low-precision form: rows longer than 256
// nonzeros and rows split between tiles or partitions, unless the caller
// forces all / none.
__device__ __forceinline__ bool want_comp(unsigned mode, int64_t len, bool split) {
  if (mode & MSREP_COMP_ALL) return true;
  if (mode & MSREP_COMP_NONE) return false;
  return split || len > 256;
}

// ---------------------------------------------------------------------------
// warp segmented scan of (flag, value) over the lanes of a tile.  A set flag
// means "this lane finished a row": the running sum restarts after it.
// Returns the exclusive prefix (the partial that flows into the lane's first
// finished row) and, in `last`, the inclusive value of lane 31 (the partial
// of the row that continues past the tile).
// ---------------------------------------------------------------------------

template <class Pol>
__device__ __forceinline__ typename Pol::Acc warp_seg_scan(bool flag, typename Pol::Acc v,
                                                           typename Pol::Acc &last) {
  using Acc = typename Pol::Acc;
  const int lane = threadIdx.x & 31;
  Acc inc = v;
  int f = flag;
  // Hillis-Steele doubling, stopped as soon as every lane's sum reaches back
  // to a lane that finished a row (usually after one or two steps); each
  // step costs one warp-wide FP64 add.
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (__all_sync(0xffffffffu, f || lane < o)) break;
    Acc u = Pol::shfl_up(inc, o);
    int fu = __shfl_up_sync(0xffffffffu, f, o);
    if (lane >= o) {
      if (!f) inc = Pol::combine(u, inc);
      f |= fu;
    }
  }
  Acc ex = Pol::shfl_up(inc, 1);
  if (lane == 0) ex = Pol::zero();
  last = Pol::shfl(inc, 31);
  return ex;
}

// first index in s[0, n) with s[i] > key (s ascending)
__device__ __forceinline__ int upper_bound_smem(const int32_t *s, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s[mid] <= key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// register type of a loaded value: bf16 values widen to float
template <class V>
struct LoadT {
  using type = V;
};
template <>
struct LoadT<bf16_t> {
  using type = float;
};

// ---------------------------------------------------------------------------
// group sources: 8 aligned consecutive elements from global memory (direct
// 256-bit loads) or from a shared-memory stage filled by bulk copies
// ---------------------------------------------------------------------------

// One group of 8 nonzeros starting at g8 (a multiple of 8): a single vector
// load, or element-wise loads for the last group of the array.
template <class T, class U>
__device__ __forceinline__ void load_group(const T *arr, int64_t g8, int64_t nnz, U (&out)[8]) {
  if (g8 + 8 <= nnz) {
    ld8(arr + g8, out);
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) out[u] = (g8 + u < nnz) ? U(ld_stream(arr + g8 + u)) : U(0);
  }
}

__device__ __forceinline__ void lds8(const int32_t *p, int32_t (&r)[8]) {
  const int4 a = reinterpret_cast<const int4 *>(p)[0], b = reinterpret_cast<const int4 *>(p)[1];
  r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
  r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}
__device__ __forceinline__ void lds8(const double *p, double (&v)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 d = reinterpret_cast<const double2 *>(p)[i];
    v[2 * i] = d.x;
    v[2 * i + 1] = d.y;
  }
}
__device__ __forceinline__ void lds8(const float *p, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void lds8(const bf16_t *p, float (&v)[8]) {
  const uint4 w = *reinterpret_cast<const uint4 *>(p);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(ws[i] << 16);
    v[2 * i + 1] = __uint_as_float(ws[i] & 0xffff0000u);
  }
}

// An array as seen by a tile: element e lives at p[e - base].
template <class T>
struct Seg {
  const T *p;
  int64_t base;
};

struct GlobalSrc {
  template <class T, class U>
  __device__ __forceinline__ void group(Seg<T> s, int64_t g8, int64_t nnz, U (&out)[8]) const {
    load_group(s.p, g8, nnz, out);
  }
};

struct SharedSrc {
  template <class T, class U>
  __device__ __forceinline__ void group(Seg<T> s, int64_t g8, int64_t, U (&out)[8]) const {
    lds8(s.p + (g8 - s.base), out);
  }
};

// The lanes of a warp split the 8-aligned groups that cover the tile's
// nonzeros [k0, k1) evenly (Alg. 2's floor(i*n/P) rule over groups); lane
// `lane` owns groups [glo, ghi) and nonzeros [ka, kb) = their intersection
// with [k0, k1).  Lane ranges are contiguous and cover [k0, k1) in order.
struct LaneRange {
  int64_t glo, ghi, ka, kb;
};
__device__ __forceinline__ LaneRange lane_range(int64_t k0, int64_t k1, int lane) {
  const int64_t gA = k0 >> 3, ng = ((k1 + 7) >> 3) - gA;
  LaneRange r;
  r.glo = gA + ((lane * ng) >> 5);
  r.ghi = gA + (((lane + 1) * ng) >> 5);
  r.ka = min(max(k0, r.glo << 3), k1);
  r.kb = min(max(k0, r.ghi << 3), k1);
  return r;
}

// The tiles warp `wid` of this block walks: by default tiles wid + 8 k,
// wid + 8 k + 8 G, ... over all T tiles (block k of G blocks), so every
// partition's tiles spread over the whole grid; with one block per
// partition, block i walks tiles [toff_i, toff_{i+1}) of partition i only.
struct TileWalk {
  int first, end, step;
};
__device__ __forceinline__ TileWalk tile_walk(int T, int warps, const int32_t *part_toff) {
  const int wid = threadIdx.x >> 5;
  if (part_toff)
    return TileWalk{__ldg(part_toff + blockIdx.x) + wid, __ldg(part_toff + blockIdx.x + 1), warps};
  return TileWalk{static_cast<int>(blockIdx.x) * warps + wid, T,
                  static_cast<int>(gridDim.x) * warps};
}

// ---------------------------------------------------------------------------
// CSR tile
// ---------------------------------------------------------------------------

template <class Pol>
struct CsrArgs {
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  typename Pol::X *y;
  double alpha, beta;
  int finish;               // kFinish*
  const int32_t *tile_row;  // [T+1]
  const int32_t *tile_k;    // [T+1]
  double *head, *tail;      // [T] FP64 partials of rows split between tiles
  int32_t m;
  unsigned comp_mode;
  int *err;                 // device error word
  const int32_t *part_toff; // one block per partition: its first tile, or null
};

template <class Pol>
__device__ __forceinline__ void write_row(const CsrArgs<Pol> &a, int32_t row,
                                          typename Pol::Acc v) {
  a.y[row] = Pol::finish(v, a.finish, a.alpha, a.beta, a.y + row);
}

// One merge-path tile b = rows [r0, r1] x nonzeros [k0, k1), processed by
// one warp.  rp[j] = row_ptr[r0 + j] for j = 0..r1-r0, and also j = r1-r0+1
// when r1 < m; rp must be in shared memory (it is searched).
// cf (low-precision form, optional): this warp's nrows + 1 bytes of shared
// memory for the tile's per-row compensation flags, filled once here by all
// lanes; the row-finishing path, which the lanes of a warp reach at
// different steps, then reads one byte instead of recomputing the predicate.
// kCopy: the caller knows that alpha = 1 and beta = 0 (every row finished
// by the copy mode, decided at compile time).
template <class Pol, class Src, bool kCopy = false>
__device__ __forceinline__ void csr_tile_compute(const CsrArgs<Pol> &a, int b, int32_t r0,
                                                 int32_t k0, int32_t r1, int32_t k1,
                                                 const int32_t *rp, Seg<int32_t> col,
                                                 Seg<typename Pol::V> val, int64_t nnz,
                                                 Src src, uint8_t *cf = nullptr) {
  using Acc = typename Pol::Acc;
  using LV = typename LoadT<typename Pol::V>::type;
  const int lane = threadIdx.x & 31;
  const int fin = kCopy ? int(kFinishCopy) : a.finish;
  auto write_row_k = [&](int32_t row, Acc v) {
    a.y[row] = Pol::finish(v, fin, a.alpha, a.beta, a.y + row);
  };
  const int nrows = r1 - r0;
  const int32_t rs0 = rp[0];
  const int32_t *s_end = rp + 1;  // s_end[i]: end of row r0 + i
  const bool flag = rs0 < k0;     // the first row started in an earlier tile

  const LaneRange lr = lane_range(k0, k1, lane);
  const int32_t ka = static_cast<int32_t>(lr.ka), kb = static_cast<int32_t>(lr.kb);
  // rows finished by this lane: ends in (ka, kb], plus ends <= k0 for lane 0
  int r = lane == 0 ? 0 : upper_bound_smem(s_end, nrows, ka);
  const int r_end = upper_bound_smem(s_end, nrows, kb);
  int32_t next_end = r < r_end ? s_end[r] : INT32_MAX;

  // compensation predicate (low-precision form only)
  int32_t re_last = 0;
  if (Pol::kLow) re_last = (r1 < a.m) ? rp[nrows + 1] : k1;
  auto row_comp_of = [&](int rr) -> bool {
    int64_t st = rr == 0 ? int64_t(rs0) : int64_t(s_end[rr - 1]);
    int64_t en = rr < nrows ? int64_t(s_end[rr]) : int64_t(re_last);
    return want_comp(a.comp_mode, en - st, (rr == 0 && flag) || rr == nrows);
  };
  if (Pol::kLow && cf) {
    for (int rr = lane; rr <= nrows; rr += 32) cf[rr] = row_comp_of(rr);
    __syncwarp();
  }
  auto row_comp = [&](int rr) -> bool {
    if (!Pol::kLow) return false;
    return cf ? cf[rr] != 0 : row_comp_of(rr);
  };

  Acc acc = Pol::zero(), first_acc = Pol::zero();
  bool emitted = false, comp = row_comp(r);
  int first_r = 0;
  // finish every row whose end is <= kk (several when rows are empty)
  auto finish_rows = [&](int32_t kk) {
    while (next_end <= kk) {
      if (!emitted) {
        emitted = true;
        first_r = r;
        first_acc = acc;
      } else {
        write_row_k(r0 + r, acc);
      }
      acc = Pol::zero();
      ++r;
      next_end = r < r_end ? s_end[r] : INT32_MAX;
      comp = row_comp(r);
    }
  };
  finish_rows(ka);

  for (int64_t g = lr.glo; g < lr.ghi; ++g) {
    const int64_t g8 = g << 3;
    int32_t c[8];
    LV v[8];
    typename Pol::X xv[8];
    src.group(col, g8, nnz, c);
    src.group(val, g8, nnz, v);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = g8 + u >= ka && g8 + u < kb;
      xv[u] = in ? load_x(a.x, c[u]) : typename Pol::X(0);
      if (!in) v[u] = LV(0);
    }
    // One multiply-add per element on every lane (masked elements add 0),
    // so the FP64 instructions of a warp never diverge; row ends branch
    // only around FP64-free code.  Positions outside the lane's range never
    // finish a row: rows ending at or before ka were finished above, and
    // r stops at r_end.
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      acc = Pol::fma(acc, v[u], xv[u], comp);
      const int32_t kk = static_cast<int32_t>(g8 + u + 1);
      if (next_end <= kk) finish_rows(kk);
    }
  }

  Acc last;
  const Acc carry = warp_seg_scan<Pol>(emitted, acc, last);
  if (emitted) {
    const Acc tot = Pol::combine(carry, first_acc);
    if (first_r == 0 && flag)
      a.head[b] = Pol::to_f64(tot);
    else
      write_row_k(r0 + first_r, tot);
  }
  if (lane == 31) {
    if (nrows == 0) {
      if (flag)
        a.head[b] = Pol::to_f64(last);
      else if (k1 > k0)
        a.tail[b] = Pol::to_f64(last);
    } else if (k1 > rp[nrows]) {
      a.tail[b] = Pol::to_f64(last);
    }
  }
}

// ---------------------------------------------------------------------------
// COO tile (rows sorted)
// ---------------------------------------------------------------------------

template <class Pol>
struct CooArgs {
  const int32_t *row_idx;
  const int32_t *col_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  typename Pol::X *y;
  double alpha, beta;
  int finish;
  const int32_t *start_idx, *end_idx;  // partition metadata (Alg. 6)
  int32_t np, G, m;
  int64_t nnz;
  double *head, *tail;
  unsigned comp_mode;
  int *err;
  bool per_part;  // one block per partition (tiles i*G .. i*G+G-1)
};

// nonzero range of COO tile b: sub-range g of partition i (Alg. 2's split
// applied inside the partition)
template <class Pol>
__device__ __forceinline__ void coo_tile_range(const CooArgs<Pol> &a, int b, int32_t &k0,
                                               int32_t &k1) {
  const int i = b / a.G, g = b % a.G;
  const int64_t s = __ldg(a.start_idx + i), L = int64_t(__ldg(a.end_idx + i)) - s + 1;
  k0 = static_cast<int32_t>(s + (int64_t(g) * L) / a.G);
  k1 = static_cast<int32_t>(s + (int64_t(g + 1) * L) / a.G);
}

// In-tile length of the run of row rv around nonzero j of a row-sorted
// COO tile [k0, k1), or 0 when two probes 128 positions either side of j
// both miss rv (the run is then shorter than 256).  Out of line: a lane
// calls it for a few runs at most, and inlined at every call site it made
// the low-precision COO kernel wait on instruction fetch.
static __device__ __noinline__ int64_t coo_run_length(const int32_t *row_idx, int64_t k0,
                                                      int64_t k1, int32_t rv, int64_t j) {
  const int64_t pa = max(k0, j - 128), pb = min(k1 - 1, j + 128);
  const bool reach_a = pa < j && __ldg(row_idx + pa) == rv;
  const bool reach_b = pb > j && __ldg(row_idx + pb) == rv;
  if (!reach_a && !reach_b) return 0;
  int64_t lo = k0, hi = j;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(row_idx + mid) < rv) lo = mid + 1; else hi = mid;
  }
  const int64_t st = lo;
  lo = j;
  hi = k1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(row_idx + mid) <= rv) lo = mid + 1; else hi = mid;
  }
  return lo - st;
}

// kCopy: the caller knows that alpha = 1 and beta = 0, so every row is
// finished by the copy mode (compile-time: the finishing code shrinks to
// that case, which keeps the low-precision kernel's loop in the
// instruction cache).
template <class Pol, class Src, bool kCopy = false>
__device__ __forceinline__ void coo_tile_compute(const CooArgs<Pol> &a, int b, int32_t k0,
                                                 int32_t k1, Seg<int32_t> row,
                                                 Seg<int32_t> col, Seg<typename Pol::V> val,
                                                 Src src) {
  using Acc = typename Pol::Acc;
  using LV = typename LoadT<typename Pol::V>::type;
  const int lane = threadIdx.x & 31;
  const int fin = kCopy ? int(kFinishCopy) : a.finish;
  auto write_row = [&](int32_t row, Acc v) {
    a.y[row] = Pol::finish(v, fin, a.alpha, a.beta, a.y + row);
  };
  auto write_empty = [&](int32_t row) {
    a.y[row] = Pol::finish(Pol::zero(), fin, a.alpha, a.beta, a.y + row);
  };
  if (lane == 0) {
    a.head[b] = 0.0;
    a.tail[b] = 0.0;
  }
  __syncwarp();
  if (k1 == k0) return;  // uniform across the warp
  const int32_t prev_row = k0 > 0 ? __ldg(a.row_idx + k0 - 1) : -1;
  const int32_t next_row = k1 < a.nnz ? __ldg(a.row_idx + k1) : a.m;
  const int32_t first_row = __ldg(a.row_idx + k0), last_row = __ldg(a.row_idx + k1 - 1);
  const bool flag = prev_row == first_row;
  const bool cont = next_row == last_row;

  if (k0 == 0)
    for (int32_t rr = lane; rr < first_row; rr += 32) write_empty(rr);

  const LaneRange lr = lane_range(k0, k1, lane);
  const int64_t ka = lr.ka, kb = lr.kb;

  // compensation predicate of the run of row rv that contains nonzero j:
  // split if it touches a tile end that the row crosses (rows are sorted,
  // so it touches the tile's start iff rv is the tile's first row), long if
  // its length inside the tile exceeds 256 (coo_run_length; a split run is
  // caught first, so the length test alone decides the rest).  A row that
  // crosses the tile is split anyway; inside the tile, its in-tile length
  // is its full length.
  auto run_comp = [&](int32_t rv, int64_t j) -> bool {
    if (!Pol::kLow) return false;
    if (a.comp_mode & (MSREP_COMP_ALL | MSREP_COMP_NONE))
      return want_comp(a.comp_mode, 0, false);
    const bool split = (rv == first_row && flag) || (rv == last_row && cont);
    if (split) return true;
    return coo_run_length(a.row_idx, k0, k1, rv, j) > 256;
  };

  // A lane whose range holds at most 256 nonzeros needs the predicate for
  // two runs at most: every run it both starts and ends is shorter than 257
  // and touches neither tile end, so only its first and last runs (the rows
  // at ka and kb - 1) can be long or split.  Those two are settled here,
  // before the nonzero loop, instead of at each row change inside it.
  const bool two_runs = Pol::kLow && kb - ka <= 256;
  bool comp_first = false, comp_last = false;
  int32_t row_first = -1, row_last = -1;
  if (two_runs && kb > ka) {
    row_first = __ldg(a.row_idx + ka);
    row_last = __ldg(a.row_idx + kb - 1);
    comp_first = run_comp(row_first, ka);
    comp_last = row_last == row_first ? comp_first : run_comp(row_last, kb - 1);
  }
  const bool comp_mid = Pol::kLow && want_comp(a.comp_mode, 0, false);
  auto comp_of = [&](int32_t rv, int64_t j) -> bool {
    if (!two_runs) return run_comp(rv, j);
    return rv == row_first ? comp_first : rv == row_last ? comp_last : comp_mid;
  };

  Acc acc = Pol::zero(), first_acc = Pol::zero();
  bool emitted = false, comp = false;
  int32_t first_r = 0, cur = -1, lane_next = -1;
  auto emit = [&]() {
    if (!emitted) {
      emitted = true;
      first_r = cur;
      first_acc = acc;
    } else {
      write_row(cur, acc);
    }
    acc = Pol::zero();
  };
  for (int64_t gg = lr.glo; gg < lr.ghi; ++gg) {
    const int64_t g8 = gg << 3;
    int32_t rw[8], c[8];
    LV v[8];
    typename Pol::X xv[8];
    src.group(row, g8, a.nnz, rw);
    src.group(col, g8, a.nnz, c);
    src.group(val, g8, a.nnz, v);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = g8 + u >= ka && g8 + u < kb;
      xv[u] = in ? load_x(a.x, c[u]) : typename Pol::X(0);
      if (!in) v[u] = LV(0);
    }
    const int ulo = static_cast<int>(max(ka - g8, int64_t(0)));
    const int uhi = static_cast<int>(min(kb - g8, int64_t(8))) - 1;
    // row of the nonzero right after the lane's range, if it is in this group
    if (kb < k1 && kb - g8 >= 0 && kb - g8 < 8) lane_next = rw[kb - g8];
    // row changes branch around FP64-free code; the multiply-adds are the
    // same instructions on every lane (masked elements add 0)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u >= ulo && u <= uhi && rw[u] != cur) {
        if (cur >= 0) {
          emit();
          for (int32_t rr = cur + 1; rr < rw[u]; ++rr) write_empty(rr);
        }
        cur = rw[u];
        comp = comp_of(cur, g8 + u);
      }
      acc = Pol::fma(acc, v[u], xv[u], comp);
    }
  }
  // the lane's last run ends here if the next nonzero starts another row
  if (kb > ka) {
    int32_t nxt = next_row;
    if (kb < k1) nxt = (lane_next >= 0) ? lane_next : __ldg(a.row_idx + kb);
    if (nxt != cur) {
      emit();
      if (kb < k1)
        for (int32_t rr = cur + 1; rr < nxt; ++rr) write_empty(rr);
    }
  }

  Acc last;
  const Acc carry = warp_seg_scan<Pol>(emitted, acc, last);
  if (emitted) {
    const Acc tot = Pol::combine(carry, first_acc);
    if (first_r == first_row && flag)
      a.head[b] = Pol::to_f64(tot);
    else
      write_row(first_r, tot);
  }
  if (lane == 31 && cont) {
    if (last_row == first_row && flag)
      a.head[b] = Pol::to_f64(last);
    else
      a.tail[b] = Pol::to_f64(last);
  }
  // empty rows between this tile's last row and the next tile's first row
  if (!cont)
    for (int32_t rr = last_row + 1 + lane; rr < next_row; rr += 32) write_empty(rr);
}

// ---------------------------------------------------------------------------
// CSC tile: scatter-add into an FP64 accumulator (y itself on the FP64 path)
// ---------------------------------------------------------------------------

template <class Pol>
struct CscArgs {
  const int32_t *col_ptr;
  const int32_t *row_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  double *yacc;  // scatter target by row: y (FP64) or the FP64 accumulator
  double *yperm;  // permuted accumulator (pmask + 1 entries), or null
  uint32_t pmask;
  double scale;  // alpha on the FP64 path, 1 when a finishing pass follows
  bool scaled;   // scale != 1
  const int32_t *tile_row, *tile_k;
  const int32_t *hot;   // hub rows: count, then kMaxHot rows (-1 = none)
  const unsigned long long *warm;  // frequent-row table, kWarm entries
  int32_t n;
  int *err;
  const int32_t *part_toff;  // one block per partition: its first tile, or null
};

// A skewed CSC matrix (hub rows found and a permuted accumulator given)
// takes the frequent-row sums (WarmRows; the bulk-copy streaming kernel
// keeps the hub-row sums of HotRows) and the permuted scatter.
__device__ __forceinline__ bool csc_skewed(const int32_t *hot, const double *yperm) {
  return yperm != nullptr && __ldg(hot) > 0;
}

// Private sums of the hub rows of a CSC matrix (the bulk-copy streaming
// kernel; the direct kernels use WarmRows, below).  Every nonzero of a hub row
// is an atomic add to the same y entry, and same-address atomics serialise
// in L2 (about 40,000 of them on one row of the R-MAT workload cost some
// 100 us).  A warp adds its products for the hub rows to its own slots in
// shared memory instead (shared-memory atomics, rarely contended: hub
// nonzeros are a small fraction of all); the block adds its slots to y once,
// at the end.
struct HotRows {
  static_assert(kMaxHot == 4, "HotRows holds four rows");
  int32_t r0, r1, r2, r3;
  int n;
  double *slot;  // this warp's kMaxHot sums in shared memory
  __device__ __forceinline__ void load(const int32_t *hot, double (*s_hot)[kMaxHot]) {
    n = __ldg(hot);
    r0 = __ldg(hot + 1);
    r1 = __ldg(hot + 2);
    r2 = __ldg(hot + 3);
    r3 = __ldg(hot + 4);
    slot = s_hot[threadIdx.x >> 5];
    if ((threadIdx.x & 31) < kMaxHot) slot[threadIdx.x & 31] = 0.0;
    __syncwarp();
  }
  // adds v to the warp's sum of `row` if it is a hub row
  __device__ __forceinline__ bool take(int32_t row, double v) {
    const int j = row == r0 ? 0 : row == r1 ? 1 : row == r2 ? 2 : row == r3 ? 3 : -1;
    if (j < 0) return false;
    atomicAdd(slot + j, v);
    return true;
  }
  // Called by every thread of the block after its last tile: adds the
  // block's sums to the permuted accumulator.
  __device__ __forceinline__ void flush(double *yperm, uint32_t pmask, double (*s_hot)[kMaxHot]) {
    __syncthreads();
    const int j = threadIdx.x;
    const int32_t row = j == 0 ? r0 : j == 1 ? r1 : j == 2 ? r2 : j == 3 ? r3 : -1;
    if (row >= 0) {
      double t = 0.0;
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t = __dadd_rn(t, s_hot[w][j]);
      atomicAdd(yperm + perm_slot(row, pmask), t);
    }
  }
};

// Sums of the frequent rows of a skewed scatter (see kWarm): one
// direct-mapped table per thread block in shared memory, its row tags
// copied from the plan.  Each warp adds its products for the tabled rows to
// the block's slots with shared-memory atomics; the block adds every
// non-zero slot to the permuted accumulator once, at its end.  The hub rows
// hold slots of their own, so this also does what HotRows does.
struct WarmRows {
  int32_t *tag;  // kWarm row tags, row + 1 (0 = empty), shared memory
  double *acc;   // kWarm sums, shared memory
  // every thread of the block; warm: the plan's table, (priority << 32) |
  // ~row per slot, 0 = empty
  __device__ __forceinline__ void load(const unsigned long long *warm, int32_t *s_tag,
                                       double *s_acc) {
    tag = s_tag;
    acc = s_acc;
    for (int i = threadIdx.x; i < kWarm; i += blockDim.x) {
      const unsigned long long e = __ldg(warm + i);
      s_tag[i] = e ? static_cast<int32_t>(~static_cast<uint32_t>(e)) + 1 : 0;
      s_acc[i] = 0.0;
    }
    __syncthreads();
  }
  __device__ __forceinline__ bool take(int32_t row, double v) {
    const uint32_t s = warm_slot(row);
    if (tag[s] != row + 1) return false;
    atomicAdd(acc + s, v);
    return true;
  }
  // every thread of the block, after its last tile
  __device__ __forceinline__ void flush(double *yperm, uint32_t pmask) {
    __syncthreads();
    for (int i = threadIdx.x; i < kWarm; i += blockDim.x) {
      const int32_t row = tag[i] - 1;
      if (row >= 0 && acc[i] != 0.0) atomicAdd(yperm + perm_slot(row, pmask), acc[i]);
    }
  }
};

// Where a scatter's products go (Alg. 5's column merge, done in place).
// DirectSink: one FP64 atomic add per product into the row-ordered target.
struct DirectSink {
  double *y;
  __device__ __forceinline__ void add(int32_t row, double v) const { atomicAdd(y + row, v); }
};

// A skewed matrix: the hub or frequent rows' sums in shared memory (Hot is
// HotRows or WarmRows), the other rows into the permuted accumulator.
template <class Hot>
struct SkewSink {
  Hot *hot;
  double *yperm;
  uint32_t pmask;
  __device__ __forceinline__ void add(int32_t row, double v) const {
    if (!hot->take(row, v)) atomicAdd(yperm + perm_slot(row, pmask), v);
  }
};

// cp[j] = col_ptr[c0 + j], j = 0..c1-c0, in shared memory; xat(j) = scale *
// x[c0 + j] for the columns that hold nonzeros of the tile.  Every product
// goes to sink.add(row, product).  The lanes split the tile's nonzeros
// evenly, so long columns spread over the warp.
template <class Pol, class Src, class Sink, class XAt>
__device__ __forceinline__ void csc_tile_compute(const CscArgs<Pol> &a, int32_t c0, int32_t k0,
                                                 int32_t c1, int32_t k1, const int32_t *cp,
                                                 XAt xat, Seg<int32_t> row,
                                                 Seg<typename Pol::V> val, int64_t nnz, Src src,
                                                 const Sink &sink) {
  using LV = typename LoadT<typename Pol::V>::type;
  const int lane = threadIdx.x & 31;
  const int ncols = c1 - c0;
  const int32_t *s_end = cp + 1;
  const LaneRange lr = lane_range(k0, k1, lane);
  const int64_t ka = lr.ka, kb = lr.kb;
  int c = upper_bound_smem(s_end, ncols, static_cast<int32_t>(ka));
  int32_t cend = c < ncols ? s_end[c] : INT32_MAX;
  // x of the current column, reloaded only when the column changes (xat has
  // a value for every column index c <= ncols that holds nonzeros of the
  // tile)
  double xc = xat(c);
  for (int64_t gg = lr.glo; gg < lr.ghi; ++gg) {
    const int64_t g8 = gg << 3;
    int32_t rw[8];
    LV v[8];
    src.group(row, g8, nnz, rw);
    src.group(val, g8, nnz, v);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t e = g8 + u;
      const bool in = e >= ka && e < kb;
      if (in && cend <= e) {  // integer-only column advance
        do {
          ++c;
          cend = c < ncols ? s_end[c] : INT32_MAX;
        } while (cend <= e);
        xc = xat(c);
      }
      double vw;
      if constexpr (Pol::kLow)
        vw = widen(v[u]);  // integer widening: off the FP64 pipe
      else
        vw = double(v[u]);
      const double prod = __dmul_rn(vw, in ? xc : 0.0);
      if (in) sink.add(rw[u], prod);
    }
  }
}

// Nonzeros [kb, ke) of tile column j (column c0 + j < n) inside the tile's
// range [k0, k1).  cp holds col_ptr[c0 .. c1]; the last column c1 ends at
// k1 (a merge-path coordinate has col_ptr[c1] <= k1 <= col_ptr[c1 + 1]).
__device__ __forceinline__ void csc_col_range(int j, int32_t c0, int32_t k0, int32_t c1,
                                              int32_t k1, const int32_t *cp, int32_t &kb,
                                              int32_t &ke) {
  kb = max(cp[j], k0);
  ke = c0 + j < c1 ? min(cp[j + 1], k1) : k1;
}

// Longest column of a CSC tile inside its nonzero range [k0, k1) (every
// lane of the warp gets it).  cp as for csc_tile_compute.
__device__ __forceinline__ int csc_tile_max_col(int32_t c0, int32_t k0, int32_t c1, int32_t k1,
                                                int32_t n, const int32_t *cp) {
  const int lane = threadIdx.x & 31;
  int longest = 0;
  for (int j = lane; j <= c1 - c0 && c0 + j < n; j += 32) {
    int32_t kb, ke;
    csc_col_range(j, c0, k0, c1, k1, cp, kb, ke);
    longest = max(longest, ke - kb);
  }
  return __reduce_max_sync(0xffffffffu, longest);
}

// CSC tiles of short columns, lane-interleaved: step i of the warp takes
// the tile's nonzeros k0 + 32 i + lane, so every load instruction reads 32
// consecutive elements (one or two 128-byte lines) and every atomic add
// covers the rows of a few neighbouring columns.  In a banded matrix those
// rows fall in a few short runs (a 2D Laplacian's 32 consecutive nonzeros,
// about six columns, add into three runs of about eight rows), so one
// warp-wide atomic add touches a few 32-byte sectors of y instead of 32
// scattered ones; on GB300 the L2 takes such coalesced FP64 adds far faster
// than scattered ones, and the add itself stays in L2 (the SM's FP64 pipe,
// about two lane operations per clock, does only the multiply).  The
// column of each nonzero comes from colof (this warp's 32 * IPT + 8 int16
// entries of shared memory), filled first by a walk of the tile's columns
// (one lane per column: the tile's columns must be short, see
// csc_tile_max_col).  Low-precision values and x are widened to FP64 with
// integer operations (widen).  Seven steps are loaded ahead (eight spill registers
// at four resident blocks; four keep too few loads in flight).
// kUnscaled: the caller knows a.scaled is false (alpha = 1 on the FP64
// path), so the scaling multiply is left out at compile time.
template <class Pol, class Sink, bool kUnscaled = false>
__device__ __forceinline__ void csc_tile_interleaved(const CscArgs<Pol> &a, int32_t c0,
                                                     int32_t k0, int32_t c1, int32_t k1,
                                                     const int32_t *cp, const Sink &sink,
                                                     int16_t *colof) {
  using LV = typename LoadT<typename Pol::V>::type;
  constexpr int B = 7;
  const int lane = threadIdx.x & 31;
  const int ncols = c1 - c0 + 1;
  for (int j = lane; j < ncols && c0 + j < a.n; j += 32) {
    int32_t kb, ke;
    csc_col_range(j, c0, k0, c1, k1, cp, kb, ke);
    for (int32_t k = kb; k < ke; ++k) colof[k - k0] = static_cast<int16_t>(j);
  }
  __syncwarp();
  const int32_t len = k1 - k0;
  for (int32_t i0 = 0; i0 < len; i0 += 32 * B) {
    int32_t rw[B];
    LV v[B];
    if constexpr (Pol::kLow && std::is_same<Sink, DirectSink>::value) {
      // all B steps' loads first; x is widened (with its rare out-of-line
      // case) only in the second loop, so that no load waits for another
      // (Laplacian FP32 137 -> 113 us).  With the frequent-row sums the
      // widening stays with the loads: deferred, it took R-MAT from 131 to
      // 143 us.
      typename Pol::X xr[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int32_t p = i0 + 32 * u + lane;
        const bool in = p < len;
        rw[u] = in ? ld_stream(a.row_idx + k0 + p) : 0;
        v[u] = in ? LV(ld_stream(a.val + k0 + p)) : LV(0);
        xr[u] = in ? load_x(a.x, c0 + colof[p]) : typename Pol::X(0);
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (i0 + 32 * u >= len) break;  // warp-uniform
        // the low-precision form applies alpha in its finishing pass
        // (a.scaled is false), so no scaling multiply here
        const double prod = __dmul_rn(widen(v[u]), widen(xr[u]));
        if (i0 + 32 * u + lane < len) sink.add(rw[u], prod);
      }
    } else {
      double xv[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int32_t p = i0 + 32 * u + lane;
        const bool in = p < len;
        rw[u] = in ? ld_stream(a.row_idx + k0 + p) : 0;
        v[u] = in ? LV(ld_stream(a.val + k0 + p)) : LV(0);
        xv[u] = in ? widen(load_x(a.x, c0 + colof[p])) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < B; ++u) {
        if (i0 + 32 * u >= len) break;  // warp-uniform
        double xs = xv[u];
        if constexpr (!Pol::kLow && !kUnscaled) xs = a.scaled ? __dmul_rn(xv[u], a.scale) : xv[u];
        const double prod = __dmul_rn(widen(v[u]), xs);
        if (i0 + 32 * u + lane < len) sink.add(rw[u], prod);
      }
    }
  }
}

// Stages the tile's column pointers and (scaled) x values in shared memory:
// cp[j] = col_ptr[c0 + j] for j = 0..min(c1 + 1, n + 1) - c0 - 1 and
// xs[j] = scale * x[c0 + j] for columns c0 + j < n.
template <class Pol>
__device__ __forceinline__ void csc_stage_x(const CscArgs<Pol> &a, int32_t c0, int32_t c1,
                                            double *xs) {
  const int lane = threadIdx.x & 31;
  const int32_t xe = min(c1 + 1, a.n);
  for (int32_t c = c0 + lane; c < xe; c += 32) {
    const double xv = double(load_x(a.x, c));
    xs[c - c0] = a.scaled ? __dmul_rn(xv, a.scale) : xv;
  }
}

// ---------------------------------------------------------------------------
// fix-up of rows split between tiles, merged in tile (= partition) order
// ---------------------------------------------------------------------------

// alpha * s + beta * y_in for a row merged in FP64 (split rows), with the
// rounding spelled out so that every kernel that merges rows (one vector or
// k of them) rounds alike: one product when beta = 0, else
// fma(alpha, s, beta * y_in).
__device__ __forceinline__ double finish_merged(double s, double alpha, double beta,
                                                double yo) {
  return beta == 0.0 ? __dmul_rn(alpha, s) : __fma_rn(alpha, s, __dmul_rn(beta, yo));
}

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

// Merge of one row split between tiles (Sec. 3.2.1 / Sec. 4.3): the first
// tile whose first row started earlier sums, in tile order, the tail partial
// of the previous tile and the head partials of the run of tiles that
// continue the row, then applies alpha and beta once, in FP64.

// Is tile b the first of a run continuing row r from tile b - 1?
template <class View>
__device__ __forceinline__ bool fixup_run_start(const View &v, int T, int b, int32_t &r) {
  if (b <= 0 || b >= T) return false;
  bool f;
  v.row_flag(b, r, f);
  if (!f) return false;
  int32_t rp;
  bool fp;
  v.row_flag(b - 1, rp, fp);
  return !(fp && rp == r);  // else not the first flagged tile of the run
}

// Adds, in order, the head partials of tiles j0 .. j0+7 that continue row r
// to s; returns how many continued it (8: the run may go on).  The flags
// and partials of the 8 tiles are loaded together (a hub row spans dozens
// of tiles; one dependent load chain per tile made the walk latency-bound).
template <class View>
__device__ __forceinline__ int fixup_chunk(const View &v, int T, int j0, int32_t r,
                                           const double *head, double &s) {
  int32_t rj[8];
  bool fj[8];
  double hj[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    fj[u] = false;
    if (j0 + u < T) {
      v.row_flag(j0 + u, rj[u], fj[u]);
      hj[u] = head[j0 + u];
    }
  }
  int run = 8;
#pragma unroll
  for (int u = 7; u >= 0; --u)
    if (!(fj[u] && rj[u] == r)) run = u;
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (u < run) s += hj[u];
  return run;
}

template <class X>
__device__ __forceinline__ void fixup_write(X *y, int32_t r, double s, double alpha,
                                            double beta) {
  y[r] = static_cast<X>(finish_merged(s, alpha, beta, beta == 0.0 ? 0.0 : double(y[r])));
}

// One thread, tile b.
template <class X, class View>
__device__ __forceinline__ void fixup_tile(const View &v, int T, int b, const double *head,
                                           const double *tail, X *y, double alpha,
                                           double beta) {
  int32_t r;
  if (!fixup_run_start(v, T, b, r)) return;
  double s = tail[b - 1];
  for (int j0 = b; fixup_chunk(v, T, j0, r, head, s) == 8; j0 += 8) {
  }
  fixup_write(y, r, s, alpha, beta);
}

// One warp, tiles base .. base+31 (one per lane).  A run longer than one
// chunk is continued by the whole warp, 32 tiles per step, its partials
// added in tile order by every lane, so the sum (and y) is bit-identical to
// fixup_tile's.
template <class X, class View>
__device__ __forceinline__ void fixup_warp(const View &v, int T, int base, const double *head,
                                           const double *tail, X *y, double alpha,
                                           double beta) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int b = base + lane;
  int32_t r = -1;
  double s = 0.0;
  bool more = false;
  if (fixup_run_start(v, T, b, r)) {
    s = tail[b - 1];
    more = fixup_chunk(v, T, b, r, head, s) == 8;
    if (!more) fixup_write(y, r, s, alpha, beta);
  }
  unsigned pend = __ballot_sync(full, more);
  while (pend) {
    const int src = __ffs(pend) - 1;
    pend &= pend - 1;
    const int32_t rr = __shfl_sync(full, r, src);
    double ss = __shfl_sync(full, s, src);
    for (int j0 = __shfl_sync(full, b, src) + 8;; j0 += 32) {
      const int j = j0 + lane;
      bool in = false;
      double h = 0.0;
      if (j < T) {
        int32_t rj;
        bool fj;
        v.row_flag(j, rj, fj);
        in = fj && rj == rr;
        if (in) h = head[j];
      }
      const unsigned im = __ballot_sync(full, in);
      const int cnt = im == full ? 32 : __ffs(~im) - 1;
      for (int u = 0; u < cnt; ++u) ss += __shfl_sync(full, h, u);
      if (cnt < 32) break;
    }
    if (lane == src) fixup_write(y, rr, ss, alpha, beta);
  }
}

}  // namespace msrep
