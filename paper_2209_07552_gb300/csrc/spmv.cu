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
#include <map>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "spmv_core.cuh"

namespace msrep {

msrep_status check_matrix(const msrep_matrix *A);
int32_t effective_tile(int32_t tile);

// device error word of the streaming kernels (see msrep_device_status)
static __device__ int g_kernel_err = 0;

int *kernel_err_ptr() {
  static std::mutex mu;
  static int *cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!cached[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_kernel_err) != cudaSuccess) return nullptr;
    cached[dev] = static_cast<int *>(p);
  }
  return cached[dev];
}

// ---------------------------------------------------------------------------
// single-matrix kernels.  A grid of (resident blocks x SMs) walks the tiles;
// warp w of block k takes tiles w + 8k, w + 8k + 8*gridDim.x, ...
//
// Streaming variant (MSREP_STREAM_TMA): each warp keeps S tiles in flight.  Lane 0
// issues bulk copies (TMA, cp.async.bulk) of a tile's row_ptr segment and
// its nonzero arrays into one of the warp's S shared-memory stages; an
// mbarrier per stage counts the bytes; the warp computes on stage i while
// stages i+1..i+S-1 are being filled.  The nonzero stream therefore never
// passes through L1, which is left to the x gathers.
// Direct variant (default): no staging; each lane reads its groups with
// 256-bit global loads that bypass L1.  On GB300 the SpMV is bound by the
// x gathers (one L1 line lookup each, and an L2 sector request on a miss)
// and the FP64 pipe, not by DRAM latency; the direct variant keeps more
// warps resident and more of L1 for x.
// ---------------------------------------------------------------------------

// Minimum resident blocks per SM asked of the register allocator for the
// CSR and COO direct-load kernels: 3 (85 registers a thread, 24 warps per
// SM) was measured fastest at the default tile of 512 on GB300 (R-MAT and
// Laplacian CSR 108 / 99 us, COO 120 / 114 us; 1 block cap: 121 / 122 and
// 125 / 134 us; 4: 112 / 95 and 127 / 121 us).
#ifndef MSREP_MINB
#define MSREP_MINB 3
#endif
constexpr int kWarps = 8;  // warps per block; each warp owns whole tiles
constexpr int kThreads = 32 * kWarps;

constexpr size_t a128(size_t v) { return (v + 127) & ~size_t(127); }

// shared-memory stage of one tile: up to TILE + 16 entries of each array
template <class V, int IPT, int NIDX>
struct StageGeom {
  static constexpr int CAP = 32 * IPT + 16;
  static constexpr size_t IDX = a128(4 * CAP);        // one int32 array
  static constexpr size_t VAL = a128(sizeof(V) * CAP);
  static constexpr size_t BYTES = NIDX * IDX + VAL;
  static constexpr int S = BYTES <= 3000 ? 4 : (BYTES <= 4700 ? 3 : 2);
  static constexpr size_t WARP = S * BYTES + 128;      // + mbarriers and tile records
  static constexpr size_t BLOCK = kWarps * WARP;
};

// loads the elements [e0, e1) of arr that the bulk copy could not cover
template <class T>
__device__ __forceinline__ void fill_tail(T *dst, const T *arr, const SegCopy &c, int64_t e0,
                                          int64_t e1) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = max(c.cend, e0) + lane; e < e1; e += 32) dst[e - c.base] = arr[e];
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads, MSREP_MINB) csr_direct(CsrArgs<Pol> a, const int32_t *n_tiles,
                                                       int64_t nnz) {
  grid_dependency_wait();
  __shared__ int32_t s_rp[kWarps][32 * IPT + 8];
  // per-row compensation flags of the low-precision form
  __shared__ uint8_t s_cf[Pol::kLow ? kWarps : 1][Pol::kLow ? 32 * IPT + 8 : 1];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileWalk tw = tile_walk(*n_tiles, kWarps, a.part_toff);
  const int T = tw.end, stride = tw.step;
  // The next tile's coordinates and its first 64 row pointers are loaded
  // while the current tile is processed, so a tile does not start with two
  // dependent global round trips (coordinates, then row pointers).
  int b = tw.first;
  int32_t r0 = 0, k0 = 0, r1 = 0, k1 = 0, p0 = 0, p1 = 0;
  auto fetch = [&](int t) {
    r0 = __ldg(a.tile_row + t);
    k0 = __ldg(a.tile_k + t);
    r1 = __ldg(a.tile_row + t + 1);
    k1 = __ldg(a.tile_k + t + 1);
    const int32_t rend = min(r1 + 2, a.m + 1);
    p0 = r0 + lane < rend ? __ldg(a.row_ptr + r0 + lane) : 0;
    p1 = r0 + 32 + lane < rend ? __ldg(a.row_ptr + r0 + 32 + lane) : 0;
  };
  if (b < T) fetch(b);
  auto walk = [&](auto copy) {
    for (; b < T; b += stride) {
      const int32_t cr0 = r0, ck0 = k0, cr1 = r1, ck1 = k1;
      const int32_t rend = min(cr1 + 2, a.m + 1);
      if (cr0 + lane < rend) s_rp[wid][lane] = p0;
      if (cr0 + 32 + lane < rend) s_rp[wid][32 + lane] = p1;
      for (int32_t r = cr0 + 64 + lane; r < rend; r += 32)
        s_rp[wid][r - cr0] = __ldg(a.row_ptr + r);
      __syncwarp();
      if (b + stride < T) fetch(b + stride);
      csr_tile_compute<Pol, GlobalSrc, decltype(copy)::value>(
          a, b, cr0, ck0, cr1, ck1, s_rp[wid], Seg<int32_t>{a.col_idx, 0},
          Seg<typename Pol::V>{a.val, 0}, nnz, GlobalSrc{}, Pol::kLow ? s_cf[wid] : nullptr);
      __syncwarp();
    }
  };
  // alpha = 1, beta = 0 (the usual call) finishes rows by a copy, decided
  // at compile time so that no other finishing mode is issued beside it
  if (a.finish == kFinishCopy)
    walk(std::true_type{});
  else
    walk(std::false_type{});
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads) csr_stream(CsrArgs<Pol> a, const int32_t *n_tiles,
                                                       int64_t nnz) {
  grid_dependency_wait();
  using V = typename Pol::V;
  using G = StageGeom<V, IPT, 2>;
  constexpr int S = G::S;
  extern __shared__ __align__(128) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem + wid * G::WARP;
  uint64_t *bar = reinterpret_cast<uint64_t *>(wb + S * G::BYTES);
  int4 *rec = reinterpret_cast<int4 *>(wb + S * G::BYTES + 64);
  auto rp_s = [&](int s) { return reinterpret_cast<int32_t *>(wb + s * G::BYTES); };
  auto col_s = [&](int s) { return reinterpret_cast<int32_t *>(wb + s * G::BYTES + G::IDX); };
  auto val_s = [&](int s) { return reinterpret_cast<V *>(wb + s * G::BYTES + 2 * G::IDX); };
  const int T = *n_tiles;
  const int first = blockIdx.x * kWarps + wid, W = gridDim.x * kWarps;
  const int64_t mp1 = int64_t(a.m) + 1;

  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(bar + s, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto plans = [&](int4 c, SegCopy &p, SegCopy &q, SegCopy &v) {
    p = seg_plan(c.x, min(int64_t(c.z) + 2, mp1), mp1, 4, 4);
    q = seg_plan(c.y, c.w, nnz, 4, 8);
    v = seg_plan(c.y, c.w, nnz, sizeof(V), 8);
  };
  auto coords = [&](int t) {
    return make_int4(__ldg(a.tile_row + t), __ldg(a.tile_k + t), __ldg(a.tile_row + t + 1),
                     __ldg(a.tile_k + t + 1));
  };
  // lane 0: stage s <- tile with coordinates c
  auto issue = [&](int s, int4 c) {
    SegCopy p, q, v;
    plans(c, p, q, v);
    rec[s] = c;
    mbar_arrive_expect_tx(bar + s, p.bytes + q.bytes + v.bytes);
    if (p.bytes) bulk_g2s(rp_s(s), a.row_ptr + p.base, p.bytes, bar + s);
    if (q.bytes) bulk_g2s(col_s(s), a.col_idx + q.base, q.bytes, bar + s);
    if (v.bytes) bulk_g2s(val_s(s), a.val + v.base, v.bytes, bar + s);
  };
  int4 pending = make_int4(0, 0, 0, 0);
  if (lane == 0) {
    for (int s = 0; s < S; ++s)
      if (first + s * W < T) issue(s, coords(first + s * W));
    if (first + S * W < T) pending = coords(first + S * W);
  }
  __syncwarp();
  int i = 0;
  bool ok = true;
  for (; first + i * W < T; ++i) {
    const int b = first + i * W, s = i % S;
    if (!mbar_wait(bar + s, (i / S) & 1, a.err)) {
      ok = false;
      break;
    }
    const int4 c = rec[s];
    SegCopy p, q, v;
    plans(c, p, q, v);
    fill_tail(rp_s(s), a.row_ptr, p, c.x, min(int64_t(c.z) + 2, mp1));
    const int64_t g_end = min((int64_t(c.w) + 7) & ~int64_t(7), nnz);
    fill_tail(col_s(s), a.col_idx, q, q.base, g_end);
    fill_tail(val_s(s), a.val, v, v.base, g_end);
    __syncwarp();
    csr_tile_compute<Pol>(a, b, c.x, c.y, c.z, c.w, rp_s(s) + (c.x - p.base),
                          Seg<int32_t>{col_s(s), q.base}, Seg<V>{val_s(s), v.base}, nnz,
                          SharedSrc{});
    __syncwarp();
    if (lane == 0 && b + S * W < T) {
      fence_proxy_async();
      issue(s, pending);
      if (b + (S + 1) * W < T) pending = coords(b + (S + 1) * W);
    }
    __syncwarp();
  }
  if (!ok) {
    // give the copies still in flight a bounded chance to land, then leave
    for (int j = i + 1; j < i + S && first + j * W < T; ++j) mbar_wait(bar + j % S, (j / S) & 1, a.err);
  }
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads, MSREP_MINB) coo_direct(CooArgs<Pol> a) {
  grid_dependency_wait();
  const int wid = threadIdx.x >> 5;
  int T = a.np * a.G, stride = gridDim.x * kWarps, b = blockIdx.x * kWarps + wid;
  if (a.per_part) {  // block i walks partition i's G tiles alone
    T = (blockIdx.x + 1) * a.G;
    stride = kWarps;
    b = blockIdx.x * a.G + wid;
  }
  // the next tile's range is loaded while the current one is processed
  int32_t k0 = 0, k1 = 0;
  if (b < T) coo_tile_range(a, b, k0, k1);
  auto walk = [&](auto copy) {
    for (; b < T; b += stride) {
      const int32_t ck0 = k0, ck1 = k1;
      if (b + stride < T) coo_tile_range(a, b + stride, k0, k1);
      coo_tile_compute<Pol, GlobalSrc, decltype(copy)::value>(
          a, b, ck0, ck1, Seg<int32_t>{a.row_idx, 0}, Seg<int32_t>{a.col_idx, 0},
          Seg<typename Pol::V>{a.val, 0}, GlobalSrc{});
      __syncwarp();
    }
  };
  // the common alpha = 1, beta = 0 specialised at compile time
  if (a.finish == kFinishCopy)
    walk(std::true_type{});
  else
    walk(std::false_type{});
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads) coo_stream(CooArgs<Pol> a) {
  grid_dependency_wait();
  using V = typename Pol::V;
  using G = StageGeom<V, IPT, 2>;
  constexpr int S = G::S;
  extern __shared__ __align__(128) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem + wid * G::WARP;
  uint64_t *bar = reinterpret_cast<uint64_t *>(wb + S * G::BYTES);
  int4 *rec = reinterpret_cast<int4 *>(wb + S * G::BYTES + 64);
  auto row_s = [&](int s) { return reinterpret_cast<int32_t *>(wb + s * G::BYTES); };
  auto col_s = [&](int s) { return reinterpret_cast<int32_t *>(wb + s * G::BYTES + G::IDX); };
  auto val_s = [&](int s) { return reinterpret_cast<V *>(wb + s * G::BYTES + 2 * G::IDX); };
  const int T = a.np * a.G;
  const int first = blockIdx.x * kWarps + wid, W = gridDim.x * kWarps;
  const int64_t nnz = a.nnz;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(bar + s, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto plans = [&](int4 c, SegCopy &r, SegCopy &q, SegCopy &v) {
    r = seg_plan(c.x, c.y, nnz, 4, 8);
    q = seg_plan(c.x, c.y, nnz, 4, 8);
    v = seg_plan(c.x, c.y, nnz, sizeof(V), 8);
  };
  auto coords = [&](int t) {
    int32_t k0, k1;
    coo_tile_range(a, t, k0, k1);
    return make_int4(k0, k1, 0, 0);
  };
  auto issue = [&](int s, int4 c) {
    SegCopy r, q, v;
    plans(c, r, q, v);
    rec[s] = c;
    mbar_arrive_expect_tx(bar + s, r.bytes + q.bytes + v.bytes);
    if (r.bytes) bulk_g2s(row_s(s), a.row_idx + r.base, r.bytes, bar + s);
    if (q.bytes) bulk_g2s(col_s(s), a.col_idx + q.base, q.bytes, bar + s);
    if (v.bytes) bulk_g2s(val_s(s), a.val + v.base, v.bytes, bar + s);
  };
  int4 pending = make_int4(0, 0, 0, 0);
  if (lane == 0) {
    for (int s = 0; s < S; ++s)
      if (first + s * W < T) issue(s, coords(first + s * W));
    if (first + S * W < T) pending = coords(first + S * W);
  }
  __syncwarp();
  int i = 0;
  bool ok = true;
  for (; first + i * W < T; ++i) {
    const int b = first + i * W, s = i % S;
    if (!mbar_wait(bar + s, (i / S) & 1, a.err)) {
      ok = false;
      break;
    }
    const int4 c = rec[s];
    SegCopy r, q, v;
    plans(c, r, q, v);
    const int64_t g_end = min((int64_t(c.y) + 7) & ~int64_t(7), nnz);
    fill_tail(row_s(s), a.row_idx, r, r.base, g_end);
    fill_tail(col_s(s), a.col_idx, q, q.base, g_end);
    fill_tail(val_s(s), a.val, v, v.base, g_end);
    __syncwarp();
    coo_tile_compute<Pol>(a, b, c.x, c.y, Seg<int32_t>{row_s(s), r.base},
                          Seg<int32_t>{col_s(s), q.base}, Seg<V>{val_s(s), v.base}, SharedSrc{});
    __syncwarp();
    if (lane == 0 && b + S * W < T) {
      fence_proxy_async();
      issue(s, pending);
      if (b + (S + 1) * W < T) pending = coords(b + (S + 1) * W);
    }
    __syncwarp();
  }
  if (!ok)
    for (int j = i + 1; j < i + S && first + j * W < T; ++j) mbar_wait(bar + j % S, (j / S) & 1, a.err);
}

// Longest column for which a CSC tile takes the interleaved walk
// (csc_tile_interleaved, whose column table is filled one lane per
// column); tiles with longer columns split their nonzeros evenly over the
// lanes (csc_tile_compute).  On the R-MAT workload at tile 256 the limit
// 128 gave 105 us, 32 gave 115 us and 256 gave 142 us.
constexpr int kColumnWalkMax = 128;

// Dynamic shared memory of csc_direct: per warp the tile's column pointers
// (int32) and the column of each of its nonzeros (int16, for the
// interleaved walk), then the frequent-row table of matrices with hub rows.
template <int IPT>
struct CscSmem {
  static constexpr int CAP = 32 * IPT + 8;
  static constexpr size_t CP = size_t(kWarps) * CAP * sizeof(int32_t);
  static constexpr size_t COL = size_t(kWarps) * CAP * sizeof(int16_t);
  static constexpr size_t WARM = size_t(kWarm) * (sizeof(int32_t) + sizeof(double));
  static constexpr size_t BYTES = CP + COL + WARM;
};

template <class Pol, int IPT>
// Four resident blocks (64 registers a thread); the column-pointer stages,
// the column tables and the frequent-row table fit four blocks' shared
// memory.
__global__ void __launch_bounds__(kThreads, 4) csc_direct(CscArgs<Pol> a, const int32_t *n_tiles,
                                                       int64_t nnz) {
  using SM = CscSmem<IPT>;
  grid_dependency_wait();
  extern __shared__ __align__(16) unsigned char dsm[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileWalk tw = tile_walk(*n_tiles, kWarps, a.part_toff);
  const int T = tw.end, stride = tw.step, first = tw.first;
  int32_t *s_cp = reinterpret_cast<int32_t *>(dsm) + wid * SM::CAP;
  int16_t *s_col = reinterpret_cast<int16_t *>(dsm + SM::CP) + wid * SM::CAP;
  int32_t *s_wtag = reinterpret_cast<int32_t *>(dsm + SM::CP + SM::COL);
  double *s_wacc = reinterpret_cast<double *>(dsm + SM::CP + SM::COL + sizeof(int32_t) * kWarm);
  const bool skew = csc_skewed(a.hot, a.yperm);
  // The next tile's coordinates and first 64 column pointers are loaded
  // while the current tile is processed (as in csr_direct).
  int32_t n0 = 0, nk0 = 0, n1 = 0, nk1 = 0, p0 = 0, p1 = 0;
  auto fetch = [&](int t) {
    n0 = __ldg(a.tile_row + t);
    nk0 = __ldg(a.tile_k + t);
    n1 = __ldg(a.tile_row + t + 1);
    nk1 = __ldg(a.tile_k + t + 1);
    const int32_t cend = min(n1 + 1, a.n + 1);
    p0 = n0 + lane < cend ? __ldg(a.col_ptr + n0 + lane) : 0;
    p1 = n0 + 32 + lane < cend ? __ldg(a.col_ptr + n0 + 32 + lane) : 0;
  };
  // one tile (its coordinates fetched): stage its column pointers, fetch
  // the next tile's, then scatter its products to sink
  auto tile = [&](int b, const auto &sink) {
    const int32_t c0 = n0, k0 = nk0, c1 = n1, k1 = nk1;
    const int32_t cend = min(c1 + 1, a.n + 1);
    if (c0 + lane < cend) s_cp[lane] = p0;
    if (c0 + 32 + lane < cend) s_cp[32 + lane] = p1;
    for (int32_t c = c0 + 64 + lane; c < cend; c += 32) s_cp[c - c0] = __ldg(a.col_ptr + c);
    __syncwarp();
    if (b + stride < T) fetch(b + stride);
    // scale * x of tile column c, read when a lane reaches the column
    const auto xat = [&a, c0](int c) {
      const int32_t g = c0 + c;
      if (g >= a.n) return 0.0;
      const double xv = double(load_x(a.x, g));
      return a.scaled ? __dmul_rn(xv, a.scale) : xv;
    };
    if (csc_tile_max_col(c0, k0, c1, k1, a.n, s_cp) <= kColumnWalkMax) {
      // FP64 with alpha = 1: the walk without its scaling multiply
      if (Pol::kLow || a.scaled)
        csc_tile_interleaved<Pol>(a, c0, k0, c1, k1, s_cp, sink, s_col);
      else
        csc_tile_interleaved<Pol, std::decay_t<decltype(sink)>, !Pol::kLow>(
            a, c0, k0, c1, k1, s_cp, sink, s_col);
    } else
      csc_tile_compute<Pol>(a, c0, k0, c1, k1, s_cp, xat, Seg<int32_t>{a.row_idx, 0},
                            Seg<typename Pol::V>{a.val, 0}, nnz, GlobalSrc{}, sink);
    __syncwarp();
  };
  if (skew) {
    // power-law rows: the frequent-row sums and the permuted accumulator
    WarmRows warm;
    warm.load(a.warm, s_wtag, s_wacc);
    const SkewSink<WarmRows> sink{&warm, a.yperm, a.pmask};
    if (first < T) fetch(first);
    for (int b = first; b < T; b += stride) tile(b, sink);
    warm.flush(a.yperm, a.pmask);
  } else {
    const DirectSink sink{a.yacc};
    if (first < T) fetch(first);
    for (int b = first; b < T; b += stride) tile(b, sink);
  }
}

template <class Pol, int IPT>
__global__ void __launch_bounds__(kThreads) csc_stream(CscArgs<Pol> a, const int32_t *n_tiles,
                                                       int64_t nnz) {
  grid_dependency_wait();
  using V = typename Pol::V;
  using G = StageGeom<V, IPT, 2>;
  constexpr int S = G::S;
  extern __shared__ __align__(128) unsigned char smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *xs = reinterpret_cast<double *>(smem + kWarps * G::WARP) + wid * (32 * IPT + 8);
  unsigned char *wb = smem + wid * G::WARP;
  uint64_t *bar = reinterpret_cast<uint64_t *>(wb + S * G::BYTES);
  int4 *rec = reinterpret_cast<int4 *>(wb + S * G::BYTES + 64);
  auto cp_s = [&](int s) { return reinterpret_cast<int32_t *>(wb + s * G::BYTES); };
  auto row_s = [&](int s) { return reinterpret_cast<int32_t *>(wb + s * G::BYTES + G::IDX); };
  auto val_s = [&](int s) { return reinterpret_cast<V *>(wb + s * G::BYTES + 2 * G::IDX); };
  const int T = *n_tiles;
  const int first = blockIdx.x * kWarps + wid, W = gridDim.x * kWarps;
  const int64_t np1 = int64_t(a.n) + 1;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(bar + s, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto plans = [&](int4 c, SegCopy &p, SegCopy &r, SegCopy &v) {
    p = seg_plan(c.x, min(int64_t(c.z) + 1, np1), np1, 4, 4);
    r = seg_plan(c.y, c.w, nnz, 4, 8);
    v = seg_plan(c.y, c.w, nnz, sizeof(V), 8);
  };
  auto coords = [&](int t) {
    return make_int4(__ldg(a.tile_row + t), __ldg(a.tile_k + t), __ldg(a.tile_row + t + 1),
                     __ldg(a.tile_k + t + 1));
  };
  auto issue = [&](int s, int4 c) {
    SegCopy p, r, v;
    plans(c, p, r, v);
    rec[s] = c;
    mbar_arrive_expect_tx(bar + s, p.bytes + r.bytes + v.bytes);
    if (p.bytes) bulk_g2s(cp_s(s), a.col_ptr + p.base, p.bytes, bar + s);
    if (r.bytes) bulk_g2s(row_s(s), a.row_idx + r.base, r.bytes, bar + s);
    if (v.bytes) bulk_g2s(val_s(s), a.val + v.base, v.bytes, bar + s);
  };
  __shared__ double s_hot[kWarps][kMaxHot];
  HotRows hot;
  hot.load(a.hot, s_hot);
  const bool skew = csc_skewed(a.hot, a.yperm);
  int4 pending = make_int4(0, 0, 0, 0);
  if (lane == 0) {
    for (int s = 0; s < S; ++s)
      if (first + s * W < T) issue(s, coords(first + s * W));
    if (first + S * W < T) pending = coords(first + S * W);
  }
  __syncwarp();
  int i = 0;
  bool ok = true;
  for (; first + i * W < T; ++i) {
    const int b = first + i * W, s = i % S;
    if (!mbar_wait(bar + s, (i / S) & 1, a.err)) {
      ok = false;
      break;
    }
    const int4 c = rec[s];
    SegCopy p, r, v;
    plans(c, p, r, v);
    fill_tail(cp_s(s), a.col_ptr, p, c.x, min(int64_t(c.z) + 1, np1));
    const int64_t g_end = min((int64_t(c.w) + 7) & ~int64_t(7), nnz);
    fill_tail(row_s(s), a.row_idx, r, r.base, g_end);
    fill_tail(val_s(s), a.val, v, v.base, g_end);
    csc_stage_x(a, c.x, c.z, xs);
    __syncwarp();
    const auto xat = [xs](int j) { return xs[j]; };
    if (skew)
      csc_tile_compute<Pol>(a, c.x, c.y, c.z, c.w, cp_s(s) + (c.x - p.base), xat,
                            Seg<int32_t>{row_s(s), r.base}, Seg<V>{val_s(s), v.base}, nnz,
                            SharedSrc{}, SkewSink<HotRows>{&hot, a.yperm, a.pmask});
    else
      csc_tile_compute<Pol>(a, c.x, c.y, c.z, c.w, cp_s(s) + (c.x - p.base), xat,
                            Seg<int32_t>{row_s(s), r.base}, Seg<V>{val_s(s), v.base}, nnz,
                            SharedSrc{}, DirectSink{a.yacc});
    __syncwarp();
    if (lane == 0 && b + S * W < T) {
      fence_proxy_async();
      issue(s, pending);
      if (b + (S + 1) * W < T) pending = coords(b + (S + 1) * W);
    }
    __syncwarp();
  }
  if (!ok)
    for (int j = i + 1; j < i + S && first + j * W < T; ++j) mbar_wait(bar + j % S, (j / S) & 1, a.err);
  if (skew) hot.flush(a.yperm, a.pmask, s_hot);
}

// ---------------------------------------------------------------------------
// COO sorted by column or in no order (Sec. 3.2.3): a scatter, like CSC
// ---------------------------------------------------------------------------

// Every partition of such a matrix may add to any row, so its partial
// vector spans all of y (the full partial vectors Sec. 3.2.3 anticipates)
// and the merge is their sum.  Here each product is one FP64 atomic add into
// the row's entry of y (or of the accumulator): the atomic adds form the sum
// of the partials in place, so the result does not depend on the partition
// boundaries, and the nonzeros are spread over the warps of the grid in
// runs of consecutive nonzeros (coo_scatter).  Hub and frequent rows (from the plan) are summed per block in
// shared memory and the other rows go to the permuted accumulator, as for
// CSC.
template <class Pol>
struct ScatterArgs {
  const int32_t *row_idx;
  const int32_t *col_idx;
  const typename Pol::V *val;
  const typename Pol::X *x;
  double *yacc;   // scatter target by row: y (FP64) or the FP64 accumulator
  double *yperm;  // permuted accumulator (pmask + 1 entries), or null
  uint32_t pmask;
  double scale;   // alpha on the FP64 path, 1 when a finishing pass follows
  bool scaled;
  const int32_t *hot;   // hub rows, or null
  const unsigned long long *warm;  // frequent-row table (kWarm entries)
  int64_t nnz;
};

// Lane-interleaved, as CSC's interleaved walk: each warp takes runs of
// 32 * B consecutive nonzeros, step u of a run the 32 nonzeros
// base + 32 u + lane, so every load reads 32 consecutive elements and, in
// column order, the x gathers of a step touch a few columns and its atomic
// adds (for a banded matrix) a few short runs of rows.  B steps are loaded
// ahead.
template <class Pol>
__global__ void __launch_bounds__(kThreads, 4) coo_scatter(ScatterArgs<Pol> a) {
  grid_dependency_wait();
  using LV = typename LoadT<typename Pol::V>::type;
  constexpr int B = 7;
  __shared__ int32_t s_wtag[kWarm];
  __shared__ double s_wacc[kWarm];
  const bool skew = a.hot != nullptr && csc_skewed(a.hot, a.yperm);
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  auto run = [&](const auto &sink) {
    for (int64_t base = warp * 32 * B; base < a.nnz; base += nwarps * 32 * B) {
      int32_t r[B];
      LV v[B];
      if constexpr (Pol::kLow &&
                    std::is_same<std::decay_t<decltype(sink)>, DirectSink>::value) {
        // loads first; values and x are widened to FP64 (integer
        // operations, widen) after all of them are issued (direct scatter
        // only, as in the CSC walk)
        typename Pol::X xr[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int64_t k = base + 32 * u + lane;
          const bool in = k < a.nnz;
          r[u] = in ? ld_stream(a.row_idx + k) : 0;
          v[u] = in ? LV(ld_stream(a.val + k)) : LV(0);
          xr[u] = in ? load_x(a.x, ld_stream(a.col_idx + k)) : typename Pol::X(0);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
          if (base + 32 * u >= a.nnz) break;  // warp-uniform
          // the low-precision form applies alpha in its finishing pass
          // (a.scaled is false), so no scaling multiply here
          const double prod = __dmul_rn(widen(v[u]), widen(xr[u]));
          if (base + 32 * u + lane < a.nnz) sink.add(r[u], prod);
        }
      } else {
        double xv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int64_t k = base + 32 * u + lane;
          const bool in = k < a.nnz;
          r[u] = in ? ld_stream(a.row_idx + k) : 0;
          v[u] = in ? LV(ld_stream(a.val + k)) : LV(0);
          xv[u] = in ? double(load_x(a.x, ld_stream(a.col_idx + k))) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
          if (base + 32 * u >= a.nnz) break;  // warp-uniform
          const double xs = a.scaled ? __dmul_rn(xv[u], a.scale) : xv[u];
          const double prod = __dmul_rn(double(v[u]), xs);
          if (base + 32 * u + lane < a.nnz) sink.add(r[u], prod);
        }
      }
    }
  };
  if (skew) {
    WarmRows hot;
    hot.load(a.warm, s_wtag, s_wacc);
    run(SkewSink<WarmRows>{&hot, a.yperm, a.pmask});
    hot.flush(a.yperm, a.pmask);
  } else {
    run(DirectSink{a.yacc});
  }
}

// ---------------------------------------------------------------------------
// fix-up: rows split between tiles, merged in tile (= partition) order
// ---------------------------------------------------------------------------

// One warp per 32 consecutive tiles (grid-stride over warps).
template <class X, class View>
__global__ void fixup_split_rows(View v, const double *head, const double *tail,
                                 X *y, double alpha, double beta) {
  grid_dependency_wait();
  const int T = v.count();
  const int64_t warp = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < T; base += nwarps * 32)
    fixup_warp(v, T, static_cast<int>(base), head, tail, y, alpha, beta);
}

// Before a CSC scatter: a skewed matrix zeroes the permuted accumulator
// (beta is applied when y is gathered back); otherwise the row-ordered
// target is prepared: y = beta * y on the FP64 path (nothing for beta = 1),
// the FP64 accumulator zeroed on the low-precision path.
__global__ void csc_prepare(const int32_t *hot, double *yperm, int64_t perm_n, double *yrow,
                            int64_t m, double beta, int row_is_y) {
  grid_dependency_wait();
  const int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t step = int64_t(gridDim.x) * blockDim.x;
  if (csc_skewed(hot, yperm)) {
    for (int64_t i = i0; i < perm_n; i += step) yperm[i] = 0.0;
  } else if (!row_is_y || beta != 1.0) {
    for (int64_t r = i0; r < m; r += step)
      yrow[r] = (!row_is_y || beta == 0.0) ? 0.0 : __dmul_rn(beta, yrow[r]);
  }
}

// FP64 CSC, skewed matrix: y[r] = acc[slot(r)] + beta * y[r].
__global__ void csc_unpermute(const int32_t *hot, const double *yperm, uint32_t pmask,
                              double *y, int64_t m, double beta) {
  grid_dependency_wait();
  if (!csc_skewed(hot, yperm)) return;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < m;
       r += int64_t(gridDim.x) * blockDim.x) {
    const double acc = yperm[perm_slot(static_cast<int32_t>(r), pmask)];
    y[r] = beta == 0.0 ? acc : __dadd_rn(acc, __dmul_rn(beta, y[r]));
  }
}

// Low-precision CSC: y = alpha * acc + beta * y in FP64, rounded to FP32
// once; acc is read through the permutation for a skewed matrix.
__global__ void finish_csc_f32(const int32_t *hot, const double *yperm, uint32_t pmask,
                               const double *yacc, float *y, int64_t m, double alpha,
                               double beta) {
  grid_dependency_wait();
  const bool skew = csc_skewed(hot, yperm);
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < m;
       r += int64_t(gridDim.x) * blockDim.x) {
    const double acc = skew ? yperm[perm_slot(static_cast<int32_t>(r), pmask)] : yacc[r];
    y[r] = float(finish_merged(acc, alpha, beta, beta == 0.0 ? 0.0 : double(y[r])));
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
  double *head, *tail, *yacc;  // yacc: the CSC accumulator (see csc_acc_len)
  bool perm;                   // yacc is the permuted accumulator (CSC)
};

// Entries of the CSC accumulator in the workspace: the permuted accumulator
// (perm_extent(m) entries, also used in row order by the low-precision
// path) when perm_ok, else the low-precision path's row-ordered FP64 sums.
static int64_t csc_acc_len(const msrep_matrix *A, bool perm_ok) {
  if (A->fmt != MSREP_CSC && !coo_scatter_format(A->fmt)) return 0;
  if (perm_ok) return perm_extent(A->m);
  return A->val_dtype == MSREP_F64 ? 0 : A->m;
}

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
  if (coo_scatter_format(A->fmt)) return 0;
  if (A->fmt == MSREP_COO) return p->np * coo_tiles_per_part(A->nnz, p->np, tile);
  const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
  return plan_layout(n_major, A->nnz, p->np, tile).tmax;
}

}  // namespace msrep

msrep_status msrep::set_min_carveout(const void *kernel, size_t dyn_smem, int blocks) {
  int dev = 0;
  MSREP_CUDA_TRY(cudaGetDevice(&dev));
  cudaFuncAttributes fa;
  MSREP_CUDA_TRY(cudaFuncGetAttributes(&fa, kernel));
  int per_sm = 0, reserved = 0;
  MSREP_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  MSREP_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  const size_t per_block = fa.sharedSizeBytes + dyn_smem;
  if (per_block == 0 || per_sm <= 0 || blocks <= 0) return MSREP_OK;
  const size_t need = size_t(blocks) * (per_block + size_t(reserved));
  const int pct = static_cast<int>(std::min<size_t>(100, (100 * need + per_sm - 1) / per_sm));
  MSREP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
  return MSREP_OK;
}

namespace msrep {

// Resident blocks per SM of a kernel on the current device, after the
// dynamic shared-memory opt-in it needs.  With want_blocks > 0 the kernel's
// shared-memory carveout is set to the smallest that holds that many blocks
// (set_min_carveout).
template <class K>
static msrep_status kernel_occupancy(K kernel, size_t smem, int want_blocks, int *nb) {
  static std::mutex mu;
  // keyed by (device, kernel): function attributes are set per device
  static std::map<std::pair<int, const void *>, int> cache;
  int dev = 0;
  MSREP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, reinterpret_cast<const void *>(kernel));
  auto it = cache.find(key);
  if (it != cache.end()) {
    *nb = it->second;
    return MSREP_OK;
  }
  if (smem > 0)
    MSREP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(smem)));
  if (want_blocks > 0)
    MSREP_TRY(set_min_carveout(reinterpret_cast<const void *>(kernel), smem, want_blocks));
  *nb = resident_blocks(kernel, smem);
  cache[key] = *nb;
  return MSREP_OK;
}

// Launches the streaming kernel (dynamic shared-memory stages) unless the
// caller asked for direct loads.  Grid: resident blocks x SMs, capped by the
// number of tiles.
// With per_part > 0 the grid is one block per partition (per_part blocks).
template <class KS, class KD, class... Args>
static msrep_status launch_tiles(KS kstream, KD kdirect, size_t stream_smem, size_t direct_smem,
                                 int direct_blocks, bool direct, int64_t tiles, int per_part,
                                 cudaStream_t st, Args... args) {
  int nb = 1;
  if (direct)
    MSREP_TRY(kernel_occupancy(kdirect, direct_smem, direct_blocks, &nb));
  else
    MSREP_TRY(kernel_occupancy(kstream, stream_smem, 0, &nb));
  int64_t grid = std::min<int64_t>(ceil_div(tiles, kWarps), int64_t(nb) * sm_count());
  if (per_part > 0) grid = per_part;
  if (grid < 1) grid = 1;
  prof_begin(st);
  if (direct)
    MSREP_TRY(launch_dependent(kdirect, grid, kThreads, st, direct_smem, args...));
  else
    MSREP_TRY(launch_dependent(kstream, grid, kThreads, st, stream_smem, args...));
  prof_end(st);
  return MSREP_OK;
}

template <class Pol, int IPT>
static msrep_status run_csr(const msrep_matrix *A, const msrep_partition *p,
                            double alpha, const void *x, double beta, void *y,
                            unsigned flags, const Workspace &w, cudaStream_t st) {
  const int32_t tile = effective_tile_fmt(p->tile, A->fmt);
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
  a.err = kernel_err_ptr();
  if (!a.err) return fail(MSREP_ERR_CUDA, "cannot resolve the device error word");
  const bool per_part = (flags & MSREP_SCHED_PER_PARTITION) != 0;
  a.part_toff = per_part ? reinterpret_cast<const int32_t *>(plan + L.off_toff) : nullptr;
  MSREP_TRY(launch_tiles(csr_stream<Pol, IPT>, csr_direct<Pol, IPT>,
                         StageGeom<typename Pol::V, IPT, 2>::BLOCK, 0, MSREP_MINB,
                         (flags & MSREP_STREAM_TMA) == 0, L.tmax, per_part ? p->np : 0, st, a,
                         n_tiles, A->nnz));
  CsrTileView v{a.tile_row, a.tile_k, A->ptr, n_tiles};
  int64_t fg = std::min<int64_t>(ceil_div(L.tmax, 256), 4 * sm_count());
  MSREP_TRY(launch_dependent(fixup_split_rows<typename Pol::X, CsrTileView>, fg, 256, st, 0, v,
                             w.head, w.tail, a.y, alpha, beta));
  return MSREP_OK;
}

template <class Pol, int IPT>
static msrep_status run_coo(const msrep_matrix *A, const msrep_partition *p,
                            double alpha, const void *x, double beta, void *y,
                            unsigned flags, const Workspace &w, cudaStream_t st) {
  const int32_t tile = effective_tile_fmt(p->tile, A->fmt);
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
  a.err = kernel_err_ptr();
  if (!a.err) return fail(MSREP_ERR_CUDA, "cannot resolve the device error word");
  const int64_t T = int64_t(a.np) * a.G;
  a.per_part = (flags & MSREP_SCHED_PER_PARTITION) != 0;
  MSREP_TRY(launch_tiles(coo_stream<Pol, IPT>, coo_direct<Pol, IPT>,
                         StageGeom<typename Pol::V, IPT, 2>::BLOCK, 0, MSREP_MINB,
                         (flags & MSREP_STREAM_TMA) == 0, T, a.per_part ? p->np : 0, st, a));
  CooTileView v{A->idx2, p->start_idx, p->end_idx, A->nnz, a.G, a.np, A->m};
  int64_t fg = std::min<int64_t>(ceil_div(T, 256), 4 * sm_count());
  MSREP_TRY(launch_dependent(fixup_split_rows<typename Pol::X, CooTileView>, fg, 256, st, 0, v,
                             w.head, w.tail, a.y, alpha, beta));
  return MSREP_OK;
}

template <class Pol, int IPT>
static msrep_status run_csc(const msrep_matrix *A, const msrep_partition *p,
                            double alpha, const void *x, double beta, void *y,
                            unsigned flags, const Workspace &w, cudaStream_t st) {
  const int32_t tile = effective_tile_fmt(p->tile, A->fmt);
  PlanLayout L = plan_layout(A->n, A->nnz, p->np, tile, true);
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
  const bool per_part = (flags & MSREP_SCHED_PER_PARTITION) != 0;
  a.part_toff = per_part ? reinterpret_cast<const int32_t *>(plan + L.off_toff) : nullptr;
  a.n = A->n;
  a.err = kernel_err_ptr();
  if (!a.err) return fail(MSREP_ERR_CUDA, "cannot resolve the device error word");
  a.hot = reinterpret_cast<const int32_t *>(plan + L.off_hot);
  a.warm = reinterpret_cast<const unsigned long long *>(plan + L.off_warm);
  const int64_t m = A->m;
  const int sg = 4 * sm_count();
  const int64_t pn = w.perm ? perm_extent(m) : 0;
  a.yperm = w.perm ? w.yacc : nullptr;
  a.pmask = w.perm ? static_cast<uint32_t>(pn - 1) : 0u;
  // y (or the accumulator) is prepared on the device, which alone knows
  // whether the plan found hub rows
  if (kF64) {
    a.yacc = static_cast<double *>(y);
    a.scale = alpha;
    a.scaled = alpha != 1.0;
    if (w.perm || beta != 1.0)
      MSREP_TRY(launch_dependent(csc_prepare, sg, 256, st, 0, a.hot, a.yperm, pn, a.yacc, m, beta,
                                 1));
  } else {
    a.yacc = w.yacc;
    a.scale = 1.0;
    a.scaled = false;
    MSREP_TRY(launch_dependent(csc_prepare, sg, 256, st, 0, a.hot, a.yperm, pn, w.yacc, m, 0.0, 0));
  }
  MSREP_CUDA_TRY(cudaGetLastError());
  MSREP_TRY(launch_tiles(csc_stream<Pol, IPT>, csc_direct<Pol, IPT>,
                         StageGeom<typename Pol::V, IPT, 2>::BLOCK +
                             sizeof(double) * kWarps * (32 * IPT + 8),
                         CscSmem<IPT>::BYTES, 0, (flags & MSREP_STREAM_TMA) == 0, L.tmax,
                         per_part ? p->np : 0, st, a, n_tiles, A->nnz));
  if (kF64) {
    if (w.perm)
      MSREP_TRY(launch_dependent(csc_unpermute, sg, 256, st, 0, a.hot,
                                 static_cast<const double *>(a.yperm), a.pmask,
                                 static_cast<double *>(y), m, beta));
  } else {
    MSREP_TRY(launch_dependent(finish_csc_f32, sg, 256, st, 0, a.hot,
                               static_cast<const double *>(a.yperm), a.pmask,
                               static_cast<const double *>(w.yacc), static_cast<float *>(y), m,
                               alpha, beta));
  }
  return MSREP_OK;
}

// COO sorted by column or in no order: prepare the target as for CSC, one
// scatter over all nonzeros, then the gather of y from the permuted
// accumulator (FP64) or the finishing pass (low precision).
template <class Pol>
static msrep_status run_coo_scatter(const msrep_matrix *A, const msrep_partition *p,
                                    double alpha, const void *x, double beta, void *y,
                                    const Workspace &w, cudaStream_t st) {
  constexpr bool kF64 = sizeof(typename Pol::X) == 8;
  ScatterArgs<Pol> a;
  a.row_idx = A->idx2;
  a.col_idx = A->idx;
  a.val = static_cast<const typename Pol::V *>(A->val);
  a.x = static_cast<const typename Pol::X *>(x);
  a.hot = static_cast<const int32_t *>(p->plan);
  a.warm = reinterpret_cast<const unsigned long long *>(static_cast<const char *>(p->plan) +
                                                        kScatterWarmOff);
  a.nnz = A->nnz;
  const int64_t m = A->m;
  const int sg = 4 * sm_count();
  const int64_t pn = w.perm ? perm_extent(m) : 0;
  a.yperm = w.perm ? w.yacc : nullptr;
  a.pmask = w.perm ? static_cast<uint32_t>(pn - 1) : 0u;
  if (kF64) {
    a.yacc = static_cast<double *>(y);
    a.scale = alpha;
    a.scaled = alpha != 1.0;
    if (w.perm || beta != 1.0)
      MSREP_TRY(launch_dependent(csc_prepare, sg, 256, st, 0, a.hot, a.yperm, pn, a.yacc, m, beta,
                                 1));
  } else {
    a.yacc = w.yacc;
    a.scale = 1.0;
    a.scaled = false;
    MSREP_TRY(launch_dependent(csc_prepare, sg, 256, st, 0, a.hot, a.yperm, pn, w.yacc, m, 0.0, 0));
  }
  int nb = 1;
  MSREP_TRY(kernel_occupancy(coo_scatter<Pol>, 0, 0, &nb));
  const int64_t grid = std::max<int64_t>(
      1, std::min<int64_t>(ceil_div(A->nnz, 7 * kThreads), int64_t(nb) * sm_count()));
  prof_begin(st);
  MSREP_TRY(launch_dependent(coo_scatter<Pol>, grid, kThreads, st, 0, a));
  prof_end(st);
  if (kF64) {
    if (w.perm)
      MSREP_TRY(launch_dependent(csc_unpermute, sg, 256, st, 0, a.hot,
                                 static_cast<const double *>(a.yperm), a.pmask,
                                 static_cast<double *>(y), m, beta));
  } else {
    MSREP_TRY(launch_dependent(finish_csc_f32, sg, 256, st, 0, a.hot,
                               static_cast<const double *>(a.yperm), a.pmask,
                               static_cast<const double *>(w.yacc), static_cast<float *>(y), m,
                               alpha, beta));
  }
  return MSREP_OK;
}

template <class Pol>
static msrep_status dispatch_tile(const msrep_matrix *A, const msrep_partition *p,
                                  double alpha, const void *x, double beta,
                                  void *y, unsigned flags, const Workspace &w,
                                  cudaStream_t st) {
  if (coo_scatter_format(A->fmt)) return run_coo_scatter<Pol>(A, p, alpha, x, beta, y, w, st);
  const int32_t tile = effective_tile_fmt(p->tile, A->fmt);
#define MSREP_FMT_CASE(IPT)                                                   \
  switch (A->fmt) {                                                           \
    case MSREP_CSR: return run_csr<Pol, IPT>(A, p, alpha, x, beta, y, flags, w, st); \
    case MSREP_COO: return run_coo<Pol, IPT>(A, p, alpha, x, beta, y, flags, w, st); \
    default: return run_csc<Pol, IPT>(A, p, alpha, x, beta, y, flags, w, st); \
  }
  switch (tile) {
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

msrep_status msrep_device_status(void *stream, int *status) {
  if (!status) return fail(MSREP_ERR_INVALID_ARG, "status is NULL");
  cudaStream_t st = as_stream(stream);
  int zero = 0;
  MSREP_CUDA_TRY(cudaMemcpyFromSymbolAsync(status, g_kernel_err, sizeof(int), 0,
                                           cudaMemcpyDeviceToHost, st));
  MSREP_CUDA_TRY(cudaStreamSynchronize(st));
  MSREP_CUDA_TRY(cudaMemcpyToSymbolAsync(g_kernel_err, &zero, sizeof(int), 0,
                                         cudaMemcpyHostToDevice, st));
  MSREP_CUDA_TRY(cudaStreamSynchronize(st));
  if (*status) return fail(MSREP_ERR_TIMEOUT, "a kernel gave up on a bounded wait (code %d)", *status);
  return ok();
}

msrep_status msrep_profile_events(void *start, void *stop) {
  g_prof_start = reinterpret_cast<cudaEvent_t>(start);
  g_prof_stop = reinterpret_cast<cudaEvent_t>(stop);
  return ok();
}

msrep_status msrep_spmv_workspace_size(const msrep_matrix *A,
                                       const msrep_partition *part,
                                       size_t *bytes) {
  return spmv_workspace_bytes(A, part, true, bytes);
}

msrep_status msrep_spmv(const msrep_matrix *A, const msrep_partition *part,
                        double alpha, const void *x, double beta, void *y,
                        int32_t xy_dtype, unsigned flags, void *workspace,
                        void *stream) {
  return spmv_run(A, part, alpha, x, beta, y, xy_dtype, flags, workspace, stream, true);
}

}  // extern "C"

namespace msrep {

msrep_status spmv_workspace_bytes(const msrep_matrix *A, const msrep_partition *part,
                                  bool perm_ok, size_t *bytes) {
  MSREP_TRY(check_matrix(A));
  if (!part || part->np < 1 || !bytes)
    return fail(MSREP_ERR_INVALID_ARG, "bad partition or bytes pointer");
  const int32_t tile = effective_tile_fmt(part->tile, A->fmt);
  if (!tile_supported(tile)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", part->tile);
  const int64_t tiles = tiles_for(A, part, tile);
  *bytes = ws_layout(tiles, csc_acc_len(A, perm_ok), nullptr, nullptr);
  return ok();
}

msrep_status spmv_run(const msrep_matrix *A, const msrep_partition *part, double alpha,
                      const void *x, double beta, void *y, int32_t xy_dtype, unsigned flags,
                      void *workspace, void *stream, bool perm_ok) {
  MSREP_TRY(check_matrix(A));
  if (!part || part->np < 1 || !part->start_idx || !part->end_idx)
    return fail(MSREP_ERR_INVALID_ARG, "bad partition");
  const int32_t tile = effective_tile_fmt(part->tile, A->fmt);
  if (!tile_supported(tile)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", part->tile);
  if ((flags & MSREP_STREAM_TMA) && tile > 512)
    return fail(MSREP_ERR_INVALID_ARG, "MSREP_STREAM_TMA supports tiles up to 512");
  if ((flags & MSREP_SCHED_PER_PARTITION) &&
      ((flags & MSREP_STREAM_TMA) || coo_scatter_format(A->fmt)))
    return fail(MSREP_ERR_INVALID_ARG,
                "MSREP_SCHED_PER_PARTITION takes CSR, CSC or row-sorted COO, without "
                "MSREP_STREAM_TMA");
  if ((A->m > 0 && !y) || (A->n > 0 && !x && A->nnz > 0))
    return fail(MSREP_ERR_INVALID_ARG, "x or y is NULL");
  const bool f64 = A->val_dtype == MSREP_F64;
  if (f64 != (xy_dtype == MSREP_F64) || (xy_dtype != MSREP_F64 && xy_dtype != MSREP_F32))
    return fail(MSREP_ERR_INVALID_ARG,
                "unsupported types: val %d with x/y %d (F64/F64, F32/F32 or BF16/F32)",
                A->val_dtype, xy_dtype);
  cudaStream_t st = as_stream(stream);
  if (A->m == 0) return ok();
  if (coo_scatter_format(A->fmt)) {
    if (!part->plan || part->plan_bytes < static_cast<int64_t>(kScatterPlanBytes))
      return fail(MSREP_ERR_WORKSPACE,
                  "column-sorted or unsorted COO SpMV needs the partition's plan (%zu bytes)",
                  kScatterPlanBytes);
  } else if (A->fmt != MSREP_COO) {
    const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
    const int64_t need = static_cast<int64_t>(
        plan_layout(n_major, A->nnz, part->np, tile, A->fmt == MSREP_CSC).bytes);
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
    if ((mis & (A->val_dtype == MSREP_BF16 ? 15 : 31)) || (reinterpret_cast<uintptr_t>(A->ptr) & 15))
      return fail(MSREP_ERR_INVALID_ARG,
                  "idx, idx2 and val must be 32-byte aligned (16-byte for bf16 val), ptr 16-byte");
  }
  if (!workspace) return fail(MSREP_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) & 15)
    return fail(MSREP_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  const int64_t tiles = tiles_for(A, part, tile);
  Workspace w;
  ws_layout(tiles, csc_acc_len(A, perm_ok), &w, workspace);
  w.perm = perm_ok && (A->fmt == MSREP_CSC || coo_scatter_format(A->fmt));
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

}  // namespace msrep

