// Device partitioner: CSR -> pCSR (Alg. 2), CSC -> pCSC (Alg. 4),
// row-sorted COO -> pCOO (Alg. 6), the optional local pointers computed on
// the GPU (Sec. 4.1), and the merge-path tile plan that msrep_spmv runs on.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"

namespace msrep {

// ---------------------------------------------------------------------------
// status plumbing (declared in common.cuh)
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

msrep_status fail(msrep_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

msrep_status ok() {
  g_last_error.clear();
  return MSREP_OK;
}

int sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cached[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
    cached[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// ---------------------------------------------------------------------------
// searches over a compressed pointer array
// ---------------------------------------------------------------------------

// Largest r in [lo, hi] with ptr[r] <= k (the row owning nonzero k), found
// by a whole warp: each round the 32 lanes probe 32 evenly spaced points of
// [lo, hi] and the range shrinks about 33-fold (about five dependent loads
// for a million rows instead of twenty for a binary search).  Every lane
// returns the result.  Requires ptr[lo] <= k.
template <typename T>
__device__ __forceinline__ int32_t last_le_warp(const T *__restrict__ ptr, int32_t lo,
                                                int32_t hi, int64_t k) {
  const int lane = threadIdx.x & 31;
  while (hi - lo >= 32) {
    const int64_t span = int64_t(hi) - lo;
    const int32_t q = lo + static_cast<int32_t>((int64_t(lane) + 1) * span / 33);
    const bool le = static_cast<int64_t>(__ldg(ptr + q)) <= k;
    // ptr is non-decreasing and q increases with the lane: the lanes with
    // ptr[q] <= k form a prefix
    const int t = __popc(__ballot_sync(0xffffffffu, le));
    const int32_t qlo = __shfl_sync(0xffffffffu, q, t > 0 ? t - 1 : 0);
    const int32_t qhi = __shfl_sync(0xffffffffu, q, t < 32 ? t : 31);
    if (t > 0) lo = qlo;
    if (t < 32) hi = qhi - 1;
  }
  const bool le = lo + lane <= hi && static_cast<int64_t>(__ldg(ptr + lo + lane)) <= k;
  return lo + __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// last_le_warp on the merge path: largest r in [lo, hi] with
// ptr[r] + r <= d, the row coordinate of item d of the merged sequence of
// row ends and nonzeros.  ptr[r] + r is strictly increasing.  Requires
// ptr[lo] + lo <= d; every lane returns the result.
__device__ __forceinline__ int32_t path_row_warp(const int32_t *__restrict__ ptr, int32_t lo,
                                                 int32_t hi, int64_t d) {
  const int lane = threadIdx.x & 31;
  while (hi - lo >= 32) {
    const int64_t span = int64_t(hi) - lo;
    const int32_t q = lo + static_cast<int32_t>((int64_t(lane) + 1) * span / 33);
    const bool le = static_cast<int64_t>(__ldg(ptr + q)) + q <= d;
    const int t = __popc(__ballot_sync(0xffffffffu, le));
    const int32_t qlo = __shfl_sync(0xffffffffu, q, t > 0 ? t - 1 : 0);
    const int32_t qhi = __shfl_sync(0xffffffffu, q, t < 32 ? t : 31);
    if (t > 0) lo = qlo;
    if (t < 32) hi = qhi - 1;
  }
  const bool le =
      lo + lane <= hi && static_cast<int64_t>(__ldg(ptr + lo + lane)) + lo + lane <= d;
  return lo + __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// Merge-path coordinate of diagonal d: largest r in [lo, hi] with
// ptr[r] + r <= d (rows 0..r-1 have ended; ties consume the row end first).
__device__ __forceinline__ int32_t path_row(const int32_t *__restrict__ ptr,
                                            int32_t lo, int32_t hi, int64_t d) {
  while (lo < hi) {
    int32_t mid = lo + (hi - lo + 1) / 2;
    if (static_cast<int64_t>(__ldg(ptr + mid)) + mid <= d)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Alg. 2 / Alg. 4: metadata, one thread per partition
// ---------------------------------------------------------------------------

// Cut rules of part_meta_compressed.
enum : int { kCutNonzeros = 0, kCutMergePath = 1, kCutRowBlock = 2 };

// One warp per partition i (and one for the closing cut i = np).
// kCutNonzeros: Alg. 2's nonzero split, cut i at nonzero floor(i nnz/np).
// kCutMergePath: cut i at item floor(i (n_major + nnz) / np) of the merged
// sequence of row ends and nonzeros; partition i then holds the nonzeros
// between cuts i and i+1, with Alg. 2's metadata for that range.
// kCutRowBlock: the Baseline of Sec. 5.1, cut i at row floor(i n_major /
// np), so partition i holds rows [r_i, r_{i+1}) and all their nonzeros
// (ptr[r_i] .. ptr[r_{i+1}] - 1), with Alg. 2's metadata for that range;
// its tile-plan cut is the merge-path point (r_i, ptr[r_i]).
__global__ void part_meta_compressed(const int32_t *__restrict__ ptr,
                                     int32_t n_major, int64_t nnz, int32_t np,
                                     int32_t *start_idx, int32_t *end_idx,
                                     int32_t *start_major, int32_t *end_major,
                                     uint8_t *start_flag, int64_t *plan_D,
                                     int32_t *plan_R, int cut) {
  grid_dependency_wait();
  const int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const bool lead = (threadIdx.x & 31) == 0;
  if (i > np) return;  // warp-uniform
  int64_t s, e;
  if (cut == kCutRowBlock) {
    const int32_t r0 = static_cast<int32_t>((i * n_major) / np);
    s = __ldg(ptr + r0);
    if (plan_D && lead) {
      plan_R[i] = r0;
      plan_D[i] = s + r0;
    }
    if (i == np) return;
    const int32_t r1 = static_cast<int32_t>(((i + 1) * n_major) / np);
    e = int64_t(__ldg(ptr + r1)) - 1;
  } else if (cut == kCutMergePath) {
    const int64_t total = int64_t(n_major) + nnz;
    const int64_t d = (i * total) / np;
    const int32_t R = path_row_warp(ptr, static_cast<int32_t>(d > nnz ? d - nnz : 0),
                                    static_cast<int32_t>(d < n_major ? d : n_major), d);
    s = d - R;
    if (plan_D && lead) {
      plan_R[i] = R;
      plan_D[i] = d;
    }
    if (i == np) return;
    const int64_t d1 = ((i + 1) * total) / np;
    const int32_t R1 = path_row_warp(ptr, R, static_cast<int32_t>(d1 < n_major ? d1 : n_major), d1);
    e = d1 - R1 - 1;
  } else {
    s = (i * nnz) / np;
    if (plan_D) {
      // level-1 cut of the tile plan: (R(s_i), s_i) with R over [0, n_major]
      int32_t R;
      if (i == 0)
        R = 0;
      else if (i == np)
        R = n_major;
      else
        R = last_le_warp(ptr, 0, n_major, s);
      if (lead) {
        plan_R[i] = R;
        plan_D[i] = (i == 0) ? 0 : s + R;
      }
    }
    if (i == np) return;
    e = ((i + 1) * nnz) / np - 1;
  }
  if (e < s) {
    if (lead) {
      start_idx[i] = static_cast<int32_t>(s);
      end_idx[i] = static_cast<int32_t>(e);
      start_major[i] = 0;
      end_major[i] = -1;
      start_flag[i] = 0;
    }
    return;
  }
  const int32_t sr = last_le_warp(ptr, 0, n_major - 1, s);
  const int32_t er = last_le_warp(ptr, sr, n_major - 1, e);
  if (lead) {
    start_idx[i] = static_cast<int32_t>(s);
    end_idx[i] = static_cast<int32_t>(e);
    start_major[i] = sr;
    end_major[i] = er;
    start_flag[i] = (s > static_cast<int64_t>(__ldg(ptr + sr))) ? 1 : 0;
  }
}

// first k in [0, nnz) with idx[k] >= v (idx ascending), nnz if none
__device__ __forceinline__ int64_t lower_bound_idx(const int32_t *__restrict__ idx, int64_t nnz,
                                                   int32_t v) {
  int64_t lo = 0, hi = nnz;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(idx + mid) < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Alg. 6 (reading for sorted COO): metadata from row_idx directly.  With
// row_block (the Baseline of Sec. 5.1), partition i holds the rows
// [floor(i m / np), floor((i+1) m / np)) and the nonzero range is found by
// a binary search of row_idx for those rows (Sec. 5.3 searches for each row
// block's start and end).
__global__ void part_meta_coo(const int32_t *__restrict__ row_idx, int64_t nnz,
                              int32_t np, int32_t *start_idx, int32_t *end_idx,
                              int32_t *start_major, int32_t *end_major,
                              uint8_t *start_flag, int32_t m, int row_block) {
  grid_dependency_wait();
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= np) return;
  int64_t s, e;
  if (row_block) {
    s = lower_bound_idx(row_idx, nnz, static_cast<int32_t>((i * m) / np));
    e = lower_bound_idx(row_idx, nnz, static_cast<int32_t>(((i + 1) * m) / np)) - 1;
  } else {
    s = (i * nnz) / np;
    e = ((i + 1) * nnz) / np - 1;
  }
  start_idx[i] = static_cast<int32_t>(s);
  end_idx[i] = static_cast<int32_t>(e);
  if (e < s) {
    start_major[i] = 0;
    end_major[i] = -1;
    start_flag[i] = 0;
    return;
  }
  int32_t rs = __ldg(row_idx + s);
  start_major[i] = rs;
  end_major[i] = __ldg(row_idx + e);
  start_flag[i] = (s > 0 && __ldg(row_idx + s - 1) == rs) ? 1 : 0;
}

// pCOO of a COO matrix in no particular order: Alg. 6's nonzero ranges; a
// partition may reach any row (Sec. 3.2.3), so a non-empty one spans rows
// 0..m-1, and no first row is known to be split.
__global__ void part_meta_coo_unsorted(int64_t nnz, int32_t m, int32_t np, int32_t *start_idx,
                                       int32_t *end_idx, int32_t *start_major,
                                       int32_t *end_major, uint8_t *start_flag) {
  grid_dependency_wait();
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= np) return;
  const int64_t s = (i * nnz) / np;
  const int64_t e = ((i + 1) * nnz) / np - 1;
  start_idx[i] = static_cast<int32_t>(s);
  end_idx[i] = static_cast<int32_t>(e);
  start_major[i] = 0;
  end_major[i] = e < s ? -1 : m - 1;
  start_flag[i] = 0;
}

// ---------------------------------------------------------------------------
// single-block exclusive scan (np is at most a few hundred thousand)
// ---------------------------------------------------------------------------

template <typename T>
__device__ T block_exclusive_scan(T v, T &total) {
  __shared__ T warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    T w = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  T base = wid > 0 ? warp_sums[wid - 1] : T(0);
  total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + inc - v;
}

// local_off[i] = sum_{j<i} (end_major[j] - start_major[j] + 2) (CSR/CSC).
__global__ void __launch_bounds__(1024)
    local_off_scan(const int32_t *start_major, const int32_t *end_major,
                   int32_t np, int64_t *local_off) {
  grid_dependency_wait();
  int64_t carry = 0;
  for (int32_t base = 0; base < np; base += blockDim.x) {
    int32_t i = base + threadIdx.x;
    int64_t len = (i < np) ? int64_t(end_major[i]) - start_major[i] + 2 : 0;
    int64_t total;
    int64_t ex = block_exclusive_scan<int64_t>(len, total);
    if (i < np) local_off[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) local_off[np] = carry;
}

// Local row_ptr / col_ptr (Alg. 2/4 inner loop, computed on the GPU as in
// Sec. 4.1).  The outputs of all partitions form one array of local_off[np]
// entries.  Each warp writes 256 consecutive entries, 8 per lane: a warp-wide
// search over local_off brackets the partitions of the 256, a short binary
// search gives each lane the partition of its first entry, and the lane walks
// forward from there, so the work is spread evenly whatever P and the
// partitions' row spans are.  Entry j of partition i: 0 (j = 0),
// end - start + 1 (j = span + 1), else ptr[start_major + j] - start_idx.
template <bool kVec>
__global__ void __launch_bounds__(256)
    local_fill_compressed(const int32_t *__restrict__ ptr, const int32_t *start_idx,
                          const int32_t *end_idx, const int32_t *start_major,
                          const int32_t *end_major, const int64_t *local_off, int32_t np,
                          int32_t *local) {
  grid_dependency_wait();
  const int64_t total = local_off[np];
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t w0 = (blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5)) * 256;
       w0 < total; w0 += warps * 256) {
    // partitions of the warp's first and last entries (warp-uniform)
    const int32_t ia = last_le_warp(local_off, 0, np - 1, w0);
    const int32_t ib = last_le_warp(local_off, ia, np - 1, w0 + 255 < total ? w0 + 255 : total - 1);
    const int64_t t0 = w0 + 8 * lane;
    if (t0 >= total) continue;
    int32_t lo = ia, hi = ib;  // last i in [ia, ib] with local_off[i] <= t0
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (__ldg(local_off + mid) <= t0) lo = mid; else hi = mid - 1;
    }
    int32_t i = lo;
    int64_t base = __ldg(local_off + i), next = __ldg(local_off + i + 1);
    int32_t sm = __ldg(start_major + i), span = __ldg(end_major + i) - sm;
    int32_t s = __ldg(start_idx + i), e = __ldg(end_idx + i);
    int32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t t = t0 + u;
      while (t >= next && i + 1 < np) {
        ++i;
        base = next;
        next = __ldg(local_off + i + 1);
        sm = __ldg(start_major + i);
        span = __ldg(end_major + i) - sm;
        s = __ldg(start_idx + i);
        e = __ldg(end_idx + i);
      }
      const int32_t j = static_cast<int32_t>(t - base);
      v[u] = j == 0 ? 0 : (j == span + 1 ? e - s + 1 : __ldg(ptr + sm + j) - s);
    }
    if (kVec && t0 + 8 <= total) {
      reinterpret_cast<int4 *>(local + t0)[0] = make_int4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<int4 *>(local + t0)[1] = make_int4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t0 + u < total) local[t0 + u] = v[u];
    }
  }
}

// pCOO local row-index array: lrow[k] = row_idx[k] - start_row(partition of
// k).  Each thread converts 8 consecutive nonzeros.  Partition i starts at
// floor(i nnz / np) (Alg. 6), so the partition owning k is
// floor(((k + 1) np - 1) / nnz); the walk over start_idx confirms it and
// moves on at a partition boundary inside the 8.
template <bool kVec>
__global__ void __launch_bounds__(256)
    local_fill_coo(const int32_t *__restrict__ row_idx, int64_t nnz, int32_t np,
                   const int32_t *start_idx, const int32_t *start_major, int32_t *local) {
  grid_dependency_wait();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x * 8;
  for (int64_t k0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) * 8; k0 < nnz;
       k0 += stride) {
    // Alg. 2's split gives the owner directly; for other cuts (row blocks)
    // the last partition starting at or before k0 is searched for
    int32_t i = static_cast<int32_t>(((k0 + 1) * np - 1) / nnz);
    if (__ldg(start_idx + i) > k0 || (i + 1 < np && __ldg(start_idx + i + 1) <= k0)) {
      int32_t lo = 0, hi = np - 1;
      while (lo < hi) {
        const int32_t mid = lo + (hi - lo + 1) / 2;
        if (__ldg(start_idx + mid) <= k0)
          lo = mid;
        else
          hi = mid - 1;
      }
      i = lo;
    }
    int64_t next = i + 1 < np ? __ldg(start_idx + i + 1) : nnz;
    int32_t r0 = __ldg(start_major + i);
    int32_t r[8];
    const bool full = kVec && k0 + 8 <= nnz;
    if (full) {
      const int4 a = __ldcs(reinterpret_cast<const int4 *>(row_idx + k0));
      const int4 b = __ldcs(reinterpret_cast<const int4 *>(row_idx + k0) + 1);
      r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
      r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = k0 + u < nnz ? __ldcs(row_idx + k0 + u) : 0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      while (k0 + u >= next && i + 1 < np) {
        ++i;
        next = i + 1 < np ? __ldg(start_idx + i + 1) : nnz;
        r0 = __ldg(start_major + i);
      }
      r[u] -= r0;
    }
    if (full) {
      __stcs(reinterpret_cast<int4 *>(local + k0), make_int4(r[0], r[1], r[2], r[3]));
      __stcs(reinterpret_cast<int4 *>(local + k0) + 1, make_int4(r[4], r[5], r[6], r[7]));
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < nnz) local[k0 + u] = r[u];
    }
  }
}

// ---------------------------------------------------------------------------
// tile plan (CSR/CSC): each partition's stretch of the merge path
// [D_i, D_{i+1}) is split into ceil(len / tile) equal pieces
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024)
    plan_scan(const int64_t *D, int32_t np, int32_t tile, int32_t *tile_off) {
  grid_dependency_wait();
  int64_t carry = 0;
  for (int32_t base = 0; base < np; base += blockDim.x) {
    int32_t i = base + threadIdx.x;
    int64_t g = 0;
    if (i < np) g = (D[i + 1] - D[i] + tile - 1) / tile;
    int64_t total;
    int64_t ex = block_exclusive_scan<int64_t>(g, total);
    if (i < np) tile_off[i] = static_cast<int32_t>(carry + ex);
    carry += total;
  }
  if (threadIdx.x == 0) tile_off[np] = static_cast<int32_t>(carry);
}

__global__ void plan_tiles(const int32_t *__restrict__ ptr, int32_t n_major,
                           int64_t nnz, int32_t np, const int64_t *D,
                           const int32_t *R, const int32_t *tile_off,
                           int32_t *tile_row, int32_t *tile_k) {
  grid_dependency_wait();
  const int32_t i = blockIdx.x;
  const int32_t t0 = tile_off[i], G = tile_off[i + 1] - t0;
  const int64_t d0 = D[i], len = D[i + 1] - d0;
  const int32_t lo = R[i], hi = R[i + 1];
  for (int32_t g = threadIdx.x; g < G; g += blockDim.x) {
    int64_t d = d0 + (static_cast<int64_t>(g) * len) / G;
    int32_t r = path_row(ptr, lo, hi, d);
    tile_row[t0 + g] = r;
    tile_k[t0 + g] = static_cast<int32_t>(d - r);
  }
  if (i == np - 1 && threadIdx.x == 0) {
    const int32_t T = tile_off[np];
    tile_row[T] = n_major;
    tile_k[T] = static_cast<int32_t>(nnz);
  }
}

// ---------------------------------------------------------------------------
// structural validation (MSREP_VALIDATE)
// ---------------------------------------------------------------------------

__device__ unsigned int g_validate_err;

// Hub rows of a CSC matrix, or of a COO matrix sorted by column or in no
// order (at most kMaxHot): the row indices of
// kHotSample evenly spaced nonzeros are counted in an open-addressing table
// in shared memory (twice as many slots as samples, so probing ends), and
// the most frequent rows with at least kHotMin samples kept, most frequent
// first, ties to the smaller row.  Deterministic; one block.
constexpr int kHotSlotBits = 13;
constexpr int kHotSlots = 1 << kHotSlotBits;
static_assert(kHotSlots >= 2 * kHotSample, "hub-row table needs load <= 1/2");
constexpr size_t kHotSmem = 2 * sizeof(int32_t) * kHotSlots;

__global__ void __launch_bounds__(1024) hot_rows(const int32_t *__restrict__ row_idx,
                                                 int64_t nnz, int32_t *hot) {
  grid_dependency_wait();
  extern __shared__ int32_t hs[];
  int32_t *tkey = hs, *tcnt = hs + kHotSlots;
  __shared__ unsigned long long wbest[32];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < kHotSlots; i += nt) {
    tkey[i] = -1;
    tcnt[i] = 0;
  }
  __syncthreads();
  const int S = static_cast<int>(nnz < kHotSample ? nnz : kHotSample);
  for (int i = t; i < S; i += nt) {
    const int32_t r = __ldg(row_idx + (2 * int64_t(i) + 1) * nnz / (2 * int64_t(S)));
    uint32_t h = (static_cast<uint32_t>(r) * kPermMul) >> (32 - kHotSlotBits);
    for (int probe = 0; probe < kHotSlots; ++probe) {
      const int32_t old = atomicCAS(tkey + h, -1, r);
      if (old == -1 || old == r) {
        atomicAdd(tcnt + h, 1);
        break;
      }
      h = (h + 1) & (kHotSlots - 1);
    }
  }
  __syncthreads();
  int found = 0;
  for (int q = 0; q < kMaxHot; ++q) {
    // block-wide max of (count, smaller row first)
    unsigned long long best = 0;
    for (int i = t; i < kHotSlots; i += nt)
      if (tcnt[i] >= kHotMin) {
        const unsigned long long c = (static_cast<unsigned long long>(tcnt[i]) << 32) |
                                     (0xffffffffu - static_cast<uint32_t>(tkey[i]));
        best = c > best ? c : best;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, best, o);
      best = u > best ? u : best;
    }
    if ((t & 31) == 0) wbest[t >> 5] = best;
    __syncthreads();
    best = 0;
    for (int w = 0; w < (nt >> 5); ++w) best = wbest[w] > best ? wbest[w] : best;
    __syncthreads();
    if (best == 0) break;
    const int32_t r = static_cast<int32_t>(0xffffffffu - static_cast<uint32_t>(best & 0xffffffffu));
    if (t == 0) hot[1 + found] = r;
    ++found;
    for (int i = t; i < kHotSlots; i += nt)
      if (tkey[i] == r) tcnt[i] = 0;
    __syncthreads();
  }
  if (t == 0) {
    hot[0] = found;
    for (int q = found; q < kMaxHot; ++q) hot[1 + q] = -1;
  }
}

// hot_rows needs more than the default 48 KB of dynamic shared memory: opt
// in once per device.
static msrep_status hot_rows_smem_opt_in() {
  static std::mutex mu;
  static bool done[128] = {false};
  int dev = 0;
  MSREP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(MSREP_ERR_CUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    MSREP_CUDA_TRY(cudaFuncSetAttribute(hot_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(kHotSmem)));
    done[dev] = true;
  }
  return MSREP_OK;
}

// A frequent-row table slot during the search: (priority << 32) | ~row,
// 0 = empty.  atomicMax keeps the row of highest priority (sample count;
// hub rows highest), the smaller row on ties, whatever the order of the
// claims, so the table is the same on every run.
__device__ __forceinline__ unsigned long long warm_entry(uint32_t prio, int32_t row) {
  return (static_cast<unsigned long long>(prio) << 32) | ~static_cast<uint32_t>(row);
}

// Frequent-row search (only for a matrix with hub rows), step 1: the hub
// rows claim their slots of the frequent-row table at top priority; the
// rows of kWarmSample evenly spaced nonzeros are counted in an
// open-addressing table of kWarmTab slots (twice the samples, so probing
// ends), which holds row + 1 (0 = empty).  Everything starts all zero.
__global__ void warm_count(const int32_t *__restrict__ row_idx, int64_t nnz, const int32_t *hot,
                           unsigned long long *warm, int32_t *key, int32_t *cnt) {
  grid_dependency_wait();
  const int nh = hot[0];
  if (nh == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int q = 0; q < nh && q < kMaxHot; ++q) {
      const int32_t r = hot[1 + q];
      if (r >= 0) atomicMax(warm + warm_slot(r), warm_entry(0xffffffffu, r));
    }
  const int S = static_cast<int>(nnz < kWarmSample ? nnz : kWarmSample);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
    const int32_t r = __ldg(row_idx + (2 * int64_t(i) + 1) * nnz / (2 * int64_t(S)));
    uint32_t h = (static_cast<uint32_t>(r) * kPermMul) >> (32 - kWarmTabBits);
    for (int probe = 0; probe < kWarmTab; ++probe) {
      const int32_t old = atomicCAS(key + h, 0, r + 1);
      if (old == 0 || old == r + 1) {
        atomicAdd(cnt + h, 1);
        break;
      }
      h = (h + 1) & (kWarmTab - 1);
    }
  }
}

// Step 2: histogram of the sample counts >= kWarmMin (counts above 255 as
// 255) into hist[256].  Rows seen fewer times never qualify; they are most
// rows and would all land in one bin.
__global__ void warm_hist(const int32_t *hot, const int32_t *cnt, int32_t *hist) {
  grid_dependency_wait();
  __shared__ int h[256];
  if (hot[0] == 0) return;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kWarmTab; i += gridDim.x * blockDim.x) {
    const int c = cnt[i];
    if (c >= kWarmMin) atomicAdd(h + min(c, 255), 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, h[i]);
}

// Step 3: every counted row whose count reaches T claims its slot with its
// count as priority, T the smallest count >= kWarmMin that at most kWarm
// rows reach.
__global__ void warm_select(const int32_t *hot, const int32_t *key, const int32_t *cnt,
                            const int32_t *hist, unsigned long long *warm) {
  grid_dependency_wait();
  __shared__ int thresh;
  if (hot[0] == 0) return;
  if (threadIdx.x == 0) {
    int cum = 0, T = 256;
    for (int c = 255; c >= kWarmMin; --c) {
      if (cum + hist[c] > kWarm) break;
      cum += hist[c];
      T = c;
    }
    thresh = T;
  }
  __syncthreads();
  const int T = thresh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kWarmTab; i += gridDim.x * blockDim.x) {
    const int c = cnt[i];
    if (c < T) continue;
    const int32_t k = key[i];
    if (k > 0) atomicMax(warm + warm_slot(k - 1), warm_entry(static_cast<uint32_t>(c), k - 1));
  }
}

// Clears the frequent-row table and the scratch of its search (n words)
// when the matrix has hub rows; the others never read them.
__global__ void warm_clear(const int32_t *hot, uint32_t *p, int64_t n) {
  grid_dependency_wait();
  if (__ldg(hot) == 0) return;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    p[i] = 0u;
}

// A second stream of this host thread on the current device, with a fork
// and a join event: the frequent-row search depends on nothing else a
// partitioning call computes, so it runs beside the metadata and tile-plan
// chain.  The caller's stream still orders the whole call: the side stream
// waits for a fork event recorded on it and the caller's stream waits for
// the join event (a stream capture sees one fork and one join).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

static msrep_status side_stream(SideStream **out) {
  static thread_local std::map<int, SideStream> per_device;
  int dev = 0;
  MSREP_CUDA_TRY(cudaGetDevice(&dev));
  SideStream &ss = per_device[dev];
  if (!ss.s) {
    MSREP_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
    MSREP_CUDA_TRY(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
    MSREP_CUDA_TRY(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming));
  }
  *out = &ss;
  return MSREP_OK;
}

static msrep_status fork_side(cudaStream_t st, SideStream **ss) {
  MSREP_TRY(side_stream(ss));
  MSREP_CUDA_TRY(cudaEventRecord((*ss)->fork, st));
  MSREP_CUDA_TRY(cudaStreamWaitEvent((*ss)->s, (*ss)->fork, 0));
  return MSREP_OK;
}

static msrep_status join_side(cudaStream_t st, SideStream *ss) {
  MSREP_CUDA_TRY(cudaEventRecord(ss->join, ss->s));
  MSREP_CUDA_TRY(cudaStreamWaitEvent(st, ss->join, 0));
  return MSREP_OK;
}

// Hub rows, then the frequent-row table, of a scatter (CSC, or COO sorted by
// column or in no order): hot, warm and the search scratch (key, cnt) are
// in the plan.
static msrep_status find_frequent_rows(const int32_t *row_idx, int64_t nnz, int32_t *hot,
                                       unsigned long long *warm, int32_t *key, int32_t *cnt,
                                       cudaStream_t st) {
  MSREP_TRY(hot_rows_smem_opt_in());
  MSREP_TRY(launch_dependent(hot_rows, 1, 1024, st, kHotSmem, row_idx, nnz, hot));
  // table, scratch and histogram lie back to back, all starting at zero
  // (cleared only for a matrix with hub rows, which alone uses them)
  int32_t *hist = cnt + kWarmTab;
  const int64_t words = (reinterpret_cast<char *>(hist + 256) - reinterpret_cast<char *>(warm)) /
                        int64_t(sizeof(uint32_t));
  MSREP_TRY(launch_dependent(warm_clear, 2 * sm_count(), 256, st, 0, hot,
                             reinterpret_cast<uint32_t *>(warm), words));
  const int S = static_cast<int>(nnz < kWarmSample ? nnz : kWarmSample);
  MSREP_TRY(launch_dependent(warm_count,
                             std::max<int64_t>(1, std::min<int64_t>(ceil_div(S, 256),
                                                                    4 * sm_count())),
                             256, st, 0, row_idx, nnz, static_cast<const int32_t *>(hot), warm,
                             key, cnt));
  MSREP_TRY(launch_dependent(warm_hist, kWarmTab / 256, 256, st, 0,
                             static_cast<const int32_t *>(hot), static_cast<const int32_t *>(cnt),
                             hist));
  MSREP_TRY(launch_dependent(warm_select, kWarmTab / 256, 256, st, 0,
                             static_cast<const int32_t *>(hot), static_cast<const int32_t *>(key),
                             static_cast<const int32_t *>(cnt), static_cast<const int32_t *>(hist),
                             warm));
  return MSREP_OK;
}


__global__ void validate_compressed(const int32_t *__restrict__ ptr,
                                    int32_t n_major, int64_t nnz,
                                    const int32_t *__restrict__ idx,
                                    int32_t n_minor) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t stride = int64_t(gridDim.x) * blockDim.x;
  if (t == 0 && (ptr[0] != 0 || ptr[n_major] != nnz)) atomicOr(&g_validate_err, 1u);
  for (int64_t r = t; r < n_major; r += stride)
    if (ptr[r] > ptr[r + 1]) atomicOr(&g_validate_err, 2u);
  for (int64_t k = t; k < nnz; k += stride) {
    int32_t c = idx[k];
    if (c < 0 || c >= n_minor) atomicOr(&g_validate_err, 4u);
  }
}

// order: 0 = by (row, col), 1 = by (col, row), 2 = none
__global__ void validate_coo(const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                             int64_t nnz, int32_t m, int32_t n, int order) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t k = t; k < nnz; k += stride) {
    int32_t r = row[k], c = col[k];
    if (r < 0 || r >= m || c < 0 || c >= n) atomicOr(&g_validate_err, 4u);
    if (order < 2 && k + 1 < nnz) {
      const int32_t r2 = row[k + 1], c2 = col[k + 1];
      const int32_t a = order == 0 ? r : c, b = order == 0 ? c : r;
      const int32_t a2 = order == 0 ? r2 : c2, b2 = order == 0 ? c2 : r2;
      if (a2 < a || (a2 == a && b2 <= b)) atomicOr(&g_validate_err, 8u);
    }
  }
}

static std::mutex g_validate_mu;

static msrep_status run_validation(const msrep_matrix *A, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_validate_mu);
  unsigned int zero = 0, err = 0;
  MSREP_CUDA_TRY(cudaMemcpyToSymbolAsync(g_validate_err, &zero, sizeof zero, 0,
                                         cudaMemcpyHostToDevice, st));
  const int blocks = 4 * sm_count();
  if (coo_format(A->fmt)) {
    const int order = A->fmt == MSREP_COO ? 0 : A->fmt == MSREP_COO_BY_COL ? 1 : 2;
    validate_coo<<<blocks, 256, 0, st>>>(A->idx2, A->idx, A->nnz, A->m, A->n, order);
  } else {
    const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
    const int32_t n_minor = A->fmt == MSREP_CSR ? A->n : A->m;
    validate_compressed<<<blocks, 256, 0, st>>>(A->ptr, n_major, A->nnz, A->idx,
                                                n_minor);
  }
  MSREP_CUDA_TRY(cudaGetLastError());
  MSREP_CUDA_TRY(cudaMemcpyFromSymbolAsync(&err, g_validate_err, sizeof err, 0,
                                           cudaMemcpyDeviceToHost, st));
  MSREP_CUDA_TRY(cudaStreamSynchronize(st));
  if (err)
    return fail(MSREP_ERR_BAD_MATRIX,
                "matrix failed validation (code 0x%x: 1=ptr ends, 2=ptr not "
                "monotone, 4=index out of range, 8=COO not in its order)",
                err);
  return MSREP_OK;
}

// ---------------------------------------------------------------------------
// argument checks shared by the entry points
// ---------------------------------------------------------------------------

msrep_status check_matrix(const msrep_matrix *A) {
  if (!A) return fail(MSREP_ERR_INVALID_ARG, "matrix is NULL");
  if (A->m < 0 || A->n < 0 || A->nnz < 0 || A->nnz > INT32_MAX)
    return fail(MSREP_ERR_INVALID_ARG, "bad sizes m=%d n=%d nnz=%lld", A->m,
                A->n, (long long)A->nnz);
  if (A->val_dtype < MSREP_F64 || A->val_dtype > MSREP_BF16)
    return fail(MSREP_ERR_INVALID_ARG, "bad val_dtype %d", A->val_dtype);
  switch (A->fmt) {
    case MSREP_CSR:
    case MSREP_CSC:
      if (!A->ptr) return fail(MSREP_ERR_INVALID_ARG, "ptr is NULL");
      break;
    case MSREP_COO:
    case MSREP_COO_BY_COL:
    case MSREP_COO_UNSORTED:
      if (!A->idx2 && A->nnz > 0)
        return fail(MSREP_ERR_INVALID_ARG, "COO row_idx (idx2) is NULL");
      break;
    default:
      return fail(MSREP_ERR_INVALID_ARG, "bad format %d", A->fmt);
  }
  if (A->nnz > 0 && (!A->idx || !A->val))
    return fail(MSREP_ERR_INVALID_ARG, "idx or val is NULL");
  return MSREP_OK;
}

int32_t effective_tile(int32_t tile) { return tile == 0 ? kDefaultTile : tile; }

static msrep_status check_partition(const msrep_partition *p) {
  if (!p) return fail(MSREP_ERR_INVALID_ARG, "partition is NULL");
  if (p->np < 1) return fail(MSREP_ERR_INVALID_ARG, "np must be >= 1 (got %d)", p->np);
  if (!p->start_idx || !p->end_idx || !p->start_major || !p->end_major ||
      !p->start_flag)
    return fail(MSREP_ERR_INVALID_ARG, "a partition metadata array is NULL");
  if (!tile_supported(effective_tile(p->tile)))
    return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", p->tile);
  return MSREP_OK;
}

static msrep_status partition_compressed(const msrep_matrix *A,
                                         msrep_partition *p, unsigned flags,
                                         void *stream, int expect_fmt) {
  MSREP_TRY(check_matrix(A));
  if (A->fmt != expect_fmt)
    return fail(MSREP_ERR_INVALID_ARG, "matrix format %d does not match call",
                A->fmt);
  MSREP_TRY(check_partition(p));
  if (p->local && !p->local_off)
    return fail(MSREP_ERR_INVALID_ARG, "local pointers need local_off");
  cudaStream_t st = as_stream(stream);
  if (flags & MSREP_VALIDATE) MSREP_TRY(run_validation(A, st));
  const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
  const int32_t tile = effective_tile_fmt(p->tile, A->fmt);
  PlanLayout L = plan_layout(n_major, A->nnz, p->np, tile, A->fmt == MSREP_CSC);
  if (p->plan && p->plan_bytes < static_cast<int64_t>(L.bytes))
    return fail(MSREP_ERR_WORKSPACE, "plan buffer has %lld bytes, needs %zu",
                (long long)p->plan_bytes, L.bytes);
  if (p->plan && (reinterpret_cast<uintptr_t>(p->plan) & 15))
    return fail(MSREP_ERR_INVALID_ARG, "plan must be 16-byte aligned");
  char *plan = static_cast<char *>(p->plan);
  int64_t *D = plan ? reinterpret_cast<int64_t *>(plan + L.off_D) : nullptr;
  int32_t *R = plan ? reinterpret_cast<int32_t *>(plan + L.off_R) : nullptr;
  const int threads = 256;
  const int blocks = static_cast<int>(ceil_div(int64_t(p->np + 1) * 32, threads));
  if ((flags & MSREP_PART_MERGE_PATH) && (flags & MSREP_PART_ROW_BLOCK))
    return fail(MSREP_ERR_INVALID_ARG,
                "MSREP_PART_MERGE_PATH and MSREP_PART_ROW_BLOCK exclude each other");
  // CSC: the frequent-row search beside the rest
  SideStream *side = nullptr;
  if (plan && A->fmt == MSREP_CSC) {
    MSREP_TRY(fork_side(st, &side));
    int32_t *wtab = reinterpret_cast<int32_t *>(plan + L.off_wtab);
    MSREP_TRY(find_frequent_rows(A->idx, A->nnz, reinterpret_cast<int32_t *>(plan + L.off_hot),
                                 reinterpret_cast<unsigned long long *>(plan + L.off_warm), wtab,
                                 wtab + kWarmTab, side->s));
  }
  MSREP_TRY(launch_dependent(
      part_meta_compressed, blocks, threads, st, 0, A->ptr, n_major, A->nnz, p->np, p->start_idx,
      p->end_idx, p->start_major, p->end_major, p->start_flag, D, R,
      (flags & MSREP_PART_MERGE_PATH) ? int(kCutMergePath)
                                      : (flags & MSREP_PART_ROW_BLOCK) ? int(kCutRowBlock)
                                                                       : int(kCutNonzeros)));
  if (p->local_off) {
    MSREP_TRY(launch_dependent(local_off_scan, 1, 1024, st, 0,
                               static_cast<const int32_t *>(p->start_major),
                               static_cast<const int32_t *>(p->end_major), p->np, p->local_off));
    if (p->local) {
      // at most m + 2 np entries (n + 2 np for CSC)
      const int64_t most = int64_t(n_major) + 2 * int64_t(p->np);
      const int grid = static_cast<int>(
          std::max<int64_t>(1, std::min<int64_t>(ceil_div(most, 8 * 256), 8 * sm_count())));
      if ((reinterpret_cast<uintptr_t>(p->local) & 15) == 0)
        MSREP_TRY(launch_dependent(local_fill_compressed<true>, grid, 256, st, 0, A->ptr,
                                   p->start_idx, p->end_idx, p->start_major, p->end_major,
                                   p->local_off, p->np, p->local));
      else
        MSREP_TRY(launch_dependent(local_fill_compressed<false>, grid, 256, st, 0, A->ptr,
                                   p->start_idx, p->end_idx, p->start_major, p->end_major,
                                   p->local_off, p->np, p->local));
    }
  }
  if (plan) {
    int32_t *toff = reinterpret_cast<int32_t *>(plan + L.off_toff);
    int32_t *trow = reinterpret_cast<int32_t *>(plan + L.off_row);
    int32_t *tk = reinterpret_cast<int32_t *>(plan + L.off_k);
    MSREP_TRY(launch_dependent(plan_scan, 1, 1024, st, 0, D, p->np, tile, toff));
    MSREP_TRY(launch_dependent(plan_tiles, p->np, 128, st, 0, A->ptr, n_major, A->nnz, p->np, D,
                               R, toff, trow, tk));
  }
  if (side) MSREP_TRY(join_side(st, side));
  return ok();
}

}  // namespace msrep

using namespace msrep;

extern "C" {

const char *msrep_version(void) { return "msrep-gb300 0.1 (sm_103a)"; }

const char *msrep_last_error(void) { return g_last_error.c_str(); }

int msrep_tile_supported(int32_t tile) { return tile_supported(tile) ? 1 : 0; }

msrep_status msrep_partition_local_bound(const msrep_matrix *A, int32_t np,
                                         int64_t *entries) {
  MSREP_TRY(check_matrix(A));
  if (np < 1 || !entries) return fail(MSREP_ERR_INVALID_ARG, "bad np or entries");
  if (coo_format(A->fmt))
    *entries = A->nnz;
  else
    *entries = int64_t(A->fmt == MSREP_CSR ? A->m : A->n) + 2 * int64_t(np);
  return ok();
}

msrep_status msrep_plan_size(const msrep_matrix *A, int32_t np, int32_t tile,
                             int64_t *bytes) {
  MSREP_TRY(check_matrix(A));
  if (np < 1 || !bytes) return fail(MSREP_ERR_INVALID_ARG, "bad np or bytes");
  const int32_t t = effective_tile_fmt(tile, A->fmt);
  if (!tile_supported(t)) return fail(MSREP_ERR_INVALID_ARG, "unsupported tile %d", tile);
  if (A->fmt == MSREP_COO) {
    *bytes = 0;
    return ok();
  }
  if (coo_scatter_format(A->fmt)) {
    *bytes = static_cast<int64_t>(kScatterPlanBytes);
    return ok();
  }
  const int32_t n_major = A->fmt == MSREP_CSR ? A->m : A->n;
  *bytes = static_cast<int64_t>(plan_layout(n_major, A->nnz, np, t, A->fmt == MSREP_CSC).bytes);
  return ok();
}

msrep_status msrep_partition_csr(const msrep_matrix *A, msrep_partition *part,
                                 unsigned flags, void *stream) {
  return partition_compressed(A, part, flags, stream, MSREP_CSR);
}

msrep_status msrep_partition_csc(const msrep_matrix *A, msrep_partition *part,
                                 unsigned flags, void *stream) {
  return partition_compressed(A, part, flags, stream, MSREP_CSC);
}

msrep_status msrep_partition_coo(const msrep_matrix *A, msrep_partition *p,
                                 unsigned flags, void *stream) {
  MSREP_TRY(check_matrix(A));
  if (!coo_format(A->fmt))
    return fail(MSREP_ERR_INVALID_ARG, "matrix format %d is not COO", A->fmt);
  MSREP_TRY(check_partition(p));
  if (flags & MSREP_PART_MERGE_PATH)
    return fail(MSREP_ERR_INVALID_ARG, "merge-path partitioning takes CSR or CSC");
  if ((flags & MSREP_PART_ROW_BLOCK) && A->fmt == MSREP_COO_UNSORTED)
    return fail(MSREP_ERR_INVALID_ARG, "row-block partitioning needs sorted COO");
  const bool scatter = coo_scatter_format(A->fmt);
  if (scatter && p->plan) {
    if (p->plan_bytes < static_cast<int64_t>(kScatterPlanBytes))
      return fail(MSREP_ERR_WORKSPACE, "plan buffer has %lld bytes, needs %zu",
                  (long long)p->plan_bytes, kScatterPlanBytes);
    if (reinterpret_cast<uintptr_t>(p->plan) & 15)
      return fail(MSREP_ERR_INVALID_ARG, "plan must be 16-byte aligned");
  }
  cudaStream_t st = as_stream(stream);
  if (flags & MSREP_VALIDATE) MSREP_TRY(run_validation(A, st));
  // the major index: rows (sorted by row), columns (sorted by column)
  const int32_t *major = A->fmt == MSREP_COO_BY_COL ? A->idx : A->idx2;
  // scatter orders: the frequent-row search beside the metadata
  SideStream *side = nullptr;
  if (scatter && p->plan) {
    MSREP_TRY(fork_side(st, &side));
    char *plan = static_cast<char *>(p->plan);
    int32_t *wtab = reinterpret_cast<int32_t *>(plan + kScatterTabOff);
    MSREP_TRY(find_frequent_rows(A->idx2, A->nnz, reinterpret_cast<int32_t *>(plan),
                                 reinterpret_cast<unsigned long long *>(plan + kScatterWarmOff), wtab,
                                 wtab + kWarmTab, side->s));
  }
  const int threads = 256;
  const int blocks = static_cast<int>(ceil_div(p->np, threads));
  if (A->fmt == MSREP_COO_UNSORTED)
    MSREP_TRY(launch_dependent(part_meta_coo_unsorted, blocks, threads, st, 0, A->nnz, A->m,
                               p->np, p->start_idx, p->end_idx, p->start_major, p->end_major,
                               p->start_flag));
  else
    MSREP_TRY(launch_dependent(part_meta_coo, blocks, threads, st, 0, major, A->nnz, p->np,
                               p->start_idx, p->end_idx, p->start_major, p->end_major,
                               p->start_flag, A->fmt == MSREP_COO_BY_COL ? A->n : A->m,
                               (flags & MSREP_PART_ROW_BLOCK) ? 1 : 0));
  if (p->local && A->nnz > 0) {
    const int grid = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>(ceil_div(A->nnz, 8 * 256), 8 * sm_count())));
    if (((reinterpret_cast<uintptr_t>(p->local) | reinterpret_cast<uintptr_t>(major)) & 15) == 0)
      MSREP_TRY(launch_dependent(local_fill_coo<true>, grid, 256, st, 0, major, A->nnz, p->np,
                                 p->start_idx, p->start_major, p->local));
    else
      MSREP_TRY(launch_dependent(local_fill_coo<false>, grid, 256, st, 0, major, A->nnz, p->np,
                                 p->start_idx, p->start_major, p->local));
  }
  if (side) MSREP_TRY(join_side(st, side));
  return ok();
}

}  // extern "C"
