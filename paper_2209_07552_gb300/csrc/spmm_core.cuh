// k right-hand sides at once (Y = alpha * A * X + beta * Y, k <= 8) over
// the same CSR tiles as the SpMV: the served form's sweep of up to eight x
// vectors per request.  X is read interleaved, row c of X holding the KP
// values x_0[c] .. x_{KP-1}[c] (KP = k rounded up to 1, 2, 4 or 8), so a
// nonzero gathers one contiguous 4..64-byte segment, and the matrix is
// streamed once for all k vectors.
//
// Thread layout: TPV threads share lane vl of a tile, each holding VPT =
// KP / TPV of the vectors (one vector load of its part of the x row per
// nonzero).  A block of 256 threads holds G = 8 / TPV tile groups of 32 *
// TPV threads, each walking its own tiles and synchronising only with
// itself.
// Each thread walks exactly the nonzeros that lane vl of the SpMV's warp
// walks, with the same FMAs in the same order for each of its vectors
// (masked positions included), and finishes the same rows; the SpMV's warp
// segmented scan then runs once per (tile, vector) on the lane partials,
// gathered through shared memory.  So Y[:, v] equals msrep_spmv of x_v bit
// for bit.  TPV is kept small (VPT up to 4 FP32 or 2 FP64 values) so that a
// block holds many tiles: the tile walk is a chain of dependent memory
// round trips, and tiles in flight set the throughput.
#pragma once

#include "spmv_core.cuh"

namespace msrep {

template <class Pol, int KP>
struct SpmmArgs {
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const typename Pol::V *val;
  const typename Pol::X *xt;  // [n][KP] interleaved
  typename Pol::X *y;         // y[v * ldy + row], v < k
  int64_t ldy;
  int k;
  double alpha, beta;
  int finish;
  const int32_t *tile_row, *tile_k;
  double *head, *tail;  // [T][hs]: tile b's partial of vector v at b * hs + v
  int hs;               // head / tail stride (>= KP)
  int32_t m;
  unsigned comp_mode;
};

// KP of a request of k vectors: k rounded up to 1, 2, 4 or 8
__host__ __device__ constexpr int spmm_width(int k) {
  return k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : 8;
}

// threads per lane: at most 4 FP32 (16 bytes) or 2 FP64 x values a thread
template <class X, int KP>
struct KvShape {
  static constexpr int VMAX = sizeof(X) == 8 ? 2 : 4;
  static constexpr int TPV = KP > VMAX ? KP / VMAX : 1;
  static constexpr int VPT = KP / TPV;
  static constexpr int G = 8 / TPV;  // tile groups of a 256-thread block
  static constexpr int GT = 32 * TPV;  // threads of a tile group
};

constexpr int kKvWarps = 8;
constexpr int kKvThreads = 32 * kKvWarps;
constexpr int kKvRowSlots = 32 * 32 + 8;  // row pointers of a tile of <= 1024

// Shared memory of a block: the row pointers of its GS tile groups, the
// lane partials of the scans (four rows of 33 per warp, [vector][lane],
// 33 against bank conflicts) and the lanes' row-finished flags.
template <class Acc, int GS>
struct KvSmem {
  int32_t rp[GS][kKvRowSlots];
  Acc part[32 * 33];
  int32_t flag[GS * 32];
};

// VPT consecutive x values (16-byte vector loads where they fit)
template <int VPT>
__device__ __forceinline__ void ldx(const float *p, float (&o)[VPT]) {
  if constexpr (VPT == 1) {
    o[0] = __ldg(p);
  } else if constexpr (VPT == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = t.x;
    o[1] = t.y;
  } else {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
}
template <int VPT>
__device__ __forceinline__ void ldx(const double *p, double (&o)[VPT]) {
  if constexpr (VPT == 1) {
    o[0] = __ldg(p);
  } else {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = t.x;
    o[1] = t.y;
  }
}

// kCopy: alpha = 1, beta = 0 known at compile time (the copy finish)
template <class Pol, int KP, bool kCopy = false>
__device__ __forceinline__ void spmm_write_row(const SpmmArgs<Pol, KP> &a, int v, int32_t row,
                                               typename Pol::Acc acc) {
  if (v < a.k) {
    typename Pol::X *yp = a.y + v * a.ldy + row;
    *yp = Pol::finish(acc, kCopy ? int(kFinishCopy) : a.finish, a.alpha, a.beta, yp);
  }
}

// Synchronise the GT threads of tile group ts (a warp, or a named barrier
// over the group's warps).
template <int GT>
__device__ __forceinline__ void group_sync(int ts) {
  if constexpr (GT == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(ts + 1), "n"(GT) : "memory");
}

// Tile b by tile group ts (threads ts*GT .. ts*GT+GT-1 of the block; all
// of them call it).  Shared memory used: rp[ts] and the partial rows
// ts*TPV*4 .. ts*TPV*4 + KP - 1, so groups never touch each other's
// slots and synchronise only among themselves.
template <class Pol, int KP, int GS, bool kCopy = false>
__device__ __forceinline__ void kv_tile(const SpmmArgs<Pol, KP> &a, int b, int64_t nnz,
                                        KvSmem<typename Pol::Acc, GS> &sm, int ts) {
  using Acc = typename Pol::Acc;
  using LV = typename LoadT<typename Pol::V>::type;
  using X = typename Pol::X;
  using Sh = KvShape<X, KP>;
  constexpr int TPV = Sh::TPV, VPT = Sh::VPT, GT = 32 * TPV;
  static_assert(GS >= Sh::G, "too few row-pointer slots");
  const int q = threadIdx.x % GT, vl = q / TPV, v0 = (q % TPV) * VPT;
  const int prow = ts * TPV * 4;  // first partial row of the group
  int32_t *rp = sm.rp[ts];
  const int32_t r0 = __ldg(a.tile_row + b), k0 = __ldg(a.tile_k + b);
  const int32_t r1 = __ldg(a.tile_row + b + 1), k1 = __ldg(a.tile_k + b + 1);
  {
    const int32_t rend = min(r1 + 2, a.m + 1);
    for (int32_t r = r0 + q; r < rend; r += GT) rp[r - r0] = __ldg(a.row_ptr + r);
  }
  group_sync<GT>(ts);

  // lane vl of csr_tile_compute, for vectors v0 .. v0 + VPT - 1
  Acc acc[VPT], first_acc[VPT];
#pragma unroll
  for (int j = 0; j < VPT; ++j) acc[j] = first_acc[j] = Pol::zero();
  bool emitted = false;
  int first_r = 0;
  const int nrows = r1 - r0;
  const int32_t rs0 = rp[0];
  const int32_t *s_end = rp + 1;
  const bool flag = rs0 < k0;
  {
    const LaneRange lr = lane_range(k0, k1, vl);
    const int32_t ka = static_cast<int32_t>(lr.ka), kb = static_cast<int32_t>(lr.kb);
    int r = vl == 0 ? 0 : upper_bound_smem(s_end, nrows, ka);
    const int r_end = upper_bound_smem(s_end, nrows, kb);
    int32_t next_end = r < r_end ? s_end[r] : INT32_MAX;
    int32_t re_last = 0;
    if (Pol::kLow) re_last = (r1 < a.m) ? rp[nrows + 1] : k1;
    auto row_comp = [&](int rr) -> bool {
      if (!Pol::kLow) return false;
      int64_t st = rr == 0 ? int64_t(rs0) : int64_t(s_end[rr - 1]);
      int64_t en = rr < nrows ? int64_t(s_end[rr]) : int64_t(re_last);
      return want_comp(a.comp_mode, en - st, (rr == 0 && flag) || rr == nrows);
    };
    bool comp = row_comp(r);
    auto finish_rows = [&](int32_t kk) {
      while (next_end <= kk) {
        if (!emitted) {
          emitted = true;
          first_r = r;
#pragma unroll
          for (int j = 0; j < VPT; ++j) first_acc[j] = acc[j];
        } else {
#pragma unroll
          for (int j = 0; j < VPT; ++j) spmm_write_row<Pol, KP, kCopy>(a, v0 + j, r0 + r, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < VPT; ++j) acc[j] = Pol::zero();
        ++r;
        next_end = r < r_end ? s_end[r] : INT32_MAX;
        comp = row_comp(r);
      }
    };
    finish_rows(ka);
    const X *xv_base = a.xt + v0;
    for (int64_t g = lr.glo; g < lr.ghi; ++g) {
      const int64_t g8 = g << 3;
      int32_t c[8];
      LV vv[8];
      X xv[8][VPT];
      load_group(a.col_idx, g8, nnz, c);
      load_group(a.val, g8, nnz, vv);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = g8 + u >= ka && g8 + u < kb;
        if (in) {
          ldx<VPT>(xv_base + int64_t(c[u]) * KP, xv[u]);
        } else {
#pragma unroll
          for (int j = 0; j < VPT; ++j) xv[u][j] = X(0);
          vv[u] = LV(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        // a branch, not a select: the compensated update is about ten
        // instructions a vector and rows that need it are few
        if (Pol::kLow && comp) {
#pragma unroll
          for (int j = 0; j < VPT; ++j) acc[j] = Pol::fma(acc[j], vv[u], xv[u][j], true);
        } else {
#pragma unroll
          for (int j = 0; j < VPT; ++j) acc[j] = Pol::fma(acc[j], vv[u], xv[u][j], false);
        }
        const int32_t kk = static_cast<int32_t>(g8 + u + 1);
        if (next_end <= kk) finish_rows(kk);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < VPT; ++j) sm.part[(prow + v0 + j) * 33 + vl] = acc[j];
  if (v0 == 0) sm.flag[ts * 32 + vl] = emitted;
  group_sync<GT>(ts);

  // the group's warps scan its KP vectors (warp wg: vectors wg*VPT ..),
  // each as warp_seg_scan does for the SpMV's warp
  {
    const int lane = threadIdx.x & 31, wg = q >> 5;
    const bool f = sm.flag[ts * 32 + lane] != 0;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const int vw = wg * VPT + j, idx = (prow + vw) * 33 + lane;
      Acc last;
      const Acc ex = warp_seg_scan<Pol>(f, sm.part[idx], last);
      sm.part[idx] = ex;
      if (lane == 31) {
        double *dst = nullptr;
        if (nrows == 0) {
          if (flag)
            dst = a.head;
          else if (k1 > k0)
            dst = a.tail;
        } else if (k1 > rp[nrows]) {
          dst = a.tail;
        }
        if (dst) dst[int64_t(b) * a.hs + vw] = Pol::to_f64(last);
      }
    }
  }
  group_sync<GT>(ts);
  if (emitted) {
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const Acc tot = Pol::combine(sm.part[(prow + v0 + j) * 33 + vl], first_acc[j]);
      if (first_r == 0 && flag)
        a.head[int64_t(b) * a.hs + v0 + j] = Pol::to_f64(tot);
      else
        spmm_write_row<Pol, KP, kCopy>(a, v0 + j, r0 + first_r, tot);
    }
  }
  // the next tile of this group rewrites rp only after every thread of
  // the group has passed the scan above (which read it)
}

// fixup_tile for KP vectors: partials at head/tail[tile * KP + v]; the sums
// are formed in the same order as fixup_tile's, vector by vector.
template <class X, int KP, class View>
__device__ __forceinline__ void fixup_tile_k(const View &v, int T, int b, const double *head,
                                             const double *tail, X *y, int64_t ldy, int k,
                                             double alpha, double beta) {
  int32_t r;
  if (!fixup_run_start(v, T, b, r)) return;
  // length of the run of tiles b, b+1, ... that continue row r
  int run = 0;
  for (int j0 = b;; j0 += 8) {
    int32_t rj[8];
    bool fj[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      fj[u] = false;
      if (j0 + u < T) v.row_flag(j0 + u, rj[u], fj[u]);
    }
    int n8 = 8;
#pragma unroll
    for (int u = 7; u >= 0; --u)
      if (!(fj[u] && rj[u] == r)) n8 = u;
    run += n8;
    if (n8 < 8) break;
  }
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    if (j >= k) break;
    double s = tail[int64_t(b - 1) * KP + j];
    for (int t = 0; t < run; ++t) s += head[int64_t(b + t) * KP + j];
    X *yp = y + j * ldy + r;
    *yp = static_cast<X>(finish_merged(s, alpha, beta, beta == 0.0 ? 0.0 : double(*yp)));
  }
}

}  // namespace msrep
