// k right-hand sides at once (Y = alpha * A * X + beta * Y, k <= 8) over
// the same CSR tiles as the SpMV: the served form's sweep of up to eight x
// vectors per request.  X is read interleaved, row c of X holding the KP
// values x_0[c] .. x_{KP-1}[c] (KP = k rounded up to 1, 2, 4 or 8), so one
// nonzero gathers one 4..64-byte segment instead of k scattered values, and
// the matrix is streamed once for all k vectors.  Every vector's sums follow
// the SpMV's order exactly (one FMA per nonzero in the lane's order, the
// same warp scan and tile merge), so Y[:, v] equals msrep_spmv of x_v bit
// for bit.
#pragma once

#include "spmv_core.cuh"
#include "tma.cuh"

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
  double *head, *tail;  // [T][KP]
  int32_t m;
  unsigned comp_mode;
};

template <class Pol, int KP>
__device__ __forceinline__ void spmm_write_row(const SpmmArgs<Pol, KP> &a, int32_t row,
                                               const typename Pol::Acc (&acc)[KP]) {
#pragma unroll
  for (int j = 0; j < KP; ++j)
    if (j < a.k) {
      typename Pol::X *yp = a.y + j * a.ldy + row;
      *yp = Pol::finish(acc[j], a.finish, a.alpha, a.beta, yp);
    }
}

// warp_seg_scan over KP values at once (same flags, same steps, so each
// value's scan is the one warp_seg_scan would do)
template <class Pol, int KP>
__device__ __forceinline__ void warp_seg_scan_k(bool flag, typename Pol::Acc (&inc)[KP],
                                                typename Pol::Acc (&ex)[KP],
                                                typename Pol::Acc (&last)[KP]) {
  const int lane = threadIdx.x & 31;
  int f = flag;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (__all_sync(0xffffffffu, f || lane < o)) break;
    const int fu = __shfl_up_sync(0xffffffffu, f, o);
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const typename Pol::Acc u = Pol::shfl_up(inc[j], o);
      if (lane >= o && !f) inc[j] = Pol::combine(u, inc[j]);
    }
    if (lane >= o) f |= fu;
  }
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    ex[j] = Pol::shfl_up(inc[j], 1);
    if (lane == 0) ex[j] = Pol::zero();
    last[j] = Pol::shfl(inc[j], 31);
  }
}

// Shared-memory slots of one lane: S gathered x rows (ROW bytes each), then
// the S values they multiply.
template <class Pol, int KP>
struct SpmmStage {
  using X = typename Pol::X;
  using LV = typename LoadT<typename Pol::V>::type;
  static constexpr int ROW = KP * sizeof(X);
  static constexpr int S = ROW > 32 ? 4 : 8;  // nonzeros staged at a time
  static constexpr int LANE = (S * ROW + S * sizeof(LV) + 15) / 16 * 16;
  static constexpr int WARP = 32 * LANE;
};

// Asynchronous copy of one ROW-byte x row into shared memory (cp.async,
// 4, 8 or 16 bytes per instruction); a row that is not needed is filled
// with zeros (source size 0, nothing read).
template <int ROW>
__device__ __forceinline__ void gather_row(void *dst, const void *src, bool in) {
  const uint32_t d = smem_addr(dst);
  if constexpr (ROW < 16) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(ROW),
                 "r"(in ? ROW : 0)
                 : "memory");
  } else {
#pragma unroll
    for (int i = 0; i < ROW / 16; ++i)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d + 16 * i),
                   "l"(static_cast<const char *>(src) + 16 * i), "r"(in ? 16 : 0)
                   : "memory");
  }
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int KP>
__device__ __forceinline__ void lds_row(const float *p, float (&o)[KP]) {
  if constexpr (KP == 1) {
    o[0] = p[0];
  } else if constexpr (KP == 2) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    o[0] = t.x;
    o[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < KP / 4; ++i) {
      const float4 t = reinterpret_cast<const float4 *>(p)[i];
      o[4 * i] = t.x;
      o[4 * i + 1] = t.y;
      o[4 * i + 2] = t.z;
      o[4 * i + 3] = t.w;
    }
  }
}
template <int KP>
__device__ __forceinline__ void lds_row(const double *p, double (&o)[KP]) {
  if constexpr (KP == 1) {
    o[0] = p[0];
  } else {
#pragma unroll
    for (int i = 0; i < KP / 2; ++i) {
      const double2 t = reinterpret_cast<const double2 *>(p)[i];
      o[2 * i] = t.x;
      o[2 * i + 1] = t.y;
    }
  }
}

// csr_tile_compute with KP accumulators per lane; see there for the layout
// of rp and the meaning of the tile coordinates.  `stage`: this lane's
// SpmmStage slots (16-byte aligned shared memory).
template <class Pol, int KP>
__device__ __forceinline__ void csr_tile_compute_k(const SpmmArgs<Pol, KP> &a, int b, int32_t r0,
                                                   int32_t k0, int32_t r1, int32_t k1,
                                                   const int32_t *rp, int64_t nnz,
                                                   unsigned char *stage) {
  using Acc = typename Pol::Acc;
  using LV = typename LoadT<typename Pol::V>::type;
  using X = typename Pol::X;
  const int lane = threadIdx.x & 31;
  const int nrows = r1 - r0;
  const int32_t rs0 = rp[0];
  const int32_t *s_end = rp + 1;
  const bool flag = rs0 < k0;

  const LaneRange lr = lane_range(k0, k1, lane);
  const int32_t ka = static_cast<int32_t>(lr.ka), kb = static_cast<int32_t>(lr.kb);
  int r = lane == 0 ? 0 : upper_bound_smem(s_end, nrows, ka);
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

  Acc acc[KP], first_acc[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) acc[j] = first_acc[j] = Pol::zero();
  bool emitted = false, comp = row_comp(r);
  int first_r = 0;
  auto finish_rows = [&](int32_t kk) {
    while (next_end <= kk) {
      if (!emitted) {
        emitted = true;
        first_r = r;
#pragma unroll
        for (int j = 0; j < KP; ++j) first_acc[j] = acc[j];
      } else {
        spmm_write_row(a, r0 + r, acc);
      }
#pragma unroll
      for (int j = 0; j < KP; ++j) acc[j] = Pol::zero();
      ++r;
      next_end = r < r_end ? s_end[r] : INT32_MAX;
      comp = row_comp(r);
    }
  };
  finish_rows(ka);

  // Each lane gathers the x rows of S nonzeros at a time into its own
  // shared-memory slots with asynchronous copies (all S gathers in flight,
  // no registers held), then consumes them in a rolled loop, so the
  // per-row code (KP accumulators, compensation, row finishing) exists once
  // in the kernel instead of once per unrolled element: unrolled 8-fold it
  // overflowed the instruction cache.
  using St = SpmmStage<Pol, KP>;
  X *sx = reinterpret_cast<X *>(stage);
  LV *sv = reinterpret_cast<LV *>(stage + St::S * St::ROW);
  for (int64_t g = lr.glo; g < lr.ghi; ++g) {
    const int64_t g8 = g << 3;
    int32_t c[8];
    LV v[8];
    load_group(a.col_idx, g8, nnz, c);
    load_group(a.val, g8, nnz, v);
#pragma unroll
    for (int h = 0; h < 8; h += St::S) {
#pragma unroll
      for (int u = 0; u < St::S; ++u) {
        const bool in = g8 + h + u >= ka && g8 + h + u < kb;
        const X *src = a.xt + (in ? int64_t(c[h + u]) * KP : 0);
        gather_row<St::ROW>(sx + u * KP, src, in);
        sv[u] = in ? v[h + u] : LV(0);
      }
      cp_async_wait_all();
#pragma unroll 1
      for (int u = 0; u < St::S; ++u) {
        X xr[KP];
        lds_row<KP>(sx + u * KP, xr);
        const LV vu = sv[u];
        // a branch, not a select: the compensated update is about ten
        // instructions a vector and rows that need it are few
        if (Pol::kLow && comp) {
#pragma unroll
          for (int j = 0; j < KP; ++j) acc[j] = Pol::fma(acc[j], vu, xr[j], true);
        } else {
#pragma unroll
          for (int j = 0; j < KP; ++j) acc[j] = Pol::fma(acc[j], vu, xr[j], false);
        }
        const int32_t kk = static_cast<int32_t>(g8 + h + u + 1);
        if (next_end <= kk) finish_rows(kk);
      }
    }
  }

  Acc carry[KP], last[KP];
  warp_seg_scan_k<Pol, KP>(emitted, acc, carry, last);
  if (emitted) {
    Acc tot[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) tot[j] = Pol::combine(carry[j], first_acc[j]);
    if (first_r == 0 && flag) {
#pragma unroll
      for (int j = 0; j < KP; ++j) a.head[int64_t(b) * KP + j] = Pol::to_f64(tot[j]);
    } else {
      spmm_write_row(a, r0 + first_r, tot);
    }
  }
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
    if (dst) {
#pragma unroll
      for (int j = 0; j < KP; ++j) dst[int64_t(b) * KP + j] = Pol::to_f64(last[j]);
    }
  }
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
