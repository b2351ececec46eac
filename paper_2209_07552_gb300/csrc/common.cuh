// Shared helpers of the msRep CUDA library: status plumbing, typed loads,
// error-free FP32 transformations and launch-shape queries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>

#include "msrep.h"

namespace msrep {

// ---------------------------------------------------------------------------
// host-side status plumbing
// ---------------------------------------------------------------------------

// Records a message for msrep_last_error() and returns `st`.
msrep_status fail(msrep_status st, const char *fmt, ...);
// Clears the thread's last error and returns MSREP_OK.
msrep_status ok();

#define MSREP_CUDA_TRY(expr)                                                  \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return ::msrep::fail(MSREP_ERR_CUDA, "%s: %s (%s:%d)", #expr,           \
                           cudaGetErrorString(e_), __FILE__, __LINE__);       \
  } while (0)

#define MSREP_TRY(expr)                                                       \
  do {                                                                        \
    msrep_status s_ = (expr);                                                 \
    if (s_ != MSREP_OK) return s_;                                            \
  } while (0)

// Number of SMs of the current device (cached per device).
int sm_count();

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// tile shapes
// ---------------------------------------------------------------------------

// A tile is 32 * IPT merge-path items (rows + nonzeros for CSR/CSC,
// nonzeros for COO), processed by one warp.  The supported shapes are
// instantiated in spmv.cu.
constexpr int kDefaultTile = 256;
inline bool tile_supported(int t) {
  return t == 128 || t == 256 || t == 512 || t == 1024;
}

// ---------------------------------------------------------------------------
// tile plan layout (CSR/CSC), all in one device buffer
// ---------------------------------------------------------------------------
//   int64  D[np+1]        merge-path diagonal of each level-1 cut
//   int32  R[np+1]        row (column) coordinate of each cut
//   int32  tile_off[np+1] first tile of each partition; tile_off[np] = T
//   int32  tile_row[Tmax+1], tile_k[Tmax+1]  tile start coordinates; the
//                         entry after the last tile is (n_major, nnz).
struct PlanLayout {
  int64_t tmax;
  size_t off_D, off_R, off_toff, off_row, off_k, bytes;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

inline PlanLayout plan_layout(int64_t n_major, int64_t nnz, int32_t np,
                              int32_t tile) {
  PlanLayout L;
  // sum over partitions of ceil(len_i / tile) <= (n_major + nnz)/tile + np
  L.tmax = (n_major + nnz) / tile + np + 1;
  size_t o = 0;
  L.off_D = o;    o = align256(o + sizeof(int64_t) * (np + 1));
  L.off_R = o;    o = align256(o + sizeof(int32_t) * (np + 1));
  L.off_toff = o; o = align256(o + sizeof(int32_t) * (np + 1));
  L.off_row = o;  o = align256(o + sizeof(int32_t) * (L.tmax + 1));
  L.off_k = o;    o = align256(o + sizeof(int32_t) * (L.tmax + 1));
  L.bytes = o;
  return L;
}

// COO tiles: each partition is split into the same number G of sub-ranges
// (Alg. 2's split applied inside the partition).
inline int64_t coo_tiles_per_part(int64_t nnz, int32_t np, int32_t tile) {
  int64_t per = ceil_div(nnz, np);
  int64_t g = ceil_div(per, tile);
  return g < 1 ? 1 : g;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

struct bf16_t {
  uint16_t bits;
};

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ double to_double(double v) { return v; }

// Streaming loads of the nonzero arrays: read once, keep out of L1 and mark
// evict-first in L2 so that x stays resident.
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const bf16_t *p) {
  unsigned short b = __ldcs(reinterpret_cast<const unsigned short *>(p));
  return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no FMA
// contraction possible on these operations because each is a single add).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float aa = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// TwoProduct via FMA: p + e == a * b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

}  // namespace msrep
