// Shared helpers of the msRep CUDA library: status plumbing, typed loads,
// error-free FP32 transformations and launch-shape queries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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

// Sets a kernel's preferred shared-memory carveout to the smallest share of
// the SM's unified L1/shared memory that holds `blocks` resident blocks
// (static + dyn_smem bytes each), leaving the rest to L1.  The x gathers of
// the CSR kernels hit L1 (17-60%); with CUDA's default carveout R-MAT
// CSR took 108 us, with the smallest one 103 us.  No-op for kernels without
// shared memory (they keep the default, all L1).  Current device.
msrep_status set_min_carveout(const void *kernel, size_t dyn_smem, int blocks);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// tile shapes
// ---------------------------------------------------------------------------

// A tile is 32 * IPT merge-path items (rows + nonzeros for CSR/CSC,
// nonzeros for COO), processed by one warp.  The supported shapes are
// instantiated in spmv.cu.
constexpr int kDefaultTile = 512;
// CSC's default: the interleaved walk of its scatter (csc_tile_interleaved)
// is fastest at 256 items per tile on both the R-MAT and the Laplacian
// workloads (105 / 75 us against 111 / 84 us at 512).
constexpr int kDefaultTileCsc = 256;
inline bool tile_supported(int t) {
  return t == 256 || t == 512 || t == 1024;
}
// The tile a partition of format fmt uses (0 = the format's default).
inline int32_t effective_tile_fmt(int32_t tile, int32_t fmt) {
  return tile != 0 ? tile : (fmt == MSREP_CSC ? kDefaultTileCsc : kDefaultTile);
}

// ---------------------------------------------------------------------------
// tile plan layout (CSR/CSC), all in one device buffer
// ---------------------------------------------------------------------------
//   int64  D[np+1]        merge-path diagonal of each level-1 cut
//   int32  R[np+1]        row (column) coordinate of each cut
//   int32  tile_off[np+1] first tile of each partition; tile_off[np] = T
//   int32  tile_row[Tmax+1], tile_k[Tmax+1]  tile start coordinates; the
//                         entry after the last tile is (n_major, nnz).
//   int32  hot[1+kMaxHot] CSC only: count, then the hub rows (-1 = none)
//   uint64 warm[kWarm]    CSC only: the frequent-row table,
//                         (priority << 32) | ~row per slot, 0 = empty
//   int32  wkey[kWarmTab], wcnt[kWarmTab], whist[256]  CSC only:
//                         partition-time scratch of the frequent-row search
struct PlanLayout {
  int64_t tmax;
  size_t off_D, off_R, off_toff, off_row, off_k, off_hot, off_warm, off_wtab, bytes;
};

// Hub rows of a CSC matrix: rows holding a large share of the nonzeros, so
// that their atomic adds to one y entry serialise in L2.  At most kMaxHot
// of them are found at partition time, from kHotSample evenly spaced
// nonzeros; a row needs at least kHotMin samples (about 0.1% of the
// nonzeros) to qualify.
constexpr int kMaxHot = 4;
constexpr int kHotSample = 4096;
constexpr int kHotMin = 4;

// When a CSC matrix has hub rows, its scatter accumulates into a workspace
// vector whose entry for row r is slot(r) = (r * kPermMul) mod 2^k, a
// bijection of [0, 2^k) for the odd multiplier, with 2^k >= m (perm_extent).
// A power-law matrix's heavy rows crowd a few cache lines of y (in the R-MAT
// workload the rows 0..15 of one 128-byte line take 150,000 atomic adds), so
// the L2 slices holding those lines serialise the scatter; the permuted
// layout spreads them over all slices.  y is gathered back afterwards.
constexpr uint32_t kPermMul = 0x9E3779B1u;
inline int64_t perm_extent(int64_t m) {
  int64_t e = 1;
  while (e < m) e <<= 1;
  return e;
}
__host__ __device__ __forceinline__ uint32_t perm_slot(int32_t r, uint32_t mask) {
  return (static_cast<uint32_t>(r) * kPermMul) & mask;
}

// Frequent rows of a scatter with hub rows: each thread block sums the
// products of up to kWarm frequent rows in shared memory and adds each sum
// to the accumulator once, at its end, instead of one atomic add per
// nonzero.  The rows sit in a direct-mapped table, row r in slot
// warm_slot(r) (the top bits of r * kPermMul, so rows that differ only in
// their high bits spread out); a slot holds one row.  They are chosen at
// partition time from kWarmSample evenly spaced nonzeros, counted in a
// kWarmTab-slot hash table: the hub rows and every row whose sample count
// reaches the largest threshold (>= kWarmMin) that at most kWarm rows reach
// claim their slots, and a slot keeps the most frequent claimant (hub rows
// first, the smaller row on ties).  On the R-MAT workload this removes about
// a fifth of the atomic adds of its scatter.
constexpr int kWarmBits = 11;
constexpr int kWarm = 1 << kWarmBits;
constexpr int kWarmSample = 1 << 16;
constexpr int kWarmTabBits = 17;
constexpr int kWarmTab = 1 << kWarmTabBits;
constexpr int kWarmMin = 2;
__host__ __device__ __forceinline__ uint32_t warm_slot(int32_t r) {
  return (static_cast<uint32_t>(r) * kPermMul) >> (32 - kWarmBits);
}

// Internal entry of msrep_spmv.  perm_ok: the workspace holds the permuted
// CSC accumulator (msrep_spmv_workspace_size counts it); without it a CSC
// SpMV scatters into y directly (msrep_spmv_noalloc when its scratch array
// is too small for the accumulator).
msrep_status spmv_workspace_bytes(const msrep_matrix *A, const msrep_partition *part,
                                  bool perm_ok, size_t *bytes);
msrep_status spmv_run(const msrep_matrix *A, const msrep_partition *part, double alpha,
                      const void *x, double beta, void *y, int32_t xy_dtype, unsigned flags,
                      void *workspace, void *stream, bool perm_ok);

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// warm: the CSC plan, which also holds the frequent-row table and its
// partition-time scratch.
inline PlanLayout plan_layout(int64_t n_major, int64_t nnz, int32_t np,
                              int32_t tile, bool warm = false) {
  PlanLayout L;
  // sum over partitions of ceil(len_i / tile) <= (n_major + nnz)/tile + np
  L.tmax = (n_major + nnz) / tile + np + 1;
  size_t o = 0;
  L.off_D = o;    o = align256(o + sizeof(int64_t) * (np + 1));
  L.off_R = o;    o = align256(o + sizeof(int32_t) * (np + 1));
  L.off_toff = o; o = align256(o + sizeof(int32_t) * (np + 1));
  L.off_row = o;  o = align256(o + sizeof(int32_t) * (L.tmax + 1));
  L.off_k = o;    o = align256(o + sizeof(int32_t) * (L.tmax + 1));
  L.off_hot = o;  o = align256(o + sizeof(int32_t) * (1 + kMaxHot));
  L.off_warm = o;
  L.off_wtab = o;
  if (warm) {
    o = align256(o + sizeof(uint64_t) * kWarm);
    L.off_wtab = o;
    o = align256(o + sizeof(int32_t) * (2 * kWarmTab + 256));
  }
  L.bytes = o;
  return L;
}

// COO sorted by column or in no order: every partition may add to any row,
// so its SpMV is a scatter, and its plan holds only what that scatter
// needs: the hub rows (int32 hot[1+kMaxHot] at offset 0), the frequent-row
// table (uint64 warm[kWarm] at kScatterWarmOff) and the scratch of its
// search (at kScatterTabOff).
inline bool coo_scatter_format(int32_t fmt) {
  return fmt == MSREP_COO_BY_COL || fmt == MSREP_COO_UNSORTED;
}
inline bool coo_format(int32_t fmt) { return fmt == MSREP_COO || coo_scatter_format(fmt); }
constexpr size_t kScatterWarmOff = 256;
constexpr size_t kScatterTabOff = kScatterWarmOff + sizeof(uint64_t) * kWarm;
constexpr size_t kScatterPlanBytes = kScatterTabOff + sizeof(int32_t) * (2 * kWarmTab + 256);

// COO tiles: each partition is split into the same number G of sub-ranges
// (Alg. 2's split applied inside the partition).
inline int64_t coo_tiles_per_part(int64_t nnz, int32_t np, int32_t tile) {
  int64_t per = ceil_div(nnz, np);
  int64_t g = ceil_div(per, tile);
  return g < 1 ? 1 : g;
}

// ---------------------------------------------------------------------------
// programmatic dependent launch
// ---------------------------------------------------------------------------

// Kernels launched with launch_dependent may start while the kernel before
// them on the stream drains; they wait here (a no-op without that launch
// attribute) before reading what it wrote.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launches a kernel that depends on the previous one on the stream as a
// programmatic dependent launch: its blocks may be scheduled while that
// kernel's last blocks drain, hiding the launch gap; the kernel itself waits
// (grid_dependency_wait) before touching the results.
template <class... KArgs, class... Args>
inline msrep_status launch_dependent(void (*kernel)(KArgs...), int64_t grid, int block,
                                     cudaStream_t st, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(std::max<int64_t>(grid, 1)));
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MSREP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
  return MSREP_OK;
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

// Group loads: 8 consecutive elements starting at an index that is a
// multiple of 8, as one 256-bit (or 128-bit for bf16) load that bypasses L1
// (the nonzero stream is read once; L1 is left to the x gathers).  The
// arrays must be 32-byte aligned (16-byte for bf16 values).
__device__ __forceinline__ void ld8(const int32_t *p, int32_t (&r)[8]) {
  asm("ld.global.nc.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7])
      : "l"(p));
}
__device__ __forceinline__ void ld8(const double *p, double (&v)[8]) {
  asm("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
      : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
      : "l"(p));
  asm("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
      : "=d"(v[4]), "=d"(v[5]), "=d"(v[6]), "=d"(v[7])
      : "l"(p + 4));
}
__device__ __forceinline__ void ld8(const float *p, float (&v)[8]) {
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
        "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}
__device__ __forceinline__ void ld8(const bf16_t *p, float (&v)[8]) {
  uint32_t w[4];
  asm("ld.global.nc.L1::no_allocate.v4.b32 {%0,%1,%2,%3}, [%4];"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
      : "l"(p));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// binary32 -> binary64 widening for the scatter's exact FP64 products.  A
// normal number is widened by the IEEE-754 formats' definition in integer
// operations: its 8-bit exponent and 23-bit fraction, shifted right by 3,
// land on the 11-bit exponent and top 20 fraction bits of the high word,
// where adding (1023 - 127) << 20 rebiases the exponent; the last 3
// fraction bits go to the top of the low word; the sign stays.  Zero,
// subnormal, infinite and NaN inputs take the hardware conversion, called
// out of line so that the compiler cannot evaluate it for every element: on
// GB300 it runs on the FP64 pipe (about two lane operations per clock per
// SM), where a scatter that widened two operands per nonzero spent most of
// its time.
static __device__ __noinline__ double widen_rare(float f) { return static_cast<double>(f); }
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) - 0x00800000u >= 0x7f000000u) return widen_rare(f);
  const uint32_t hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
}
__device__ __forceinline__ double widen(double d) { return d; }

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
