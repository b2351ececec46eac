// The batch directory shared by the batched form and the server: one entry
// per SpMV item, and the launcher of the persistent batched kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "msrep.h"

namespace msrep {

// one matrix of a batch, as the kernels see it (x and y come from the
// launch's pointer arrays)
struct BatchItem {
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const void *val;
  const int32_t *tile_row;
  const int32_t *tile_k;
  int32_t m, n;
  int64_t nnz;
  int32_t k;    // vectors of the item (the k-vector form; 1 for the SpMV form)
  int32_t pad;
};

// Width of the interleaved x of the batched k-vector form (the server's
// requests with 2..8 vectors): row c holds x_0[c] .. x_7[c], one 32-byte
// segment per nonzero for FP32.
constexpr int kBatchWidth = 8;

// Persistent batched kernel + fix-up over `count` items whose tiles are
// numbered toff[j] .. toff[j+1]-1 (toff has count+1 entries, device).
// xs, ys: device arrays of count device pointers; head, tail: device
// arrays of total_tiles doubles.  cta_threads: 128, 256 or 512 threads
// per block; max_tile: the largest tile of any item.  Asynchronous on st.
msrep_status launch_batched(const BatchItem *items, const int64_t *toff, int count,
                            int64_t total_tiles, int32_t val_dtype, const void *const *xs,
                            void *const *ys, double *head, double *tail, double alpha,
                            double beta, unsigned flags, cudaStream_t st,
                            int cta_threads = 256, int max_tile = 1024);

// Batched k-vector form (FP32 values and vectors): item j carries
// 2 <= k_j <= 8 vectors, xin[j] = its k_j x vectors of n_j values each
// (device), xt[j] = device space for n_j * kBatchWidth values (filled here
// with the x interleaved by width spmm_width(k_j)), ys[j] = its k_j y
// vectors of m_j values.  Tiles numbered by toff as for launch_batched;
// uoff (count+1 entries, device) numbers the block work units, item j
// having batched_k_units(tiles_j, k_j) of them, total_units in all; head,
// tail: total_tiles * kBatchWidth doubles each.  y = A x for every vector
// (alpha 1, beta 0).  Asynchronous.
msrep_status launch_batched_k(const BatchItem *items, const int64_t *toff, const int64_t *uoff,
                              int count, int64_t total_tiles, int64_t total_units,
                              const void *const *xin, void *const *xt, void *const *ys,
                              double *head, double *tail, unsigned flags, cudaStream_t st);

// block work units of an item of `tiles` tiles and k vectors in the
// batched k-vector kernel
int64_t batched_k_units(int64_t tiles, int k);

}  // namespace msrep
