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
};

// Persistent batched kernel + fix-up over `count` items whose tiles are
// numbered toff[j] .. toff[j+1]-1 (toff has count+1 entries, device).
// xs, ys: device arrays of count device pointers; head, tail: device
// arrays of total_tiles doubles.  Asynchronous on st.
msrep_status launch_batched(const BatchItem *items, const int64_t *toff, int count,
                            int64_t total_tiles, int32_t val_dtype, const void *const *xs,
                            void *const *ys, double *head, double *tail, double alpha,
                            double beta, unsigned flags, cudaStream_t st);

}  // namespace msrep
