/*
 * msrep.h -- C ABI of the GB300 implementation of the msRep SpMV hot path
 * (arXiv 2209.07552, "msRep: A Fast yet Light Sparse Matrix Framework for
 * Multi-GPU Systems").
 *
 * The paper cuts the nonzeros of a CSR, CSC or COO matrix into np partitions
 * of equal nonzero count (pCSR/pCSC/pCOO, Sec. 3.2), runs an SpMV kernel per
 * partition and merges the partial sums of rows that a partition boundary
 * splits (Alg. 3, 5, 7; Sec. 4.3).  Here the partitions map to thread blocks
 * of one GPU instead of to GPUs.
 *
 * Conventions shared by every entry point:
 *  - Pointers named "device" must be CUDA device (or managed) memory; the
 *    library never copies them to the host.  Every buffer is BORROWED: the
 *    caller owns it and keeps it alive until the work queued on `stream` has
 *    finished.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls are asynchronous unless their comment says "syncs".
 *  - Index and pointer arrays are int32 (nnz < 2^31); partition arithmetic
 *    (i * nnz) is done in 64-bit integers.
 *  - No entry point allocates device memory, except msrep_serve_* (the server
 *    owns the memory of the matrices it holds, counted against its budget).
 *  - On error a call returns a non-zero msrep_status, queues nothing further
 *    and records a message readable by msrep_last_error() (per host thread).
 *  - y = alpha*A*x + beta*y (Alg. 1).  beta == 0 means y is write-only (its
 *    old contents may be NaN).
 */
#ifndef MSREP_H
#define MSREP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSREP_OK = 0,
  MSREP_ERR_INVALID_ARG = 1, /* a NULL pointer, bad size or bad enum value */
  MSREP_ERR_BAD_MATRIX = 2,  /* structural check failed (MSREP_VALIDATE)   */
  MSREP_ERR_OOM = 3,         /* server-side allocation failed              */
  MSREP_ERR_CUDA = 4,        /* a CUDA runtime call failed                 */
  MSREP_ERR_TIMEOUT = 5,     /* a bounded wait expired                     */
  MSREP_ERR_BUDGET = 6,      /* the server's memory budget is exhausted    */
  MSREP_ERR_NOT_FOUND = 7,   /* unknown matrix or request id               */
  MSREP_ERR_SHUTDOWN = 8,    /* the server is shutting down                */
  MSREP_ERR_WORKSPACE = 9    /* workspace or plan buffer too small         */
} msrep_status;

/* MSREP_COO is sorted by (row, col), the order Sec. 3.2.3 assumes.  The
 * two other COO orders are the ones Sec. 3.2.3 names and sets aside:
 * MSREP_COO_BY_COL sorted by (col, row), MSREP_COO_UNSORTED in no order
 * (duplicate coordinates allowed; their products add up). */
typedef enum {
  MSREP_CSR = 0,
  MSREP_CSC = 1,
  MSREP_COO = 2,
  MSREP_COO_BY_COL = 3,
  MSREP_COO_UNSORTED = 4
} msrep_format;

/* Value / vector storage types.  MSREP_BF16 is bfloat16 (8-bit exponent,
 * 7-bit mantissa) stored as uint16. */
typedef enum { MSREP_F64 = 0, MSREP_F32 = 1, MSREP_BF16 = 2 } msrep_dtype;

/* A sparse matrix in one of the three formats of Sec. 2.1.  All arrays are
 * device memory, borrowed.
 *   CSR (Sec. 2.1.2): ptr = row_ptr[m+1], idx = col_idx[nnz], idx2 = NULL.
 *   CSC (Sec. 2.1.3): ptr = col_ptr[n+1], idx = row_idx[nnz], idx2 = NULL;
 *                     row indices ascend within each column.
 *   COO (Sec. 2.1.1): ptr = NULL, idx = col_idx[nnz], idx2 = row_idx[nnz],
 *                     sorted by (row, col) as Sec. 3.2.3 assumes; the same
 *                     arrays for MSREP_COO_BY_COL and MSREP_COO_UNSORTED.
 * val has nnz entries of type val_dtype. */
typedef struct {
  int32_t fmt;       /* msrep_format */
  int32_t val_dtype; /* msrep_dtype */
  int32_t m, n;      /* rows, columns */
  int64_t nnz;
  const int32_t *ptr;
  const int32_t *idx;
  const int32_t *idx2;
  const void *val;
} msrep_matrix;

/* pCSR / pCSC / pCOO metadata (Sec. 3.2) plus the library's tile plan.
 * Every array is caller-allocated device memory of the stated length.
 *   start_idx, end_idx  [np]  nonzero range of partition i, end inclusive:
 *                             floor(i*nnz/np) .. floor((i+1)*nnz/np)-1.
 *   start_major,        [np]  first / last row (CSR, COO) or column (CSC,
 *   end_major                 COO_BY_COL) that owns a nonzero of the
 *                             partition; 0 and m-1 for COO_UNSORTED, whose
 *                             partitions may reach any row.
 *   start_flag          [np]  1 if the partition's first row (column) also
 *                             has nonzeros in an earlier partition; 0 for
 *                             COO_UNSORTED.
 *   local_off  (opt.) [np+1]  offsets of each partition's local pointers.
 *   local      (opt.)         CSR/CSC: local row_ptr/col_ptr of partition i
 *                             at local_off[i], end_major-start_major+2
 *                             entries (0, ptr[start+1]-start_idx, ...,
 *                             end_idx-start_idx+1); capacity
 *                             msrep_partition_local_bound().  COO: local row
 *                             index array, nnz entries, row_idx[k] -
 *                             start_major of k's partition (COO_BY_COL: the
 *                             local column index col_idx[k] - start_major;
 *                             COO_UNSORTED: row_idx[k] itself).
 *   plan       (opt.)         opaque plan used by msrep_spmv for CSR, CSC
 *                             (tiles, hub and frequent rows), COO_BY_COL
 *                             and COO_UNSORTED (hub and frequent rows);
 *                             plan_bytes >= msrep_plan_size().
 *   tile                      nonzeros+rows per warp tile of the plan,
 *                             0 = the format's default (256 for CSC, 512
 *                             for the others); must be a supported size
 *                             (msrep_tile_supported()).
 * An empty partition (np > nnz) has start_major = 0, end_major = -1,
 * start_flag = 0 and a one-entry local pointer {0}. */
typedef struct {
  int32_t np;
  int32_t tile;
  int32_t *start_idx;
  int32_t *end_idx;
  int32_t *start_major;
  int32_t *end_major;
  uint8_t *start_flag;
  int64_t *local_off;
  int32_t *local;
  void *plan;
  int64_t plan_bytes;
} msrep_partition;

/* flags for msrep_partition_* */
#define MSREP_VALIDATE 0x1u /* check structure on the device first; syncs */
#define MSREP_PART_MERGE_PATH 0x2u /* CSR/CSC: row+nonzero merge-path cuts
                                      instead of Alg. 2's nonzero cuts (see
                                      msrep_partition_csr) */
#define MSREP_PART_ROW_BLOCK 0x4u  /* the Baseline of Sec. 5.1: equal blocks
                                      of rows (CSR, COO; columns for CSC and
                                      COO_BY_COL) whatever their nonzeros;
                                      partition i holds rows floor(i*m/np) ..
                                      floor((i+1)*m/np)-1 and the metadata of
                                      their nonzero range (start_flag 0; R4 of
                                      the empty case for blocks of empty rows).
                                      A comparison partitioning for the
                                      imbalance Sec. 2.3 describes.  Not with
                                      MSREP_PART_MERGE_PATH or COO_UNSORTED. */

/* Library version string. */
const char *msrep_version(void);

/* Message of the last failed call on this host thread ("" if none). */
const char *msrep_last_error(void);

/* Host only, no GPU work.  Capacity that `local` needs for a CSR/CSC
 * partition with np parts: n_major + 2*np entries (Alg. 2 loop bound plus
 * the two closing entries per partition); nnz entries for the COO forms. */
msrep_status msrep_partition_local_bound(const msrep_matrix *A, int32_t np,
                                         int64_t *entries);

/* Host only.  1 if `tile` is a tile size msrep_spmv supports, else 0. */
int msrep_tile_supported(int32_t tile);

/* Host only.  Bytes of the plan for (A, np, tile); tile 0 = default.  0 for
 * row-sorted COO, which needs none. */
msrep_status msrep_plan_size(const msrep_matrix *A, int32_t np, int32_t tile,
                             int64_t *bytes);

/* CSR -> pCSR, Alg. 2 (Sec. 3.2.1).  Fills the metadata arrays, and the
 * local row pointers / tile plan when those pointers are non-NULL.  All
 * results are integers and exactly reproducible.  The binary search of
 * Alg. 2 owns nonzero k by row(k) = max{r < m : row_ptr[r] <= k}.
 * With MSREP_PART_MERGE_PATH the cuts follow the merged sequence of the m
 * row ends and the nnz nonzeros (the split of merge-based CSR SpMV, which
 * the paper cites among the single-GPU kernels it builds on; a row's end
 * comes after its nonzeros): cut i is at item floor(i*(m+nnz)/np), so every
 * partition holds the same number of rows plus nonzeros, and partition i
 * takes the nonzeros between cuts i and i+1 (possibly none, when it covers
 * only empty rows), with the metadata above for that range.
 * Errors: INVALID_ARG (np < 1, NULL array, wrong format), WORKSPACE (plan
 * too small), BAD_MATRIX (with MSREP_VALIDATE: row_ptr not monotone,
 * row_ptr[0] != 0, row_ptr[m] != nnz, column out of range). */
msrep_status msrep_partition_csr(const msrep_matrix *A, msrep_partition *part,
                                 unsigned flags, void *stream);

/* CSC -> pCSC, Alg. 4 (Sec. 3.2.2): Alg. 2 over col_ptr.  With a plan, it
 * also records up to four hub rows (rows holding about 0.1% or more of the
 * nonzeros, found from 4096 evenly spaced samples of row_idx) and, when
 * there are hub rows, a table of up to 2048 frequent rows (counted from
 * 65536 evenly spaced samples; a row claims a slot of a direct-mapped
 * table, and the most frequent claimant keeps it).  msrep_spmv sums the
 * products of those rows per thread block in shared memory and adds each
 * sum once, instead of one atomic add per nonzero.  The result is the same
 * up to the order of FP64 additions, which CSC's atomic scatter leaves
 * open anyway.  The plan (msrep_plan_size) also holds the 1 MB scratch of
 * that search. */
msrep_status msrep_partition_csc(const msrep_matrix *A, msrep_partition *part,
                                 unsigned flags, void *stream);

/* COO -> pCOO, Alg. 6 (Sec. 3.2.3), for the three COO orders.
 *   MSREP_COO (row-sorted): Alg. 6 searches a row_ptr that COO does not
 *     carry; here start_major = row_idx[start_idx], end_major =
 *     row_idx[end_idx], start_flag = row_idx[start_idx-1] ==
 *     row_idx[start_idx].  The result equals msrep_partition_csr on the CSR
 *     of the same matrix.
 *   MSREP_COO_BY_COL: the same over col_idx (Sec. 3.2.3's column-sorted
 *     case); equals msrep_partition_csc on the CSC of the same matrix.
 *   MSREP_COO_UNSORTED: the nonzero ranges only; start_major = 0,
 *     end_major = m-1 (Sec. 3.2.3: a partition of unsorted COO may reach
 *     any row), start_flag = 0.
 * For COO_BY_COL and COO_UNSORTED a plan (msrep_plan_size bytes) receives
 * the hub rows and the frequent-row table, found as for
 * msrep_partition_csc.  Validation checks the
 * indices' range and, for the two sorted orders, the order.
 * MSREP_PART_MERGE_PATH is INVALID_ARG here. */
msrep_status msrep_partition_coo(const msrep_matrix *A, msrep_partition *part,
                                 unsigned flags, void *stream);

/* Host only.  Device workspace bytes msrep_spmv needs for (A, part): two
 * FP64 partials per tile, and for CSC, COO_BY_COL and COO_UNSORTED an FP64
 * accumulator of 2^k >= m entries (the permuted accumulator of matrices
 * with hub rows, see msrep_partition_csc; the low-precision path also
 * accumulates there). */
msrep_status msrep_spmv_workspace_size(const msrep_matrix *A,
                                       const msrep_partition *part,
                                       size_t *bytes);

/* flags for msrep_spmv */
#define MSREP_COMP_ALL 0x10u  /* low precision: compensate every row      */
#define MSREP_COMP_NONE 0x20u /* low precision: plain FP32 accumulation   */
#define MSREP_STREAM_TMA 0x40u /* stage the nonzeros through shared memory
                                  with bulk copies (TMA) instead of direct
                                  256-bit loads; tiles up to 512         */
#define MSREP_SCHED_PER_PARTITION 0x80u /* CSR, CSC, row-sorted COO: one
                                  thread block per partition, which walks
                                  that partition's tiles alone (as the paper
                                  gives each partition one GPU), instead of
                                  spreading every partition's tiles over all
                                  blocks; the kernel then lasts as long as
                                  its largest partition.  Same results.
                                  Not with MSREP_STREAM_TMA. */

/* y = alpha*A*x + beta*y over the partitions of `part` (Alg. 3 for CSR,
 * Alg. 5 for CSC, Alg. 7 for COO).  `part` must come from the matching
 * msrep_partition_* call on the same matrix; CSR, CSC, COO_BY_COL and
 * COO_UNSORTED also need its plan.  COO_BY_COL and COO_UNSORTED scatter
 * like CSC: every partition may add to any row, so each product is an
 * FP64 atomic add into y (or the accumulator), which is the sum of the
 * partitions' full partial vectors; the result does not depend on where
 * the partition boundaries fall, and the kernel spreads the nonzeros over
 * its warps in equal runs.
 *
 * Types: val_dtype F64 with xy_dtype F64 (the plain path), or val_dtype F32
 * or BF16 with xy_dtype F32 (the low-precision form: FP32 products, FP32
 * accumulation with TwoSum compensation on rows longer than 256 nonzeros
 * and on rows split between thread-block tiles, partial sums of split rows
 * merged in FP64).  x has n entries, y has m entries, device memory.
 *
 * Merge: every row split by a partition (or tile) boundary gets
 * alpha * (sum of its partials, in partition order) + beta * y_in, beta
 * applied once (Sec. 3.2.1, Sec. 4.3).  CSR and COO merge without atomics;
 * CSC scatters with atomic adds (the column merge of Alg. 5), so its
 * rounding order varies from run to run; when the plan found hub rows it
 * scatters into a permuted accumulator in the workspace (which spreads the
 * hub rows' cache lines over all L2 slices) and gathers y from it after.
 * `workspace` must hold msrep_spmv_workspace_size() bytes, 16-byte
 * aligned.  idx, idx2 and val must be 32-byte aligned and ptr 16-byte
 * aligned (the kernels bulk-copy them in aligned segments and read groups
 * of 8 elements).  Errors: INVALID_ARG, WORKSPACE, CUDA. */
msrep_status msrep_spmv(const msrep_matrix *A, const msrep_partition *part,
                        double alpha, const void *x, double beta, void *y,
                        int32_t xy_dtype, unsigned flags, void *workspace,
                        void *stream);

/* ---------------------------------------------------------------------- */
/* k right-hand sides (no counterpart in the paper, which multiplies one  */
/* vector; the served form's requests carry up to eight).                 */
/* ---------------------------------------------------------------------- */

/* Vectors msrep_spmm multiplies in one pass over A (more take several). */
#define MSREP_SPMM_MAX_K 8

/* Host only.  Workspace bytes of msrep_spmm for (A, part, k): two FP64
 * partials per tile and vector, and the interleaved copy of X (n rows of
 * min(k, 8) rounded up to 1, 2, 4 or 8 values).  CSR only. */
msrep_status msrep_spmm_workspace_size(const msrep_matrix *A, const msrep_partition *part,
                                       int32_t k, size_t *bytes);

/* Y = alpha*A*X + beta*Y for k >= 1 vectors, A in CSR over the
 * tiles of `part` (from msrep_partition_csr, with its plan).  X holds the k
 * x vectors one after another (x_v = X + v*ldx, n values each, ldx >= n);
 * Y the k y vectors (y_v = Y + v*ldy, ldy >= m); device memory, types as
 * for msrep_spmv.  The vectors are taken in passes of up to
 * MSREP_SPMM_MAX_K (8): each pass first copies its vectors into the
 * workspace with their values of each row side by side, so that each
 * nonzero gathers one segment for all of them and A is read once per pass
 * (ceil(k / 8) times in all).  Every column of Y is computed exactly as
 * msrep_spmv computes y for that x (same order of operations,
 * bit-identical results).  `flags`: MSREP_COMP_ALL / MSREP_COMP_NONE as
 * for msrep_spmv.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (format not CSR, k < 1, ldx < n, ldy < m,
 * types, alignment as for msrep_spmv), WORKSPACE (no plan, NULL
 * workspace), CUDA. */
msrep_status msrep_spmm(const msrep_matrix *A, const msrep_partition *part, int32_t k,
                        double alpha, const void *x, int64_t ldx, double beta, void *y,
                        int64_t ldy, int32_t xy_dtype, unsigned flags, void *workspace,
                        void *stream);

/* ---------------------------------------------------------------------- */
/* Batched form: many independent CSR matrices in one persistent launch.  */
/* No counterpart in the paper beyond its partitions (Sec. 3.2); the      */
/* per-matrix work is Alg. 3 exactly as msrep_spmv runs it.               */
/* ---------------------------------------------------------------------- */

/* Tuning table: a matrix falls in bucket floor(log2(max(nnz, 1))); bucket
 * b uses warp tile tile[b] (0 = default) and np = ceil(nnz / part_nnz[b])
 * partitions (part_nnz[b] = 0: one partition).  One launch runs every
 * matrix of a batch, so the thread-block shape is one per batch:
 * cta_threads threads per block (128, 256 or 512; 0 = 256). */
#define MSREP_TUNE_BUCKETS 32
typedef struct {
  int32_t tile[MSREP_TUNE_BUCKETS];
  int64_t part_nnz[MSREP_TUNE_BUCKETS];
  int32_t cta_threads;
  int32_t reserved;
} msrep_tune_table;

/* A prepared batch (filled by msrep_batch_prepare; host memory, owned by
 * the caller).  `dev` is the caller's device buffer that holds every
 * matrix's partition and tile plan plus the batch's tile directory. */
typedef struct {
  int32_t count;       /* number of matrices                       */
  int32_t val_dtype;   /* common value type of the batch           */
  int64_t total_tiles; /* tiles over all matrices                  */
  int64_t ws_bytes;    /* workspace msrep_spmv_batched needs       */
  void *dev;
  int64_t dev_bytes;
  int64_t items_off;   /* byte offsets of the directory in dev     */
  int64_t toff_off;
  int32_t cta_threads; /* threads per block of the launch          */
  int32_t max_tile;    /* largest warp tile of the batch           */
} msrep_batch;

/* Host only: the library's default table (default tile, one partition). */
msrep_status msrep_tune_default(msrep_tune_table *tune);

/* Host only: device bytes msrep_batch_prepare needs for As[0..count). */
msrep_status msrep_batch_plan_size(int32_t count, const msrep_matrix *As,
                                   const msrep_tune_table *tune,
                                   int64_t *dev_bytes);

/* Partitions every matrix (Alg. 2, np and tile from `tune`, NULL = the
 * default table), builds its tile plan and the batch's tile directory in
 * `dev`, and fills *out.  As is a host array of CSR matrices (device
 * arrays) sharing one val_dtype.  Syncs `stream`. */
msrep_status msrep_batch_prepare(int32_t count, const msrep_matrix *As,
                                 const msrep_tune_table *tune, void *dev,
                                 int64_t dev_bytes, msrep_batch *out,
                                 void *stream);

/* y_j = alpha*A_j*x_j + beta*y_j for every matrix of the batch, as one
 * persistent kernel over all tiles plus one fix-up kernel (no host work,
 * no allocation: safe to capture in a CUDA graph).  xs, ys: DEVICE arrays
 * of `count` device pointers (F64 x/y for an F64 batch, else F32).  Each
 * y_j equals bit for bit what msrep_spmv gives for A_j with the same np
 * and tile.  workspace: B->ws_bytes, 16-byte aligned. */
msrep_status msrep_spmv_batched(const msrep_batch *B, const void *const *xs,
                                void *const *ys, double alpha, double beta,
                                unsigned flags, void *workspace, void *stream);

/* Host only: scratch bytes msrep_autotune needs for As. */
msrep_status msrep_autotune_scratch_size(int32_t count, const msrep_matrix *As,
                                         int64_t *bytes);

/* Project-written autotuner.  First, for every size bucket present in As,
 * it times msrep_spmv on up to three of the bucket's largest matrices for
 * each candidate (tile 256/512/1024 x part_nnz 0/2^14/2^18) with CUDA
 * events and keeps the fastest; absent buckets keep the default.  Then it
 * prepares the whole batch with that table in the scratch and times
 * msrep_spmv_batched with 128, 256 and 512 threads per block, keeping the
 * fastest as cta_threads.  xs/ys: HOST arrays of device pointers (ys are
 * overwritten).  Syncs `stream`. */
msrep_status msrep_autotune(int32_t count, const msrep_matrix *As,
                            const void *const *xs, void *const *ys,
                            void *scratch, int64_t scratch_bytes,
                            msrep_tune_table *out, void *stream);

/* ---------------------------------------------------------------------- */
/* Serving: a request loop over device-resident matrices with continuous */
/* batching.  No counterpart in the paper.                                */
/* ---------------------------------------------------------------------- */

/* A request with one x vector runs as an item of the batched SpMV kernel;
 * a request with 2..8 vectors as one item of the batched k-vector kernel
 * (see msrep_spmm), which reads the matrix once for all its vectors.  Each
 * launch context holds: x and y arenas (arena_bytes each), an interleaved-x
 * arena (4 * arena_bytes), two directories (max_items entries) and tile
 * partials for both kernels (max_tiles and 8 * max_tiles doubles, twice);
 * all of it counts against the budget. */
typedef struct {
  int64_t budget_bytes;   /* device memory the server may hold in total  */
  int64_t arena_bytes;    /* per in-flight launch: x and y staging (each) */
  int32_t contexts;       /* launches in flight at once (>= 1)           */
  int32_t max_items;      /* requests per launch, for each kernel        */
  int32_t max_k;          /* vectors per request (<= 8)                  */
  int32_t tile;           /* tile of every registered matrix (0 = def.)  */
  int64_t max_tiles;      /* tiles per launch, for each kernel           */
  int32_t device;         /* CUDA device ordinal                         */
} msrep_serve_config;

typedef struct msrep_server msrep_server; /* opaque */

typedef struct {
  uint64_t submitted, completed, rejected, launches;
  double p50_us, p99_us, mean_us, max_us; /* submit -> y on the host      */
  double gbs;             /* algorithmic bytes of completed work / busy s */
  double mean_items;      /* vectors per launch                           */
  double busy_s;          /* wall time with at least one launch in flight */
  int64_t resident_bytes; /* device bytes held (matrices + arenas)        */
  /* where the latency goes: */
  double wait_p50_us, wait_p99_us;     /* submit -> packed into a launch  */
  double device_p50_us, device_p99_us; /* one launch on the device, from
                                          its first x copy to its last y
                                          copy (CUDA events)              */
  double kernel_mean_us;  /* the batched kernels of one launch (events)   */
  double host_launch_p50_us, host_launch_p99_us; /* the scheduler thread
                                          issuing one launch's copies and
                                          kernels (host clock)            */
} msrep_serve_counters;

/* Defaults: 60 GB budget, 64 MB arenas, 3 contexts, 256 items, k <= 8. */
msrep_status msrep_serve_config_default(msrep_serve_config *cfg);

/* Starts a server (allocates its arenas and two host threads).  Errors:
 * INVALID_ARG, BUDGET (arenas alone exceed the budget), OOM, CUDA. */
msrep_status msrep_serve_create(const msrep_serve_config *cfg, msrep_server **out);

/* Copies a CSR matrix whose arrays are in HOST memory to the device (values
 * stored as FP32; F64 values are rounded), partitions it (Alg. 2, one
 * partition per 2^20 nonzeros) and builds its tile plan.  Syncs.  Errors:
 * BUDGET when it does not fit in what the budget leaves, OOM, INVALID_ARG. */
msrep_status msrep_serve_register(msrep_server *s, const msrep_matrix *host_csr,
                                  int64_t *matrix_id);

/* Removes a matrix once no queued or running request names it; its device
 * memory returns to the budget.  NOT_FOUND for an unknown id. */
msrep_status msrep_serve_unregister(msrep_server *s, int64_t matrix_id);

/* Queues y_v = A x_v for v = 0..k-1 (x_host: k vectors of n floats, one
 * after the other; y_host: k vectors of m floats); both host buffers stay
 * owned by the caller and must live until the request completes.  Page-
 * locked buffers (cudaMallocHost / cudaHostRegister) mapped at their own
 * address (unified addressing) are read and written by the launch's kernels
 * directly; other page-locked buffers are transferred by DMA, pageable ones
 * through the server's staging buffers.  Does not block.  The request joins a launch as soon as a context and arena space
 * are free (continuous batching).  Errors: NOT_FOUND, INVALID_ARG (k out
 * of range), SHUTDOWN. */
msrep_status msrep_serve_submit(msrep_server *s, int64_t matrix_id, int32_t k,
                                const float *x_host, float *y_host, uint64_t *req_id);

/* Waits up to timeout_us (< 0: no limit) for the request; MSREP_OK when y
 * is in place, TIMEOUT otherwise (the request stays queued or running),
 * NOT_FOUND for an unknown or already collected id. */
msrep_status msrep_serve_wait(msrep_server *s, uint64_t req_id, int64_t timeout_us);

/* Counters and latency percentiles of completed requests since creation
 * or the last reset (reset != 0 clears them after reading). */
msrep_status msrep_serve_stats(msrep_server *s, msrep_serve_counters *out, int32_t reset);

/* Load driver for measuring the server (no counterpart in the paper): from
 * the calling thread, submits `count` requests at the given arrival times
 * (t_us[i] microseconds after the call starts, non-decreasing; the thread
 * spins until then), request i naming matrix_id[i] with k[i] vectors read
 * from x[i] and written to y[i] (host buffers as for msrep_serve_submit),
 * then waits for every request.  Before submitting request i it waits for
 * request reuse[i] (< i; -1 = none), the last one that used the same y
 * buffer, which lets a caller recycle buffers without a thread of its own.
 * With reset_after_us >= 0 the server's statistics are reset once the
 * stream passes that time (to drop a warm-up).  *late counts the requests
 * submitted more than 100 us after their arrival time, *max_lag_us is the
 * largest such delay.  The latency statistics are msrep_serve_stats'.
 * Syncs.  Errors: INVALID_ARG, and those of submit and wait. */
msrep_status msrep_serve_replay(msrep_server *s, int64_t count, const double *t_us,
                                const int64_t *matrix_id, const int32_t *k,
                                const float *const *x, float *const *y, const int64_t *reuse,
                                double reset_after_us, int64_t *late, double *max_lag_us);

/* Stops the threads after finishing queued work, frees everything. */
msrep_status msrep_serve_destroy(msrep_server *s);

/* ---------------------------------------------------------------------- */
/* SpMV without any allocation (the paper has no counterpart).            */
/* ---------------------------------------------------------------------- */

/* Bytes of the library's built-in scratch array: every GPU that loads the
 * library holds this much device memory until the process exits. */
#define MSREP_NOALLOC_SCRATCH_BYTES (1u << 20)

/* Same result as msrep_spmv, for callers that cannot allocate device
 * memory: code that only receives the matrix and vector buffers from a host
 * framework which owns all device memory, or a latency-critical loop where
 * a cudaMalloc is not acceptable.  Instead of a caller workspace it uses
 * one scratch array compiled into the library (MSREP_NOALLOC_SCRATCH_BYTES,
 * a static device array), so this call allocates nothing.
 *  - Every call made outside a stream capture looks up the array's device
 *    address with cudaGetSymbolAddress (for the current device), so a
 *    context destroyed and recreated in between (cudaDeviceReset) is
 *    handled.  A call inside a capture reuses the address of the device's
 *    last uncaptured call: make one call on each device before capturing.
 *  - The scratch must hold what msrep_spmv_workspace_size reports, minus
 *    the permuted accumulator when that does not fit (below); problems that
 *    need more are rejected with MSREP_ERR_WORKSPACE and nothing is queued.
 *    Two FP64 partials per tile: CSR about (m + nnz)/tile + np tiles, CSC
 *    (n + nnz)/tile + np, row-sorted COO np * ceil(ceil(nnz/np)/tile), so
 *    about 65,000 tiles in all (e.g. m + nnz up to about 32 million for CSR
 *    at the default tile of 512); CSC, COO_BY_COL and COO_UNSORTED with
 *    FP32/BF16 values also need m doubles for their FP64 accumulator.
 *  - A CSC or scatter-COO SpMV whose permuted accumulator (2^k >= m
 *    doubles) does not fit scatters into y (or into the row-ordered
 *    accumulator) directly: the same result up to the order of the FP64
 *    additions, slower on matrices with hub rows.
 *  - Every call shares the one array and leaves its contents behind: two
 *    calls whose work overlaps on the GPU (different streams, or several
 *    host threads) race on it and give wrong results; serialise them.
 *    Nothing in the array needs to start at zero: each call writes every
 *    value it later reads.
 * Arguments and errors as for msrep_spmv, minus the workspace. */
msrep_status msrep_spmv_noalloc(const msrep_matrix *A, const msrep_partition *part,
                                double alpha, const void *x, double beta, void *y,
                                int32_t xy_dtype, unsigned flags, void *stream);

/* Host; syncs `stream`.  Reads and clears the device error word that the
 * streaming kernels set when a bounded wait on one of their bulk copies
 * expires (which means the copy engine stalled or an argument was wrong).
 * *status = 0 and MSREP_OK when no kernel failed, else MSREP_ERR_TIMEOUT. */
msrep_status msrep_device_status(void *stream, int *status);

/* Self-test of the bounded device wait (no counterpart in the paper; the
 * failure-detection check of the streaming kernels' waits).  Launches one
 * kernel whose thread initialises an mbarrier expecting two arrivals,
 * arrives once and issues no copy, so the barrier can never complete; its
 * bounded wait gives up after max_cycles SM clock cycles (1 ..
 * 2,000,000,000, the limit the streaming kernels use), writes 1 to
 * *gave_up (a device int32; 0 if the wait had completed) and records the
 * timeout in the device error word, exactly as a stalled bulk copy would,
 * so that the next msrep_device_status reports MSREP_ERR_TIMEOUT.  Nothing
 * faults or hangs: the kernel returns either way.  Asynchronous on
 * `stream`.  Errors: INVALID_ARG, CUDA. */
msrep_status msrep_wait_selftest(int64_t max_cycles, int32_t *gave_up, void *stream);

/* Measurement aid (no counterpart in the paper): the access-pattern floor
 * of an SpMV.  One kernel that streams idx (and, modes 1 and 5, idx2) and
 * val once and, per nonzero, gathers vec[idx] (modes 0, 1: CSR, COO, eight
 * consecutive nonzeros a lane; modes 4, 5: the same, lane-interleaved, each
 * warp instruction covering 32 consecutive nonzeros) or atomically adds val
 * into vec[idx] (mode 2) or into vec[slot(idx)] (mode 3: the permuted
 * accumulator of msrep_spmv's CSC path, slot(r) = r * 0x9E3779B1 mod
 * vec_len), with no row logic.  Its time is what any SpMV kernel over
 * the same arrays pays for its gathers or scatters.  nnz elements; idx,
 * idx2, val 32-byte aligned device arrays; vec: vec_len doubles, vec_len a
 * power of two (every index is reduced modulo vec_len, so any idx is in
 * bounds); sink: one device double (written only to keep the gathers).
 * Asynchronous on `stream`.  Errors: INVALID_ARG. */
msrep_status msrep_access_floor(int32_t mode, const int32_t *idx, const int32_t *idx2,
                                const double *val, double *vec, int64_t nnz,
                                int64_t vec_len, double *sink, void *stream);

/* Profiling aid (no counterpart in the paper).  While set, every msrep_spmv
 * call made on this host thread records `start` (a cudaEvent_t passed as
 * void*) on its stream just before its main SpMV kernel and `stop` just
 * after it, so the caller can time that kernel alone with
 * cudaEventElapsedTime.  Pass NULL, NULL to stop recording. */
msrep_status msrep_profile_events(void *start, void *stop);

#ifdef __cplusplus
}
#endif

#endif /* MSREP_H */
