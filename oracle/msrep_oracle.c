/*
 * msrep_oracle.c -- the CPU oracle for the msRep SpMV hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check of the package entry
 * module and the CPU-baseline leg of the benchmark use it.  It shares no code,
 * header, table or helper with the CUDA library; it does not include
 * include/msrep.h.
 *
 * Plain, slow, single-threaded, FP64.  Each function names the passage of
 * arXiv 2209.07552 ("msRep: A Fast yet Light Sparse Matrix Framework for
 * Multi-GPU Systems") that it follows.  Readings of garbled or silent passages:
 *
 *   R1  Alg. 1 applies beta inside the nonzero loop and its inner bound looks
 *       inclusive.  Read: 0-based, half-open [row_ptr[i], row_ptr[i+1]), and
 *       y[i] = alpha * sum + beta * y[i] once per row.
 *   R2  Alg. 2/4/6 loop i = 1..np.  Read i = 0..np-1; end_idx is inclusive;
 *       i*nnz is formed in 64-bit integers.
 *   R3  BinarySearch(ptr, k) (Alg. 2/4) is read as row(k) = max{ r in [0,m) :
 *       ptr[r] <= k }, the row that owns nonzero k (empty rows are skipped).
 *       Here it is computed by a forward linear scan, never by bisection.
 *   R4  Empty partitions (end_idx < start_idx, possible when nnz < np):
 *       start_major = 0, end_major = -1, start_flag = 0.
 *   R5  Local pointers (Alg. 2/4 inner loop): lptr[0] = 0, lptr[j] =
 *       ptr[start+j] - start_idx for j = 1..end-start, and a closing entry
 *       lptr[end-start+1] = end_idx - start_idx + 1; length end-start+2.
 *       An empty partition has one entry, 0.
 *   R6  The merge of Alg. 3/7 is read from Sec. 3.2.1 and Sec. 4.3: every row
 *       split by a partition boundary receives alpha * (sum of the partials of
 *       all partitions that touch it, in partition order) + beta * y_in, with
 *       beta applied exactly once.
 *   R7  The last line of Alg. 5 is truncated; read y = alpha * sum_i py_i +
 *       beta * y_in.
 *   R8  Alg. 6 searches a row_ptr that COO does not have.  For COO sorted by
 *       (row, col): start_row = row_idx[start_idx], end_row =
 *       row_idx[end_idx], start_flag = start_idx > 0 &&
 *       row_idx[start_idx-1] == row_idx[start_idx].
 *   R10 Row+nonzero merge-path partitioning (the split of Merrill and
 *       Garland's merge-based CSR SpMV, which the paper cites among the
 *       single-GPU kernels it builds on): the m row ends and the nnz
 *       nonzeros form one merged sequence, the row end of row r placed after
 *       the row's nonzeros (an empty row's end before the next nonzero).
 *       Cut i is at item floor(i*(m+nnz)/np); partition i takes the nonzeros
 *       between cuts i and i+1, and its metadata follow Alg. 2 (R3, R4) for
 *       that nonzero range.  Optional variant: Alg. 2's pure nonzero split
 *       stays the default.
 *   R11 The Baseline partitioning of Sec. 5.1 (and the row-block split of
 *       Sec. 2.3) cuts the rows (CSR, COO) or columns (CSC) into np blocks
 *       of equal size without looking at the nonzeros: block i holds rows
 *       floor(i*n_major/np) .. floor((i+1)*n_major/np)-1 (64-bit product)
 *       and all of their nonzeros.  In the augmented metadata that is the
 *       nonzero range ptr[r_i] .. ptr[r_{i+1}]-1, with start/end major and
 *       flag as Alg. 2 gives them for that range (R3; a block starts at a
 *       row start, so its flag is 0) and R4 for a block whose rows are all
 *       empty.  For row-sorted COO the block's range is found by scanning
 *       the row index (Sec. 5.3 searches for each row block's start and
 *       end).  A comparison partitioning: its blocks carry as many
 *       nonzeros as their rows happen to hold.
 *   R9  COO sorted by (col, row) (Sec. 3.2.3 names it, with cost
 *       O(np log n)): Alg. 6 with the column index as the major index, so
 *       start_major/end_major are columns and the flag marks a split
 *       column.  COO in no order (Sec. 3.2.3: a partition may reach any
 *       row): start_major = 0, end_major = m-1 for a non-empty partition,
 *       start_flag = 0.  In both, each partition produces a full m-vector
 *       of partials and the merge sums them in partition order (as R7).
 *
 * Build: plain C11, -ffp-contract=off so every product and sum rounds alone.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Partitioning: Alg. 2 (pCSR), Alg. 4 (pCSC), Alg. 6 (pCOO).                */
/* ------------------------------------------------------------------------ */

/* Nonzero range of partition i: Alg. 2, first two statements, reading R2. */
static void part_range(int64_t nnz, int32_t np, int32_t i, int64_t *s,
                       int64_t *e) {
  *s = ((int64_t)i * nnz) / np;
  *e = ((int64_t)(i + 1) * nnz) / np - 1;
}

/* row(k) of reading R3 by a forward linear scan starting from row `from`
 * (the caller passes a row known to be <= the answer).  ptr has n_major+1
 * entries and ptr[n_major] == nnz > k. */
static int32_t owner_scan(const int32_t *ptr, int32_t n_major, int64_t k,
                          int32_t from) {
  int32_t r = from;
  while (r + 1 < n_major && (int64_t)ptr[r + 1] <= k) r++;
  return r;
}

/* Alg. 2 / Alg. 4 over a compressed pointer array (row_ptr for CSR, col_ptr
 * for CSC; CSC(A) is CSR(A^T), Sec. 2.1.3).  Arrays are length np. */
int ref_partition_compressed(int32_t n_major, int64_t nnz, const int32_t *ptr,
                             int32_t np, int32_t *start_idx, int32_t *end_idx,
                             int32_t *start_major, int32_t *end_major,
                             uint8_t *start_flag) {
  if (np < 1 || n_major < 0 || nnz < 0) return 1;
  int32_t hint = 0;
  for (int32_t i = 0; i < np; i++) {
    int64_t s, e;
    part_range(nnz, np, i, &s, &e);
    start_idx[i] = (int32_t)s;
    end_idx[i] = (int32_t)e;
    if (e < s) { /* reading R4 */
      start_major[i] = 0;
      end_major[i] = -1;
      start_flag[i] = 0;
      continue;
    }
    int32_t sr = owner_scan(ptr, n_major, s, hint);
    int32_t er = owner_scan(ptr, n_major, e, sr);
    hint = sr;
    start_major[i] = sr;
    end_major[i] = er;
    /* Alg. 2: the first row is partial when the partition starts after the
     * row's first nonzero (Sec. 3.2.1). */
    start_flag[i] = (s > (int64_t)ptr[sr]) ? 1 : 0;
  }
  return 0;
}

/* Merge-path partitioning, reading R10.  The cuts are found by walking the
 * merged sequence one item at a time from the start: at (r row ends,
 * k nonzeros) the next item is row r's end when all of row r's nonzeros
 * are behind (ptr[r+1] <= k), else nonzero k.  cut_row (np+1 entries, or
 * NULL) receives the row coordinate of every cut. */
int ref_partition_merge_path(int32_t n_major, int64_t nnz, const int32_t *ptr,
                             int32_t np, int32_t *start_idx, int32_t *end_idx,
                             int32_t *start_major, int32_t *end_major,
                             uint8_t *start_flag, int32_t *cut_row) {
  if (np < 1 || n_major < 0 || nnz < 0) return 1;
  const int64_t total = (int64_t)n_major + nnz;
  int64_t *cut_k = (int64_t *)malloc(sizeof(int64_t) * ((size_t)np + 1));
  if (!cut_k) return 2;
  int32_t r = 0;
  int64_t k = 0, d = 0;
  for (int32_t i = 0; i <= np; i++) {
    const int64_t di = ((int64_t)i * total) / np;
    while (d < di) {
      if (r < n_major && (int64_t)ptr[r + 1] <= k)
        r++;
      else
        k++;
      d++;
    }
    cut_k[i] = k;
    if (cut_row) cut_row[i] = r;
  }
  int32_t hint = 0;
  for (int32_t i = 0; i < np; i++) {
    const int64_t s = cut_k[i], e = cut_k[i + 1] - 1;
    start_idx[i] = (int32_t)s;
    end_idx[i] = (int32_t)e;
    if (e < s) { /* reading R4 */
      start_major[i] = 0;
      end_major[i] = -1;
      start_flag[i] = 0;
      continue;
    }
    int32_t sr = owner_scan(ptr, n_major, s, hint);
    int32_t er = owner_scan(ptr, n_major, e, sr);
    hint = sr;
    start_major[i] = sr;
    end_major[i] = er;
    start_flag[i] = (s > (int64_t)ptr[sr]) ? 1 : 0;
  }
  free(cut_k);
  return 0;
}

/* Baseline row-block (column-block) partitioning of a compressed pointer
 * array, reading R11. */
int ref_partition_row_block(int32_t n_major, int64_t nnz, const int32_t *ptr,
                            int32_t np, int32_t *start_idx, int32_t *end_idx,
                            int32_t *start_major, int32_t *end_major,
                            uint8_t *start_flag) {
  if (np < 1 || n_major < 0 || nnz < 0) return 1;
  int32_t hint = 0;
  for (int32_t i = 0; i < np; i++) {
    const int32_t r0 = (int32_t)(((int64_t)i * n_major) / np);
    const int32_t r1 = (int32_t)(((int64_t)(i + 1) * n_major) / np);
    const int64_t s = ptr[r0], e = (int64_t)ptr[r1] - 1;
    start_idx[i] = (int32_t)s;
    end_idx[i] = (int32_t)e;
    if (e < s) { /* reading R4 */
      start_major[i] = 0;
      end_major[i] = -1;
      start_flag[i] = 0;
      continue;
    }
    int32_t sr = owner_scan(ptr, n_major, s, hint);
    int32_t er = owner_scan(ptr, n_major, e, sr);
    hint = sr;
    start_major[i] = sr;
    end_major[i] = er;
    start_flag[i] = (s > (int64_t)ptr[sr]) ? 1 : 0;
  }
  return 0;
}

/* Baseline row-block partitioning of row-sorted COO, reading R11: the rows
 * of block i are found by scanning row_idx forward. */
int ref_partition_coo_row_block(int64_t nnz, const int32_t *row_idx, int32_t m,
                                int32_t np, int32_t *start_idx, int32_t *end_idx,
                                int32_t *start_row, int32_t *end_row,
                                uint8_t *start_flag) {
  if (np < 1 || nnz < 0 || m < 0) return 1;
  int64_t k = 0;
  for (int32_t i = 0; i < np; i++) {
    const int32_t r0 = (int32_t)(((int64_t)i * m) / np);
    const int32_t r1 = (int32_t)(((int64_t)(i + 1) * m) / np);
    while (k < nnz && row_idx[k] < r0) k++;
    const int64_t s = k;
    int64_t t = s;
    while (t < nnz && row_idx[t] < r1) t++;
    const int64_t e = t - 1;
    start_idx[i] = (int32_t)s;
    end_idx[i] = (int32_t)e;
    if (e < s) {
      start_row[i] = 0;
      end_row[i] = -1;
      start_flag[i] = 0;
      continue;
    }
    start_row[i] = row_idx[s];
    end_row[i] = row_idx[e];
    start_flag[i] = (s > 0 && row_idx[s - 1] == row_idx[s]) ? 1 : 0;
  }
  return 0;
}

/* Number of local-pointer entries of one partition under reading R5. */
static int64_t local_len(int32_t sm, int32_t em) { return (int64_t)em - sm + 2; }

/* Total local-pointer length over all partitions, and per-partition offsets
 * (off has np+1 entries). */
int64_t ref_local_offsets(int32_t np, const int32_t *start_major,
                          const int32_t *end_major, int64_t *off) {
  int64_t acc = 0;
  for (int32_t i = 0; i < np; i++) {
    off[i] = acc;
    acc += local_len(start_major[i], end_major[i]);
  }
  off[np] = acc;
  return acc;
}

/* Local row_ptr / col_ptr of every partition (Alg. 2/4 inner loop,
 * reading R5), concatenated at the offsets of ref_local_offsets. */
int ref_partition_local_compressed(const int32_t *ptr, int32_t np,
                                   const int32_t *start_idx,
                                   const int32_t *end_idx,
                                   const int32_t *start_major,
                                   const int32_t *end_major,
                                   const int64_t *off, int32_t *local) {
  for (int32_t i = 0; i < np; i++) {
    int32_t *l = local + off[i];
    int32_t span = end_major[i] - start_major[i]; /* -1 when empty */
    l[0] = 0;
    for (int32_t j = 1; j <= span; j++)
      l[j] = ptr[start_major[i] + j] - start_idx[i];
    if (span >= 0) l[span + 1] = end_idx[i] - start_idx[i] + 1;
  }
  return 0;
}

/* Alg. 6 under reading R8: COO sorted by (row, col). */
int ref_partition_coo(int64_t nnz, const int32_t *row_idx, int32_t np,
                      int32_t *start_idx, int32_t *end_idx, int32_t *start_row,
                      int32_t *end_row, uint8_t *start_flag) {
  if (np < 1 || nnz < 0) return 1;
  for (int32_t i = 0; i < np; i++) {
    int64_t s, e;
    part_range(nnz, np, i, &s, &e);
    start_idx[i] = (int32_t)s;
    end_idx[i] = (int32_t)e;
    if (e < s) {
      start_row[i] = 0;
      end_row[i] = -1;
      start_flag[i] = 0;
      continue;
    }
    start_row[i] = row_idx[s];
    end_row[i] = row_idx[e];
    start_flag[i] = (s > 0 && row_idx[s - 1] == row_idx[s]) ? 1 : 0;
  }
  return 0;
}

/* pCOO of a COO matrix in no particular order, reading R9: the nonzero
 * ranges of Alg. 6; the row range of every non-empty partition is the
 * whole matrix. */
int ref_partition_coo_unsorted(int64_t nnz, int32_t m, int32_t np,
                               int32_t *start_idx, int32_t *end_idx,
                               int32_t *start_row, int32_t *end_row,
                               uint8_t *start_flag) {
  if (np < 1 || nnz < 0 || m < 0) return 1;
  for (int32_t i = 0; i < np; i++) {
    int64_t s, e;
    part_range(nnz, np, i, &s, &e);
    start_idx[i] = (int32_t)s;
    end_idx[i] = (int32_t)e;
    start_row[i] = 0;
    end_row[i] = e < s ? -1 : m - 1;
    start_flag[i] = 0;
  }
  return 0;
}

/* Local row-index array of pCOO (Sec. 4.1): lrow[k] = row_idx[k] -
 * start_row of the partition that holds k.  Length nnz, partition i at
 * offset start_idx[i]. */
int ref_partition_local_coo(const int32_t *row_idx, int32_t np,
                            const int32_t *start_idx, const int32_t *end_idx,
                            const int32_t *start_row, int32_t *lrow) {
  for (int32_t i = 0; i < np; i++)
    for (int64_t k = start_idx[i]; k <= end_idx[i]; k++)
      lrow[k] = row_idx[k] - start_row[i];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Plain SpMV, y = alpha*A*x + beta*y (Sec. 2.2, Alg. 1 under reading R1).   */
/* beta == 0 means y is not read (its old contents may be NaN).              */
/* ------------------------------------------------------------------------ */

static double finish(double alpha, double acc, double beta, double yin) {
  return beta == 0.0 ? alpha * acc : alpha * acc + beta * yin;
}

/* Alg. 1: row loop, inner loop over the row's nonzeros in storage order. */
void ref_spmv_csr(int32_t m, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *val, double alpha, const double *x, double beta,
                  double *y) {
  for (int32_t i = 0; i < m; i++) {
    double acc = 0.0;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; j++)
      acc += val[j] * x[col_idx[j]];
    y[i] = finish(alpha, acc, beta, y[i]);
  }
}

/* CSC SpMV: Alg. 1 with the roles of x and y switched (Sec. 2.2): column
 * loop, scatter of val*x[col] into the row accumulators. */
void ref_spmv_csc(int32_t m, int32_t n, const int32_t *col_ptr,
                  const int32_t *row_idx, const double *val, double alpha,
                  const double *x, double beta, double *y) {
  double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  for (int32_t c = 0; c < n; c++)
    for (int64_t j = col_ptr[c]; j < col_ptr[c + 1]; j++)
      acc[row_idx[j]] += val[j] * x[c];
  for (int32_t i = 0; i < m; i++) y[i] = finish(alpha, acc[i], beta, y[i]);
  free(acc);
}

/* COO SpMV: one loop over all nonzeros (Sec. 2.2). */
void ref_spmv_coo(int32_t m, int64_t nnz, const int32_t *row_idx,
                  const int32_t *col_idx, const double *val, double alpha,
                  const double *x, double beta, double *y) {
  double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  for (int64_t j = 0; j < nnz; j++) acc[row_idx[j]] += val[j] * x[col_idx[j]];
  for (int32_t i = 0; i < m; i++) y[i] = finish(alpha, acc[i], beta, y[i]);
  free(acc);
}

/* Plain sparse matrix times a block of k dense vectors stored row-major
 * (X is n x k, Y is m x k): k independent applications of Alg. 1. */
void ref_spmm_csr(int32_t m, int32_t k, const int32_t *row_ptr,
                  const int32_t *col_idx, const double *val, double alpha,
                  const double *X, double beta, double *Y) {
  for (int32_t i = 0; i < m; i++)
    for (int32_t v = 0; v < k; v++) {
      double acc = 0.0;
      for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; j++)
        acc += val[j] * X[(int64_t)col_idx[j] * k + v];
      Y[(int64_t)i * k + v] = finish(alpha, acc, beta, Y[(int64_t)i * k + v]);
    }
}

/* ------------------------------------------------------------------------ */
/* Partitioned SpMV with the paper's merge (Alg. 3, 5, 7), as a CPU          */
/* simulation of the multi-device method.  Each partition computes its own   */
/* partial result py_i over its nonzeros only; the merge then combines them. */
/* ------------------------------------------------------------------------ */

/* Alg. 3 under readings R2-R6.  part_* are the Alg. 2 outputs. */
int ref_pspmv_csr(int32_t m, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *val, int32_t np, const int32_t *start_idx,
                  const int32_t *end_idx, const int32_t *start_row,
                  const int32_t *end_row, double alpha, const double *x,
                  double beta, double *y) {
  /* acc[r]: running merge of partials of row r in partition order;
   * touched[r]: whether any partition produced a partial for r. */
  double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  for (int32_t i = 0; i < np; i++) {
    if (end_idx[i] < start_idx[i]) continue;
    /* py_i: one partial per row start_row..end_row over [s_i, e_i] only. */
    int32_t nr = end_row[i] - start_row[i] + 1;
    double *py = (double *)calloc((size_t)nr, sizeof(double));
    for (int32_t r = start_row[i]; r <= end_row[i]; r++) {
      int64_t lo = row_ptr[r] > start_idx[i] ? row_ptr[r] : start_idx[i];
      int64_t hi = row_ptr[r + 1] - 1 < end_idx[i] ? row_ptr[r + 1] - 1
                                                   : end_idx[i];
      double s = 0.0;
      for (int64_t j = lo; j <= hi; j++) s += val[j] * x[col_idx[j]];
      py[r - start_row[i]] = s;
    }
    /* merge: the segment goes to rows start_row..end_row; the first row is
     * added to what earlier partitions left there (start_flag case). */
    for (int32_t r = start_row[i]; r <= end_row[i]; r++)
      acc[r] += py[r - start_row[i]];
    free(py);
  }
  for (int32_t r = 0; r < m; r++) y[r] = finish(alpha, acc[r], beta, y[r]);
  free(acc);
  return 0;
}

/* Alg. 5 under reading R7: every partition produces a full m-vector of
 * partials; the merge sums them in partition order. */
int ref_pspmv_csc(int32_t m, const int32_t *col_ptr, const int32_t *row_idx,
                  const double *val, int32_t np, const int32_t *start_idx,
                  const int32_t *end_idx, const int32_t *start_col,
                  const int32_t *end_col, double alpha, const double *x,
                  double beta, double *y) {
  double *sum = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  double *py = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  for (int32_t i = 0; i < np; i++) {
    if (end_idx[i] < start_idx[i]) continue;
    memset(py, 0, (size_t)(m > 0 ? m : 1) * sizeof(double));
    for (int32_t c = start_col[i]; c <= end_col[i]; c++) {
      int64_t lo = col_ptr[c] > start_idx[i] ? col_ptr[c] : start_idx[i];
      int64_t hi = col_ptr[c + 1] - 1 < end_idx[i] ? col_ptr[c + 1] - 1
                                                   : end_idx[i];
      for (int64_t j = lo; j <= hi; j++) py[row_idx[j]] += val[j] * x[c];
    }
    for (int32_t r = 0; r < m; r++) sum[r] += py[r];
  }
  for (int32_t r = 0; r < m; r++) y[r] = finish(alpha, sum[r], beta, y[r]);
  free(py);
  free(sum);
  return 0;
}

/* Partitioned SpMV of a COO matrix sorted by column or in no order
 * (reading R9): partition i adds val*x[col] for its nonzeros, in storage
 * order, into its own full m-vector of partials py_i (the extra memory
 * Sec. 3.2.3 mentions); then y = alpha * sum_i py_i + beta * y_in, the
 * partials summed in partition order. */
int ref_pspmv_coo_scatter(int32_t m, const int32_t *row_idx,
                          const int32_t *col_idx, const double *val, int32_t np,
                          const int32_t *start_idx, const int32_t *end_idx,
                          double alpha, const double *x, double beta,
                          double *y) {
  double *sum = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  double *py = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  for (int32_t i = 0; i < np; i++) {
    if (end_idx[i] < start_idx[i]) continue;
    memset(py, 0, (size_t)(m > 0 ? m : 1) * sizeof(double));
    for (int64_t j = start_idx[i]; j <= end_idx[i]; j++)
      py[row_idx[j]] += val[j] * x[col_idx[j]];
    for (int32_t r = 0; r < m; r++) sum[r] += py[r];
  }
  for (int32_t r = 0; r < m; r++) y[r] = finish(alpha, sum[r], beta, y[r]);
  free(py);
  free(sum);
  return 0;
}

/* Alg. 7: the COO analogue of Alg. 3 (row-sorted input). */
int ref_pspmv_coo(int32_t m, const int32_t *row_idx, const int32_t *col_idx,
                  const double *val, int32_t np, const int32_t *start_idx,
                  const int32_t *end_idx, const int32_t *start_row,
                  const int32_t *end_row, double alpha, const double *x,
                  double beta, double *y) {
  double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  for (int32_t i = 0; i < np; i++) {
    if (end_idx[i] < start_idx[i]) continue;
    int32_t nr = end_row[i] - start_row[i] + 1;
    double *py = (double *)calloc((size_t)nr, sizeof(double));
    for (int64_t j = start_idx[i]; j <= end_idx[i]; j++)
      py[row_idx[j] - start_row[i]] += val[j] * x[col_idx[j]];
    for (int32_t r = start_row[i]; r <= end_row[i]; r++)
      acc[r] += py[r - start_row[i]];
    free(py);
  }
  for (int32_t r = 0; r < m; r++) y[r] = finish(alpha, acc[r], beta, y[r]);
  free(acc);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Error-free transformation used by the low-precision form.                 */
/* ------------------------------------------------------------------------ */

/* Knuth's TwoSum in binary32: s = fl(a+b) and e with a + b = s + e exactly.
 * volatile forces every intermediate to be a rounded float. */
void ref_two_sum_f32(float a, float b, float *s, float *e) {
  volatile float sv = a + b;
  volatile float bv = sv - a;
  volatile float av = sv - bv;
  volatile float db = b - bv;
  volatile float da = a - av;
  *s = sv;
  *e = da + db;
}

/* Plain recursive binary32 summation (the uncompensated reference). */
float ref_sum_f32(const float *v, int64_t n) {
  volatile float s = 0.0f;
  for (int64_t i = 0; i < n; i++) s = s + v[i];
  return s;
}

/* Compensated binary32 summation by cascaded TwoSum (Ogita, Rump and Oishi,
 * "Accurate sum and dot product", 2005, Algorithm 4.4 "Sum2"): result is as
 * accurate as if computed in twice the working precision, then rounded. */
float ref_sum2_f32(const float *v, int64_t n) {
  float s = 0.0f, c = 0.0f;
  for (int64_t i = 0; i < n; i++) {
    float t, e;
    ref_two_sum_f32(s, v[i], &t, &e);
    s = t;
    volatile float cv = c + e;
    c = cv;
  }
  volatile float r = s + c;
  return r;
}
