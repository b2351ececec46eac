/*
 * cpu_baseline.c -- the all-core CPU baseline of the benchmark.
 *
 * NOT THE ORACLE, and no test compares against it.  It is the multi-core
 * CPU SpMV that the benchmark times beside the single-threaded oracle, so
 * that the GPU numbers stand next to a CPU program that uses every host
 * core.  Like the oracle it is measurement infrastructure only: nothing on
 * the product path calls, links or loads it, and it shares no code with the
 * CUDA library or with msrep_oracle.c.
 *
 * Design (the paper's Sec. 3.3 gives each partition a host thread): the
 * nonzeros are cut into np = the thread count partitions of equal size,
 * floor(i*nnz/np) .. floor((i+1)*nnz/np)-1 (Alg. 2/4/6), one OpenMP thread
 * per partition.
 *   CSR, row-sorted COO: each thread sums its rows in order; the partial
 *     sums of the first and last row of its range go to a side array, and
 *     rows split between partitions are merged afterwards in partition
 *     order (Alg. 3/7's merge), alpha applied to the merged sum.
 *   CSC: each thread scatters its columns into a private partial vector;
 *     the partial vectors are then summed row block by row block, in
 *     parallel (Alg. 5's merge of partial vectors).
 * y = alpha*A*x (beta = 0), FP64.  Build: gcc -O3 -fopenmp.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int cpu_threads(void) { return omp_get_max_threads(); }

/* row owning nonzero k: largest r with ptr[r] <= k (binary search) */
static int32_t owner(const int32_t *ptr, int32_t n_major, int64_t k) {
  int32_t lo = 0, hi = n_major - 1;
  while (lo < hi) {
    int32_t mid = lo + (hi - lo + 1) / 2;
    if ((int64_t)ptr[mid] <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

/* CSR (row_ptr != NULL) or row-sorted COO (row_idx != NULL). */
static int spmv_rows(int32_t m, int64_t nnz, const int32_t *row_ptr, const int32_t *row_idx,
                     const int32_t *col, const double *val, const double *x, double alpha,
                     double *y) {
  const int np = omp_get_max_threads();
  double *head = (double *)calloc((size_t)np, sizeof(double));
  double *tail = (double *)calloc((size_t)np, sizeof(double));
  int32_t *first = (int32_t *)malloc(sizeof(int32_t) * (size_t)np);
  int32_t *last = (int32_t *)malloc(sizeof(int32_t) * (size_t)np);
  if (!head || !tail || !first || !last) return 1;
  memset(y, 0, sizeof(double) * (size_t)m);
#pragma omp parallel num_threads(np)
  {
    const int i = omp_get_thread_num();
    const int64_t s = ((int64_t)i * nnz) / np, e = ((int64_t)(i + 1) * nnz) / np;
    first[i] = -1;
    last[i] = -1;
    if (s < e) {
      int32_t r = row_ptr ? owner(row_ptr, m, s) : row_idx[s];
      first[i] = r;
      double acc = 0.0;
      int in_first = 1;
      for (int64_t k = s; k < e; k++) {
        const int32_t rk = row_ptr ? r : row_idx[k];
        if (row_ptr) {
          while ((int64_t)row_ptr[r + 1] <= k) { /* row r ended before k */
            if (in_first) head[i] = acc; else y[r] = alpha * acc;
            in_first = 0;
            acc = 0.0;
            r++;
          }
        } else if (rk != r) {
          if (in_first) head[i] = acc; else y[r] = alpha * acc;
          in_first = 0;
          acc = 0.0;
          r = rk;
        }
        acc += val[k] * x[col[k]];
      }
      last[i] = r;
      if (in_first) head[i] = acc; else tail[i] = acc;
    }
  }
  /* merge in partition order: every row that some partition's first or
   * last row touches gets the sum of its partials */
  int32_t cur = -1;
  double sum = 0.0;
  for (int i = 0; i < np; i++) {
    if (first[i] < 0) continue;
    if (first[i] != cur) {
      if (cur >= 0) y[cur] = alpha * sum;
      cur = first[i];
      sum = 0.0;
    }
    sum += head[i];
    if (last[i] != first[i]) {
      y[cur] = alpha * sum;
      cur = last[i];
      sum = tail[i];
    }
  }
  if (cur >= 0) y[cur] = alpha * sum;
  free(head);
  free(tail);
  free(first);
  free(last);
  return 0;
}

int cpu_spmv_csr(int32_t m, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                 const double *val, const double *x, double alpha, double *y) {
  return spmv_rows(m, nnz, row_ptr, NULL, col, val, x, alpha, y);
}

int cpu_spmv_coo(int32_t m, int64_t nnz, const int32_t *row_idx, const int32_t *col,
                 const double *val, const double *x, double alpha, double *y) {
  return spmv_rows(m, nnz, NULL, row_idx, col, val, x, alpha, y);
}

/* CSC: private partial vectors per partition, summed afterwards.  part
 * holds np*m doubles of scratch (np = cpu_threads()). */
int cpu_spmv_csc(int32_t m, int32_t n, int64_t nnz, const int32_t *col_ptr,
                 const int32_t *row, const double *val, const double *x, double alpha,
                 double *y, double *part) {
  const int np = omp_get_max_threads();
#pragma omp parallel num_threads(np)
  {
    const int i = omp_get_thread_num();
    double *py = part + (size_t)i * (size_t)m;
    memset(py, 0, sizeof(double) * (size_t)m);
    const int64_t s = ((int64_t)i * nnz) / np, e = ((int64_t)(i + 1) * nnz) / np;
    if (s < e) {
      int32_t c = owner(col_ptr, n, s);
      for (int64_t k = s; k < e; k++) {
        while ((int64_t)col_ptr[c + 1] <= k) c++;
        py[row[k]] += val[k] * x[c];
      }
    }
#pragma omp barrier
    const int64_t r0 = ((int64_t)i * m) / np, r1 = ((int64_t)(i + 1) * m) / np;
    for (int64_t r = r0; r < r1; r++) {
      double t = 0.0;
      for (int j = 0; j < np; j++) t += part[(size_t)j * (size_t)m + (size_t)r];
      y[r] = alpha * t;
    }
  }
  return 0;
}
