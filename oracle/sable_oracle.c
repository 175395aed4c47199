/*
 * FP64 CPU oracle for sparse matrix-vector and sparse matrix-matrix products.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or constant with the CUDA library it checks.
 *
 * What it computes is the plain definition of the two kernels the paper
 * evaluates (Section 5, "Kernels"):
 *     SpMV   y_i  = sum_j A_ij * x_j
 *     SpMM   C    = A * B,  B dense row-major with N columns
 * The matrix is given in coordinate (COO) form exactly as the caller passed it;
 * duplicated coordinates therefore contribute the sum of their values, which
 * is the library's documented duplicate rule.  Every product and sum is taken
 * in double precision (FP32 inputs widen exactly).  There is no blocking,
 * reordering or format conversion: one pass over the COO triples.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* y[0..m) = A x, A given as nnz COO triples (row[k], col[k], val[k]). */
void oracle_spmv_coo(int64_t m, int64_t nnz, const int32_t *row,
                     const int32_t *col, const double *val, const double *x,
                     double *y) {
  for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
  for (int64_t k = 0; k < nnz; ++k) y[row[k]] += val[k] * x[col[k]];
}

/* Same as oracle_spmv_coo with FP32 values and vector, widened per term. */
void oracle_spmv_coo_f32(int64_t m, int64_t nnz, const int32_t *row,
                         const int32_t *col, const float *val, const float *x,
                         double *y) {
  for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
  for (int64_t k = 0; k < nnz; ++k)
    y[row[k]] += (double)val[k] * (double)x[col[k]];
}

/* C[m x N] = A B with B[n x N] row-major (leading dimension ldb) and C
 * row-major (leading dimension ldc).  FP32 inputs, FP64 output. */
void oracle_spmm_coo_f32(int64_t m, int64_t nnz, const int32_t *row,
                         const int32_t *col, const float *val, const float *B,
                         int64_t N, int64_t ldb, double *C, int64_t ldc) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < N; ++j) C[i * ldc + j] = 0.0;
  for (int64_t k = 0; k < nnz; ++k) {
    const double a = (double)val[k];
    const float *b = B + (int64_t)col[k] * ldb;
    double *c = C + (int64_t)row[k] * ldc;
    for (int64_t j = 0; j < N; ++j) c[j] += a * (double)b[j];
  }
}

/* Rows of C = A B for a subset of rows only: out[s, :] = row sel[s] of A B.
 * Used to check very large products on sampled outputs.  The rows in `sel`
 * must be distinct; `slot` is caller scratch of m int64 entries. */
void oracle_spmm_coo_rows_f32(int64_t m, int64_t nnz, const int32_t *row,
                              const int32_t *col, const float *val,
                              const float *B, int64_t N, int64_t ldb,
                              int64_t nsel, const int64_t *sel, int64_t *slot,
                              double *out) {
  for (int64_t i = 0; i < m; ++i) slot[i] = -1;
  for (int64_t s = 0; s < nsel; ++s) slot[sel[s]] = s;
  for (int64_t s = 0; s < nsel; ++s)
    for (int64_t j = 0; j < N; ++j) out[s * N + j] = 0.0;
  for (int64_t k = 0; k < nnz; ++k) {
    const int64_t s = slot[row[k]];
    if (s < 0) continue;
    const double a = (double)val[k];
    const float *b = B + (int64_t)col[k] * ldb;
    double *o = out + s * N;
    for (int64_t j = 0; j < N; ++j) o[j] += a * (double)b[j];
  }
}

/* COO -> CSR by a stable counting sort on the row index: rp[0..m] row
 * pointers, perm[0..nnz) the COO positions in row order, input order kept
 * within each row.  A CSR row loop over this order adds each row's terms in
 * the same order as the COO loop above, so its FP64 results are identical. */
void oracle_coo_rows(int64_t m, int64_t nnz, const int32_t *row, int64_t *rp,
                     int64_t *perm) {
  for (int64_t i = 0; i <= m; ++i) rp[i] = 0;
  for (int64_t k = 0; k < nnz; ++k) ++rp[row[k] + 1];
  for (int64_t i = 0; i < m; ++i) rp[i + 1] += rp[i];
  int64_t *at = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
  if (!at) return;
  for (int64_t i = 0; i < m; ++i) at[i] = rp[i];
  for (int64_t k = 0; k < nnz; ++k) perm[at[row[k]]++] = k;
  free(at);
}

/* y[0..m) = A x from the row order of oracle_coo_rows: y_i = sum over the
 * row's terms, FP32 inputs widened per term.  Built twice: plainly, and with
 * -fopenmp, where the rows are shared among the host's threads (each row
 * still summed by one thread in the order above); oracle_threads() says how
 * many threads that build runs. */
void oracle_spmv_rows_f32(int64_t m, const int64_t *rp, const int64_t *perm,
                          const int32_t *col, const float *val, const float *x,
                          double *y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024)
#endif
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
      const int64_t k = perm[q];
      s += (double)val[k] * (double)x[col[k]];
    }
    y[i] = s;
  }
}

#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
#else
int oracle_threads(void) { return 1; }
#endif
