/*
 * orc_sparse.c - CSR building blocks of the CPU oracle (test infrastructure only).
 *
 * Transpose, the Galerkin sparse-sparse product and the pattern-masked product
 * use a dense sparse accumulator (SPA) per output row: values are summed in
 * ascending order of the left operand's column index k, each term a rounded
 * multiply followed by a rounded add (the file is compiled with
 * -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include "orc_internal.h"
#ifdef _OPENMP
#include <omp.h>
#endif

void orc_csr_alloc(orc_csr *a, int32_t nrows, int32_t ncols, int64_t nnz, int with_val) {
    a->nrows = nrows;
    a->ncols = ncols;
    a->nnz = nnz;
    a->rowptr = (int32_t *)orc_xcalloc((size_t)nrows + 1, sizeof(int32_t));
    a->col = (int32_t *)orc_xmalloc((size_t)nnz * sizeof(int32_t));
    a->val = with_val ? (double *)orc_xcalloc((size_t)nnz, sizeof(double)) : NULL;
}

void orc_csr_free(orc_csr *a) {
    if (!a) return;
    free(a->rowptr);
    free(a->col);
    free(a->val);
    a->rowptr = NULL;
    a->col = NULL;
    a->val = NULL;
    a->nrows = a->ncols = 0;
    a->nnz = 0;
}

void orc_csr_copy(const orc_csr *a, orc_csr *b) {
    orc_csr_alloc(b, a->nrows, a->ncols, a->nnz, a->val != NULL);
    memcpy(b->rowptr, a->rowptr, ((size_t)a->nrows + 1) * sizeof(int32_t));
    memcpy(b->col, a->col, (size_t)a->nnz * sizeof(int32_t));
    if (a->val) memcpy(b->val, a->val, (size_t)a->nnz * sizeof(double));
}

/* Threads of the row loops (OpenMP).  Every result is independent of the
 * count: rows are computed exactly as by one thread, each with its own
 * scratch, and sums over many terms go through orc_dot's fixed chunks. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Neumaier's compensated summation step (Neumaier 1974, an improvement of
 * Kahan's): the running sum's rounding error is collected in *c. */
static inline void neumaier_add(double *s, double *c, double p) {
    const double t = *s + p;
    if (fabs(*s) >= fabs(p)) *c += (*s - t) + p;
    else *c += (p - t) + *s;
    *s = t;
}

/* Inner product with compensated summation, so the result's error does not
 * grow with n (these sums run over millions of terms: Frobenius products on
 * the interpolation pattern, where a plain sequential sum would dominate the
 * comparison).  The terms are summed in fixed chunks of ORC_DOT_CHUNK, each
 * compensated in index order, and the chunk sums are added, compensated, in
 * chunk order: the same value for any thread count (n <= ORC_DOT_CHUNK: one
 * chunk, the plain compensated sum in index order). */
#define ORC_DOT_CHUNK 4096
double orc_dot(int64_t n, const double *x, const double *y) {
    const int64_t nch = (n + ORC_DOT_CHUNK - 1) / ORC_DOT_CHUNK;
    if (nch <= 1) {
        double s = 0.0, c = 0.0;
        for (int64_t i = 0; i < n; i++) neumaier_add(&s, &c, x[i] * y[i]);
        return s + c;
    }
    double *part = (double *)orc_xmalloc((size_t)nch * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < nch; ch++) {
        const int64_t lo = ch * ORC_DOT_CHUNK, hi = lo + ORC_DOT_CHUNK < n ? lo + ORC_DOT_CHUNK : n;
        double s = 0.0, c = 0.0;
        for (int64_t i = lo; i < hi; i++) neumaier_add(&s, &c, x[i] * y[i]);
        part[ch] = s + c;
    }
    double s = 0.0, c = 0.0;
    for (int64_t ch = 0; ch < nch; ch++) neumaier_add(&s, &c, part[ch]);
    free(part);
    return s + c;
}

double orc_nrm2(int64_t n, const double *x) { return sqrt(orc_dot(n, x, x)); }

/* y = A x, each row summed in stored (ascending column) order. */
void orc_spmv(const orc_csr *A, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < A->nrows; i++) {
        double s = 0.0;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) s += A->val[e] * x[A->col[e]];
        y[i] = s;
    }
}

/* A^T: entries are visited row by row, so every output row comes out sorted. */
int orc_transpose(const orc_csr *A, orc_csr *At) {
    orc_csr_alloc(At, A->ncols, A->nrows, A->nnz, A->val != NULL);
    for (int64_t e = 0; e < A->nnz; e++) At->rowptr[A->col[e] + 1]++;
    for (int32_t j = 0; j < A->ncols; j++) At->rowptr[j + 1] += At->rowptr[j];
    int32_t *next = (int32_t *)orc_xmalloc(((size_t)A->ncols + 1) * sizeof(int32_t));
    memcpy(next, At->rowptr, ((size_t)A->ncols + 1) * sizeof(int32_t));
    for (int32_t i = 0; i < A->nrows; i++) {
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
            int32_t j = A->col[e];
            int32_t dst = next[j]++;
            At->col[dst] = i;
            if (A->val) At->val[dst] = A->val[e];
        }
    }
    free(next);
    return ORC_OK;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * C = A B (Gustavson).  The pattern of C is the symbolic product: every (i,j)
 * reached by some a_ik b_kj with both stored, explicit zeros kept (this keeps
 * patterns independent of cancellation).  Values: sum over k in ascending
 * column order of row i of A.
 */
int orc_spgemm(const orc_csr *A, const orc_csr *B, orc_csr *C) {
    if (A->ncols != B->nrows) return ORC_EINVAL;
    int32_t n = A->nrows, m = B->ncols;
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    /* symbolic: count distinct columns per row (a marker array per thread) */
#pragma omp parallel
    {
        int32_t *marker = (int32_t *)orc_xmalloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
        for (int32_t j = 0; j < m; j++) marker[j] = -1;
#pragma omp for schedule(dynamic, 256)
        for (int32_t i = 0; i < n; i++) {
            int32_t cnt = 0;
            for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
                int32_t k = A->col[e];
                for (int32_t f = B->rowptr[k]; f < B->rowptr[k + 1]; f++) {
                    int32_t j = B->col[f];
                    if (marker[j] != i) { marker[j] = i; cnt++; }
                }
            }
            rowptr[i + 1] = cnt;
        }
        free(marker);
    }
    int64_t total = 0;
    for (int32_t i = 0; i < n; i++) {
        total += rowptr[i + 1];
        if (total > INT32_MAX) { free(rowptr); return ORC_EINVAL; }
        rowptr[i + 1] = (int32_t)total;
    }
    C->nrows = n;
    C->ncols = m;
    C->nnz = total;
    C->rowptr = rowptr;
    C->col = (int32_t *)orc_xmalloc((size_t)total * sizeof(int32_t));
    int with_val = (A->val != NULL && B->val != NULL);
    C->val = with_val ? (double *)orc_xcalloc((size_t)total, sizeof(double)) : NULL;
    /* numeric: each row summed in ascending k (its own sparse accumulator) */
#pragma omp parallel
    {
        int32_t *marker = (int32_t *)orc_xmalloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
        double *spa = (double *)orc_xcalloc((size_t)(m > 0 ? m : 1), sizeof(double));
        for (int32_t j = 0; j < m; j++) marker[j] = -1;
#pragma omp for schedule(dynamic, 256)
        for (int32_t i = 0; i < n; i++) {
            int32_t start = rowptr[i], cnt = 0;
            for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
                int32_t k = A->col[e];
                double a = with_val ? A->val[e] : 0.0;
                for (int32_t f = B->rowptr[k]; f < B->rowptr[k + 1]; f++) {
                    int32_t j = B->col[f];
                    if (marker[j] != i) {
                        marker[j] = i;
                        spa[j] = 0.0;
                        C->col[start + cnt++] = j;
                    }
                    if (with_val) spa[j] = spa[j] + a * B->val[f];
                }
            }
            qsort(C->col + start, (size_t)cnt, sizeof(int32_t), cmp_i32);
            if (with_val)
                for (int32_t q = 0; q < cnt; q++) C->val[start + q] = spa[C->col[start + q]];
        }
        free(spa);
        free(marker);
    }
    return ORC_OK;
}

/*
 * W = Mask_N(A X): the product A X restricted to the pattern of X, which W
 * shares (the fixed interpolation pattern N).  Entry (i,j) of the pattern gets
 * sum_k a_ik X_kj over k in ascending order; X_kj = 0 where (k,j) is not in N.
 */
void orc_masked_product(const orc_csr *A, const orc_csr *X, orc_csr *W) {
    int32_t m = X->ncols;
#pragma omp parallel
    {
        double *spa = (double *)orc_xcalloc((size_t)(m > 0 ? m : 1), sizeof(double));
        int32_t *marker = (int32_t *)orc_xmalloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
        for (int32_t j = 0; j < m; j++) marker[j] = -1;
#pragma omp for schedule(dynamic, 256)
        for (int32_t i = 0; i < A->nrows; i++) {
            for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
                int32_t k = A->col[e];
                double a = A->val[e];
                for (int32_t f = X->rowptr[k]; f < X->rowptr[k + 1]; f++) {
                    int32_t j = X->col[f];
                    if (marker[j] != i) { marker[j] = i; spa[j] = 0.0; }
                    spa[j] = spa[j] + a * X->val[f];
                }
            }
            for (int32_t q = X->rowptr[i]; q < X->rowptr[i + 1]; q++) {
                int32_t j = X->col[q];
                W->val[q] = (marker[j] == i) ? spa[j] : 0.0;
            }
        }
        free(spa);
        free(marker);
    }
}

/* release a buffer the oracle allocated (used by the Python binding) */
void orc_free(void *p) { free(p); }
