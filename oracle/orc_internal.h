/* orc_internal.h - private helpers of the CPU oracle (test infrastructure only). */
#ifndef ORC_INTERNAL_H
#define ORC_INTERNAL_H
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

/* The oracle is a checker: on allocation failure it stops loudly. */
static inline void *orc_xmalloc(size_t n) {
    void *p = malloc(n ? n : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory (%zu bytes)\n", n); abort(); }
    return p;
}
static inline void *orc_xcalloc(size_t n, size_t s) {
    void *p = calloc(n ? n : 1, s ? s : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

/* Guard constant for floating threshold tests: keep <=> v >= theta*ref*(1-g). */
#define ORC_GUARD 1e-10
/* CG energy minimisation stops once <R,Z> <= ORC_CG_STOP * <R0,Z0> (the
 * residual is ~1e-11 of its start: the Krylov space is exhausted and further
 * steps would only amplify rounding noise). */
#define ORC_CG_STOP 1e-22
/* GMRES energy minimisation treats h_{j+1,j} <= ORC_GMRES_BREAK * beta as a
 * (happy) breakdown. */
#define ORC_GMRES_BREAK 1e-14

void orc_csr_alloc(orc_csr *a, int32_t nrows, int32_t ncols, int64_t nnz, int with_val);
void orc_csr_copy(const orc_csr *a, orc_csr *b);
double orc_dot(int64_t n, const double *x, const double *y);
double orc_nrm2(int64_t n, const double *x);
void orc_spmv(const orc_csr *A, const double *x, double *y);
struct orc_level {
    orc_csr A, S, N, T, P, R;
    int32_t *agg, *roots, *rowtype;
    int32_t nc;
    double *B, *Bc, *Bhat, *Bhatc;
    double *diag;
};

struct orc_hier {
    int nlev;           /* number of levels including the coarsest */
    orc_level *lev;     /* nlev entries; the last has only A */
    double *LU;         /* dense LU of the coarsest operator */
    int32_t *piv;
    int32_t ncoarse;
    orc_params p;
    int64_t near_ties;
};

#endif
