/*
 * orc_setup.c - root-node AMG setup (Alg. 3, Sec. 3) in the CPU oracle.
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include "orc_internal.h"

/* ------------------------------------------------------------------------ */
/* Strength of connection (Sec. 3.2, eq. soc; symmetric measure of Sec. 2.3).
 *
 * For j != i: v_ij = |a_ij| / sqrt(|a_ii| |a_jj|), strong iff v_ij >= theta.
 * Reading: the paper prints a_ij/sqrt(a_ii a_jj) > 0.25 without the absolute
 * value and with a strict '>'; for the 5-point Laplacian every off-diagonal
 * sits exactly on 0.25, so the literal reading would give no coarsening.  We
 * take |.| and '>=' with the guard band (1-g).
 * Rows are then scaled so that the largest strong off-diagonal and the
 * diagonal are both 1 (eq. soc).  A row without strong off-diagonals keeps
 * only S_ii = 1.
 */
int orc_strength(const orc_csr *A, double theta, orc_csr *S) {
    int32_t n = A->nrows;
    double *diag = (double *)orc_xmalloc((size_t)n * sizeof(double));
    for (int32_t i = 0; i < n; i++) {
        diag[i] = 0.0;
        int found = 0;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++)
            if (A->col[e] == i) { diag[i] = A->val[e]; found = 1; }
        if (!found || diag[i] == 0.0) { free(diag); return ORC_EINVAL; }
    }
    double thr = theta * (1.0 - ORC_GUARD);
    /* pass 1: count */
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) {
        int32_t cnt = 1; /* diagonal */
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
            int32_t j = A->col[e];
            if (j == i) continue;
            double v = fabs(A->val[e]) / sqrt(fabs(diag[i]) * fabs(diag[j]));
            if (v >= thr) cnt++;
        }
        rowptr[i + 1] = rowptr[i] + cnt;
    }
    S->nrows = n;
    S->ncols = n;
    S->nnz = rowptr[n];
    S->rowptr = rowptr;
    S->col = (int32_t *)orc_xmalloc((size_t)S->nnz * sizeof(int32_t));
    S->val = (double *)orc_xmalloc((size_t)S->nnz * sizeof(double));
    /* pass 2: fill in ascending column order (the diagonal takes its sorted place) */
    for (int32_t i = 0; i < n; i++) {
        double vmax = 0.0;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
            int32_t j = A->col[e];
            if (j == i) continue;
            double v = fabs(A->val[e]) / sqrt(fabs(diag[i]) * fabs(diag[j]));
            if (v >= thr && v > vmax) vmax = v;
        }
        int32_t dst = rowptr[i];
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
            int32_t j = A->col[e];
            if (j == i) {
                S->col[dst] = i;
                S->val[dst++] = 1.0;
                continue;
            }
            double v = fabs(A->val[e]) / sqrt(fabs(diag[i]) * fabs(diag[j]));
            if (v >= thr) {
                S->col[dst] = j;
                S->val[dst++] = v / vmax;
            }
        }
    }
    free(diag);
    return ORC_OK;
}

/* Classical strength (Sec. 3.2, the measure of Ruge and Stueben 1987 that
 * the paper lists beside the symmetric one): j is strong for i when
 * -a_ij >= theta (1 - g) m_i, m_i = max_{k != i} (-a_ik).  A row whose
 * off-diagonals are all >= 0 (m_i <= 0) has no strong entry.  Values are
 * -a_ij / m_i, so the row's largest off-diagonal is 1 (eq. soc); S_ii = 1. */
int orc_strength_classical(const orc_csr *A, double theta, orc_csr *S) {
    int32_t n = A->nrows;
    double thr = theta * (1.0 - ORC_GUARD);
    double *m = (double *)orc_xmalloc((size_t)n * sizeof(double));
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) {
        double mi = 0.0;
        int found = 0;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
            if (A->col[e] == i) {
                if (A->val[e] != 0.0) found = 1;
                continue;
            }
            double v = -A->val[e];
            if (v > mi) mi = v;
        }
        if (!found) { free(m); free(rowptr); return ORC_EINVAL; }
        m[i] = mi;
        int32_t cnt = 1;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++)
            if (A->col[e] != i && mi > 0.0 && -A->val[e] >= thr * mi) cnt++;
        rowptr[i + 1] = rowptr[i] + cnt;
    }
    S->nrows = n;
    S->ncols = n;
    S->nnz = rowptr[n];
    S->rowptr = rowptr;
    S->col = (int32_t *)orc_xmalloc((size_t)S->nnz * sizeof(int32_t));
    S->val = (double *)orc_xmalloc((size_t)S->nnz * sizeof(double));
    for (int32_t i = 0; i < n; i++) {
        int32_t dst = rowptr[i];
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
            int32_t j = A->col[e];
            if (j == i) {
                S->col[dst] = i;
                S->val[dst++] = 1.0;
            } else if (m[i] > 0.0 && -A->val[e] >= thr * m[i]) {
                S->col[dst] = j;
                S->val[dst++] = -A->val[e] / m[i];
            }
        }
    }
    free(m);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 mixing function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written from its published
 * definition.  Used only for aggregation priorities. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t h; int32_t i; } prio_t;

/* priority order: larger hash first, then larger node index */
static int prio_gt(uint64_t ha, int32_t ia, uint64_t hb, int32_t ib) {
    return ha > hb || (ha == hb && ia > ib);
}

static int cmp_prio_desc(const void *a, const void *b) {
    const prio_t *x = (const prio_t *)a, *y = (const prio_t *)b;
    if (prio_gt(x->h, x->i, y->h, y->i)) return -1;
    if (prio_gt(y->h, y->i, x->h, x->i)) return 1;
    return 0;
}

/*
 * Aggregation graph G = pattern(S) united with pattern(S)^T, without the
 * diagonal.  Reading: for nonsymmetric A the strength pattern is not
 * symmetric and the paper is silent; aggregation needs an undirected graph.
 */
static void build_aggregation_graph(const orc_csr *S, orc_csr *G) {
    int32_t n = S->nrows;
    orc_csr St;
    orc_transpose(S, &St);
    int32_t *mark = (int32_t *)orc_xmalloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) mark[i] = -1;
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) {
        int32_t cnt = 0;
        for (int32_t e = S->rowptr[i]; e < S->rowptr[i + 1]; e++) {
            int32_t j = S->col[e];
            if (j != i && mark[j] != i) { mark[j] = i; cnt++; }
        }
        for (int32_t e = St.rowptr[i]; e < St.rowptr[i + 1]; e++) {
            int32_t j = St.col[e];
            if (j != i && mark[j] != i) { mark[j] = i; cnt++; }
        }
        rowptr[i + 1] = rowptr[i] + cnt;
    }
    G->nrows = G->ncols = n;
    G->nnz = rowptr[n];
    G->rowptr = rowptr;
    G->col = (int32_t *)orc_xmalloc((size_t)G->nnz * sizeof(int32_t));
    G->val = NULL;
    for (int32_t i = 0; i < n; i++) mark[i] = -1;
    /* merge two sorted lists into a sorted row */
    for (int32_t i = 0; i < n; i++) {
        int32_t a = S->rowptr[i], ae = S->rowptr[i + 1], b = St.rowptr[i], be = St.rowptr[i + 1];
        int32_t dst = rowptr[i];
        while (a < ae || b < be) {
            int32_t ja = a < ae ? S->col[a] : INT32_MAX;
            int32_t jb = b < be ? St.col[b] : INT32_MAX;
            int32_t j = ja < jb ? ja : jb;
            if (ja == j) a++;
            if (jb == j) b++;
            if (j != i) G->col[dst++] = j;
        }
    }
    free(mark);
    orc_csr_free(&St);
}

/*
 * Aggregation with root nodes (Sec. 3.3).  The paper uses the sequential
 * greedy of Vanek, Mandel and Brezina; this project fixes a deterministic,
 * seeded rule instead:
 *   - priority pi(i) = (splitmix64(seed XOR i), i), compared lexicographically;
 *   - nodes without G-neighbours are isolated: unaggregated (agg = -1), no root;
 *   - roots: the distance-2 maximal independent set of G taken greedily in
 *     descending priority (a node is taken if no taken node lies within
 *     distance <= 2);
 *   - coarse indices number the roots by ascending node index;
 *   - pass 1: a non-root with a root neighbour joins the neighbouring root of
 *     largest priority;
 *   - pass 2: every other node joins the aggregate of its pass-1 neighbour
 *     whose root has the largest priority.
 * agg[i] = coarse index or -1; *roots (malloc'd) lists the root node of each
 * aggregate.
 */
int orc_aggregate(const orc_csr *S, uint64_t seed, int32_t *agg, int32_t **roots_out, int32_t *nc_out) {
    int32_t n = S->nrows;
    orc_csr G;
    build_aggregation_graph(S, &G);
    uint64_t *h = (uint64_t *)orc_xmalloc((size_t)n * sizeof(uint64_t));
    for (int32_t i = 0; i < n; i++) h[i] = orc_splitmix64(seed ^ (uint64_t)(uint32_t)i);
    prio_t *order = (prio_t *)orc_xmalloc((size_t)n * sizeof(prio_t));
    int32_t cnt = 0;
    for (int32_t i = 0; i < n; i++)
        if (G.rowptr[i + 1] > G.rowptr[i]) { order[cnt].h = h[i]; order[cnt].i = i; cnt++; }
    qsort(order, (size_t)cnt, sizeof(prio_t), cmp_prio_desc);
    char *taken = (char *)orc_xcalloc((size_t)n, 1);
    for (int32_t t = 0; t < cnt; t++) {
        int32_t i = order[t].i;
        int blocked = 0;
        for (int32_t e = G.rowptr[i]; e < G.rowptr[i + 1] && !blocked; e++) {
            int32_t j = G.col[e];
            if (taken[j]) { blocked = 1; break; }
            for (int32_t f = G.rowptr[j]; f < G.rowptr[j + 1]; f++)
                if (taken[G.col[f]]) { blocked = 1; break; }
        }
        if (!blocked) taken[i] = 1;
    }
    int32_t nc = 0;
    for (int32_t i = 0; i < n; i++) nc += taken[i];
    int32_t *roots = (int32_t *)orc_xmalloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    int32_t c = 0;
    for (int32_t i = 0; i < n; i++) {
        agg[i] = -1;
        if (taken[i]) { roots[c] = i; agg[i] = c; c++; }
    }
    /* pass 1 */
    int32_t *pass1 = (int32_t *)orc_xmalloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) {
        pass1[i] = -1;
        if (taken[i]) continue;
        int32_t best = -1;
        for (int32_t e = G.rowptr[i]; e < G.rowptr[i + 1]; e++) {
            int32_t j = G.col[e];
            if (taken[j] && (best < 0 || prio_gt(h[j], j, h[best], best))) best = j;
        }
        if (best >= 0) pass1[i] = agg[best];
    }
    /* pass 2 (reads only pass-1 assignments) */
    for (int32_t i = 0; i < n; i++) {
        if (taken[i] || pass1[i] >= 0) continue;
        if (G.rowptr[i + 1] == G.rowptr[i]) continue; /* isolated */
        int32_t best = -1; /* coarse index of chosen aggregate */
        for (int32_t e = G.rowptr[i]; e < G.rowptr[i + 1]; e++) {
            int32_t j = G.col[e];
            int32_t a = pass1[j];
            if (a < 0) continue;
            int32_t r = roots[a];
            if (best < 0 || prio_gt(h[r], r, h[roots[best]], roots[best])) best = a;
        }
        agg[i] = best; /* MIS-2 maximality guarantees best >= 0 */
        if (best < 0) {
            free(pass1); free(taken); free(order); free(h); free(roots); orc_csr_free(&G);
            return ORC_EINTERNAL;
        }
    }
    for (int32_t i = 0; i < n; i++)
        if (!taken[i] && pass1[i] >= 0) agg[i] = pass1[i];
    free(pass1);
    free(taken);
    free(order);
    free(h);
    orc_csr_free(&G);
    *roots_out = roots;
    *nc_out = nc;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Candidate improvement (Sec. 3.1, Alg. 3 'smooth'): a few relaxation sweeps
 * on A B = 0.  Reading: the relaxation is not named; we use the weighted
 * Jacobi of the cycle, B_i <- B_i - omega * ((A B)_i / a_ii), one column
 * (k = 1). */
void orc_smooth_candidates(const orc_csr *A, double *B, int sweeps, double omega) {
    int32_t n = A->nrows;
    double *Bn = (double *)orc_xmalloc((size_t)n * sizeof(double));
    for (int s = 0; s < sweeps; s++) {
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; i++) {
            double acc = 0.0, d = 0.0;
            for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++) {
                acc = acc + A->val[e] * B[A->col[e]];
                if (A->col[e] == i) d = A->val[e];
            }
            Bn[i] = B[i] - omega * (acc / d);
        }
        memcpy(B, Bn, (size_t)n * sizeof(double));
    }
    free(Bn);
}

void orc_row_types(int32_t n, const int32_t *agg, const int32_t *roots, int32_t nc, int32_t *rowtype) {
    for (int32_t i = 0; i < n; i++) rowtype[i] = (agg[i] < 0) ? ORC_UNAGG : ORC_FREE;
    for (int32_t c = 0; c < nc; c++) rowtype[roots[c]] = ORC_ROOT;
}

/*
 * Sparsity pattern N = S^d C (Sec. 3.4), pre-filter (Sec. 3.5, Alg. 4 with a
 * drop tolerance) and root_node_pattern (Sec. 3.4).
 *   N^0 = C (C_{i,agg(i)} = 1), N^t = S N^{t-1} by the SPA product.
 *   Pre-filter on non-root aggregated rows: keep N_ij >= theta_pre*max_j N_ij
 *   (with the guard band); reading: the entry of the row's own aggregate is
 *   always kept so that T has its entry there.
 *   Root rows become the identity row {agg(root)}: value 1.
 */
int orc_pattern(const orc_csr *S, const int32_t *agg, const int32_t *roots, int32_t nc, int d,
                double theta_pre, orc_csr *N) {
    int32_t n = S->nrows;
    orc_csr cur;
    int32_t naggd = 0;
    for (int32_t i = 0; i < n; i++) naggd += (agg[i] >= 0);
    orc_csr_alloc(&cur, n, nc, naggd, 1);
    for (int32_t i = 0, e = 0; i < n; i++) {
        if (agg[i] >= 0) { cur.col[e] = agg[i]; cur.val[e] = 1.0; e++; }
        cur.rowptr[i + 1] = e;
    }
    for (int t = 0; t < d; t++) {
        orc_csr nxt;
        int rc = orc_spgemm(S, &cur, &nxt);
        orc_csr_free(&cur);
        if (rc) return rc;
        cur = nxt;
    }
    int32_t *rowtype = (int32_t *)orc_xmalloc((size_t)n * sizeof(int32_t));
    orc_row_types(n, agg, roots, nc, rowtype);
    char *keep = (char *)orc_xcalloc((size_t)cur.nnz, 1);
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) {
        int32_t cnt = 0;
        if (rowtype[i] == ORC_ROOT) {
            for (int32_t e = cur.rowptr[i]; e < cur.rowptr[i + 1]; e++)
                if (cur.col[e] == agg[i]) { keep[e] = 1; cnt++; }
        } else if (rowtype[i] == ORC_FREE) {
            double m = 0.0;
            for (int32_t e = cur.rowptr[i]; e < cur.rowptr[i + 1]; e++)
                if (fabs(cur.val[e]) > m) m = fabs(cur.val[e]);
            double thr = theta_pre * m * (1.0 - ORC_GUARD);
            for (int32_t e = cur.rowptr[i]; e < cur.rowptr[i + 1]; e++) {
                int k = (theta_pre <= 0.0) || (fabs(cur.val[e]) >= thr) || (cur.col[e] == agg[i]);
                keep[e] = (char)k;
                cnt += k;
            }
        }
        rowptr[i + 1] = rowptr[i] + cnt;
    }
    N->nrows = n;
    N->ncols = nc;
    N->nnz = rowptr[n];
    N->rowptr = rowptr;
    N->col = (int32_t *)orc_xmalloc((size_t)N->nnz * sizeof(int32_t));
    N->val = (double *)orc_xmalloc((size_t)N->nnz * sizeof(double));
    for (int32_t i = 0; i < n; i++) {
        int32_t dst = rowptr[i];
        for (int32_t e = cur.rowptr[i]; e < cur.rowptr[i + 1]; e++) {
            if (!keep[e]) continue;
            N->col[dst] = cur.col[e];
            N->val[dst] = (rowtype[i] == ORC_ROOT) ? 1.0 : cur.val[e];
            dst++;
        }
    }
    free(keep);
    free(rowtype);
    orc_csr_free(&cur);
    return ORC_OK;
}

/*
 * Tentative interpolation (Sec. 3.6, eq. root-nodeform) for one candidate
 * (k = m = 1): coarse candidates by injection Bc_j = B(root_j); on the pattern
 * N, T_{i,agg(i)} = B_i / Bc_{agg(i)} (so root rows are exactly 1 and
 * T Bc = B on aggregated rows), every other pattern entry 0.  Overwrites
 * N->val with T.
 */
int orc_tentative(orc_csr *N, const int32_t *agg, const int32_t *roots, const double *B, double *Bc) {
    for (int32_t c = 0; c < N->ncols; c++) {
        Bc[c] = B[roots[c]];
        if (fabs(Bc[c]) < 1e-300) return ORC_EINVAL;
    }
    for (int32_t i = 0; i < N->nrows; i++) {
        for (int32_t e = N->rowptr[i]; e < N->rowptr[i + 1]; e++) {
            int32_t j = N->col[e];
            N->val[e] = (j == agg[i]) ? B[i] / Bc[j] : 0.0;
        }
    }
    return ORC_OK;
}

/*
 * Row-wise projection onto the constraint space {U : U Bc = 0} (eq. Tproj with
 * a zero right-hand side), restricted to each row's pattern J:
 *   free rows:  u <- u - (u.b / b.b) b,  b = Bc[J];
 *   free rows with a single pattern entry: u <- 0 (the exact projection);
 *   root and unaggregated rows are fixed: u <- 0.
 */
void orc_project(orc_csr *W, const int32_t *rowtype, const double *Bc) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < W->nrows; i++) {
        int32_t s = W->rowptr[i], e = W->rowptr[i + 1];
        /* fixed rows, and one-entry rows whose constraint space is exactly {0}
         * (the formula below would leave rounding noise there) */
        if (rowtype[i] != ORC_FREE || e - s == 1) {
            for (int32_t q = s; q < e; q++) W->val[q] = 0.0;
            continue;
        }
        double ub = 0.0, bb = 0.0;
        for (int32_t q = s; q < e; q++) {
            double b = Bc[W->col[q]];
            ub += W->val[q] * b;
            bb += b * b;
        }
        double c = ub / bb;
        for (int32_t q = s; q < e; q++) W->val[q] = W->val[q] - c * Bc[W->col[q]];
    }
}

/* ------------------------------------------------------------------------ */
/* k > 1 candidates (Sec. 3.6, eq. Tproj): every row-wise fit and projection
 * uses the k x k Gram matrix G_i = Bc_J^T Bc_J of the row's pattern J and its
 * pseudo-inverse (min-norm least squares; the system is underdetermined when
 * |J| >= k and Bc_J has full rank).  k = 1 keeps the scalar formulas above. */

/* Row fits from the singular value decomposition of Bc_J (|J| x k), not from
 * the Gram matrix G_i = Bc_J^T Bc_J: forming G squares the condition number,
 * so a fit through G carries rounding amplified by kappa(Bc_J)^2, one through
 * the SVD by kappa(Bc_J).  Singular values at most ORC_SV_CUT of the largest
 * are dropped (eigenvalues of G_i at most ORC_SV_CUT^2 = 1e-12 of the
 * largest): candidate combinations a row's pattern carries only below that
 * stay unfitted (minimal-norm least squares on the rest). */
#define ORC_KMAX 8
#define ORC_SV_CUT 1e-6

/* One-sided Jacobi SVD (Hestenes) of the len x k matrix M (row-major, k <=
 * ORC_KMAX): column pairs of W = M V are rotated until every pair is
 * orthogonal to 1e-15 of its norms (at most 30 sweeps); sigma_a = |W_a|.
 * On return U (len x k) holds W_a / sigma_a for the kept directions and zero
 * columns for the dropped ones, VS (k x k, row-major) holds V_a / sigma_a
 * (zero when dropped).  Returns the number of directions kept. */
int orc_row_svd(int len, int k, const double *M, double *U, double *VS) {
    double V[ORC_KMAX * ORC_KMAX];
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) V[i * k + j] = (i == j);
    for (int i = 0; i < len * k; i++) U[i] = M[i];  /* W, rotated in place */
    for (int sweep = 0; sweep < 30; sweep++) {
        int rotated = 0;
        for (int p = 0; p < k - 1; p++)
            for (int q = p + 1; q < k; q++) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < len; i++) {
                    const double wp = U[i * k + p], wq = U[i * k + q];
                    al += wp * wp;
                    be += wq * wq;
                    ga += wp * wq;
                }
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                rotated = 1;
                const double ze = (be - al) / (2.0 * ga);
                const double t = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(ze * ze + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int i = 0; i < len; i++) {
                    const double wp = U[i * k + p], wq = U[i * k + q];
                    U[i * k + p] = c * wp - sn * wq;
                    U[i * k + q] = sn * wp + c * wq;
                }
                for (int r = 0; r < k; r++) {
                    const double vp = V[r * k + p], vq = V[r * k + q];
                    V[r * k + p] = c * vp - sn * vq;
                    V[r * k + q] = sn * vp + c * vq;
                }
            }
        if (!rotated) break;
    }
    double sig[ORC_KMAX], smax = 0.0;
    for (int a = 0; a < k; a++) {
        double ss = 0.0;
        for (int i = 0; i < len; i++) ss += U[i * k + a] * U[i * k + a];
        sig[a] = sqrt(ss);
        if (sig[a] > smax) smax = sig[a];
    }
    int rank = 0;
    for (int a = 0; a < k; a++) {
        const int keep = sig[a] > ORC_SV_CUT * smax;
        rank += keep;
        for (int i = 0; i < len; i++) U[i * k + a] = keep ? U[i * k + a] / sig[a] : 0.0;
        for (int r = 0; r < k; r++) VS[r * k + a] = keep ? V[r * k + a] / sig[a] : 0.0;
    }
    return rank;
}

/* Min-norm update of one row's values t (pattern columns col[s..e)) so that
 * (t + u) Bc_J = target, by least squares on the kept directions of Bc_J =
 * U Sigma V^T (eq. Tproj):
 *   target given: r = target - t Bc_J, u = (r V Sigma^+) U^T;
 *   target NULL (the projection onto {u : u Bc_J = 0}): t <- t - (t U) U^T,
 *   and a row whose pattern has no more entries than the rank of Bc_J is
 *   fixed by the constraints and set to exactly 0, as a one-entry row is for
 *   k = 1. */
#define ORC_FIT_STACK 64
static void row_fit_k(int32_t s, int32_t e, const int32_t *col, double *val, const double *target,
                      const double *Bc, int k) {
    const int len = e - s;
    if (len <= 0) return;
    double Ms[ORC_FIT_STACK * ORC_KMAX], Us[ORC_FIT_STACK * ORC_KMAX], VS[ORC_KMAX * ORC_KMAX];
    double *M = Ms, *U = Us;
    if (len > ORC_FIT_STACK) {
        M = (double *)orc_xmalloc((size_t)len * k * sizeof(double));
        U = (double *)orc_xmalloc((size_t)len * k * sizeof(double));
    }
    for (int q = 0; q < len; q++)
        for (int a = 0; a < k; a++) M[q * k + a] = Bc[(size_t)col[s + q] * k + a];
    const int rank = orc_row_svd(len, k, M, U, VS);
    double c[ORC_KMAX];
    if (!target) {
        if (rank >= len) {  /* the constraints fix the row: its constraint space is {0} */
            for (int q = 0; q < len; q++) val[s + q] = 0.0;
        } else {
            for (int a = 0; a < k; a++) {
                c[a] = 0.0;
                for (int q = 0; q < len; q++) c[a] += val[s + q] * U[q * k + a];
            }
            for (int q = 0; q < len; q++) {
                double u = 0.0;
                for (int a = 0; a < k; a++) u += c[a] * U[q * k + a];
                val[s + q] = val[s + q] - u;
            }
        }
    } else {
        double r[ORC_KMAX];
        for (int b = 0; b < k; b++) {
            r[b] = target[b];
            for (int q = 0; q < len; q++) r[b] = r[b] - val[s + q] * M[q * k + b];
        }
        for (int a = 0; a < k; a++) {
            c[a] = 0.0;
            for (int b = 0; b < k; b++) c[a] += r[b] * VS[b * k + a];
        }
        for (int q = 0; q < len; q++) {
            double u = 0.0;
            for (int a = 0; a < k; a++) u += c[a] * U[q * k + a];
            val[s + q] = val[s + q] + u;
        }
    }
    if (M != Ms) { free(M); free(U); }
}

void orc_smooth_candidates_k(const orc_csr *A, double *B, int k, int sweeps, double omega) {
    if (k == 1) { orc_smooth_candidates(A, B, sweeps, omega); return; }
    int32_t n = A->nrows;
    double *col = (double *)orc_xmalloc((size_t)n * sizeof(double));
    for (int c = 0; c < k; c++) {  /* each column as the single-candidate case */
        for (int32_t i = 0; i < n; i++) col[i] = B[(size_t)i * k + c];
        orc_smooth_candidates(A, col, sweeps, omega);
        for (int32_t i = 0; i < n; i++) B[(size_t)i * k + c] = col[i];
    }
    free(col);
}

/* T for k candidates: Bc = B(roots, :); the first candidate is injected as
 * for k = 1 (root rows exactly 1), then every free row is fitted, (t + u) Bc_J
 * = B_i, on its pattern (eq. Tproj); root rows keep the identity and
 * unaggregated rows stay zero. */
int orc_tentative_k(orc_csr *N, const int32_t *agg, const int32_t *roots, const int32_t *rowtype, const double *B,
                    int k, double *Bc) {
    if (k == 1) return orc_tentative(N, agg, roots, B, Bc);
    if (k > ORC_KMAX) return ORC_EINVAL;
    for (int32_t c = 0; c < N->ncols; c++) {
        for (int a = 0; a < k; a++) Bc[(size_t)c * k + a] = B[(size_t)roots[c] * k + a];
        if (fabs(Bc[(size_t)c * k]) < 1e-300) return ORC_EINVAL;
    }
    for (int32_t i = 0; i < N->nrows; i++) {
        for (int32_t e = N->rowptr[i]; e < N->rowptr[i + 1]; e++) {
            int32_t j = N->col[e];
            N->val[e] = (j == agg[i]) ? B[(size_t)i * k] / Bc[(size_t)j * k] : 0.0;
        }
        if (rowtype[i] == ORC_FREE)
            row_fit_k(N->rowptr[i], N->rowptr[i + 1], N->col, N->val, B + (size_t)i * k, Bc, k);
    }
    return ORC_OK;
}

void orc_project_k(orc_csr *W, const int32_t *rowtype, const double *Bc, int k) {
    if (k == 1) { orc_project(W, rowtype, Bc); return; }
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < W->nrows; i++) {
        int32_t s = W->rowptr[i], e = W->rowptr[i + 1];
        if (rowtype[i] != ORC_FREE || e - s == 1) {
            for (int32_t q = s; q < e; q++) W->val[q] = 0.0;
            continue;
        }
        row_fit_k(s, e, W->col, W->val, NULL, Bc, k);
    }
}

void orc_enforce_k(orc_csr *P, const int32_t *rowtype, const double *B, const double *Bc, int k) {
    if (k == 1) { orc_enforce(P, rowtype, B, Bc); return; }
    for (int32_t i = 0; i < P->nrows; i++)
        if (rowtype[i] == ORC_FREE)
            row_fit_k(P->rowptr[i], P->rowptr[i + 1], P->col, P->val, B + (size_t)i * k, Bc, k);
}

static double frob_dot(const orc_csr *X, const double *a, const double *b) {
    return orc_dot(X->nnz, a, b);
}

static double *row_diag(const orc_csr *A) {
    double *d = (double *)orc_xmalloc((size_t)A->nrows * sizeof(double));
    for (int32_t i = 0; i < A->nrows; i++) {
        d[i] = 0.0;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++)
            if (A->col[e] == i) d[i] = A->val[e];
    }
    return d;
}

/* energy trace(P^T A P) = <P, Mask_N(A P)>_F, since P vanishes off N */
static double pattern_energy(const orc_csr *A, const orc_csr *P) {
    orc_csr W;
    orc_csr_copy(P, &W);
    orc_masked_product(A, P, &W);
    double e = frob_dot(P, P->val, W.val);
    orc_csr_free(&W);
    return e;
}

/*
 * CG energy minimisation (Sec. 3.6 'improve', Sec. 4.1 Lemma th:cg): minimise
 * trace(P^T A P) = sum of the squared A-norms of the columns of P over the
 * fixed pattern N, with root rows fixed to the identity and P Bc = B held by
 * the row projection.  Reading: the algorithm itself is deferred to a cited
 * report; we run preconditioned CG in the Frobenius inner product on the
 * constraint space, with the operator X -> Proj(Mask_N(A X)), started from
 * P = T, preconditioned by the row scaling D^{-1} (which commutes with the
 * row projection; precond = 0 disables it), formed once as the inverted
 * diagonal and applied as a product.
 * energy_trace (optional, sweeps+1 entries): energy before and after each sweep.
 */
int orc_energy_min_cg(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc,
                      int sweeps, int precond, double *energy_trace) {
    return orc_energy_min_cg_k(A, P, rowtype, Bc, 1, sweeps, precond, energy_trace);
}

int orc_energy_min_cg_k(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc, int k,
                        int sweeps, int precond, double *energy_trace) {
    int64_t nz = P->nnz;
    double *diag = row_diag(A);
    orc_csr W;
    orc_csr_copy(P, &W);
    double *R = (double *)orc_xmalloc((size_t)nz * sizeof(double));
    double *Z = (double *)orc_xmalloc((size_t)nz * sizeof(double));
    double *Dd = (double *)orc_xcalloc((size_t)nz, sizeof(double));
    orc_csr Dm = *P; /* Dd viewed on the pattern */
    Dm.val = Dd;
    int it_done = sweeps;
    /* the preconditioner D^{-1}: the inverted diagonal, applied as a product */
    double *dinv = (double *)orc_xmalloc((size_t)(P->nrows > 0 ? P->nrows : 1) * sizeof(double));
    for (int32_t i = 0; i < P->nrows; i++) dinv[i] = 1.0 / diag[i];
    if (energy_trace) energy_trace[0] = pattern_energy(A, P);
    orc_masked_product(A, P, &W);
    orc_project_k(&W, rowtype, Bc, k);
    for (int64_t q = 0; q < nz; q++) R[q] = -W.val[q];
    double rho_old = 0.0, rho0 = 0.0;
    for (int it = 0; it < sweeps; it++) {
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < P->nrows; i++)
            for (int32_t q = P->rowptr[i]; q < P->rowptr[i + 1]; q++)
                Z[q] = precond ? R[q] * dinv[i] : R[q];
        double rho = frob_dot(P, R, Z);
        if (it == 0) rho0 = rho;
        /* converged to rounding: further steps only amplify noise */
        if (rho == 0.0 || rho <= ORC_CG_STOP * rho0) { it_done = it; break; }
        if (it == 0) {
            for (int64_t q = 0; q < nz; q++) Dd[q] = Z[q];
        } else {
            double beta = rho / rho_old;
#pragma omp parallel for schedule(static)
            for (int64_t q = 0; q < nz; q++) Dd[q] = Z[q] + beta * Dd[q];
        }
        orc_masked_product(A, &Dm, &W);
        orc_project_k(&W, rowtype, Bc, k);
        double dw = frob_dot(P, Dd, W.val);
        if (dw <= 0.0) { it_done = it; break; }
        double alpha = rho / dw;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < nz; q++) {
            P->val[q] = P->val[q] + alpha * Dd[q];
            R[q] = R[q] - alpha * W.val[q];
        }
        rho_old = rho;
        if (energy_trace) energy_trace[it + 1] = pattern_energy(A, P);
    }
    if (energy_trace)
        for (int it = it_done; it < sweeps; it++) energy_trace[it + 1] = energy_trace[it_done];
    free(diag);
    free(dinv);
    free(R);
    free(Z);
    free(Dd);
    orc_csr_free(&W);
    return ORC_OK;
}

/*
 * GMRES energy minimisation for nonsymmetric A (Sec. 4.2, Sec. 5.3).
 * Reading: the paper cites fGMRES in the A*A norm from another report; we
 * take m Arnoldi steps (modified Gram-Schmidt in the Frobenius inner product,
 * no restart) for the operator X -> Proj(Mask_N(A X)) on the constraint space,
 * solving Proj(Mask_N(A (T + U))) = 0 for the correction U, i.e. U minimises
 * the pattern-restricted, projected residual ||Proj(Mask_N(A (T+U)))||_F over
 * the Krylov space.  Least squares by Givens rotations.  P <- T + V y.
 * res_trace (optional, m+1 entries): residual norms (initial, then per step).
 */
int orc_energy_min_gmres(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc,
                         int m, double *res_trace) {
    return orc_energy_min_gmres_k(A, P, rowtype, Bc, 1, m, res_trace);
}

int orc_energy_min_gmres_k(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc, int kc,
                           int m, double *res_trace) {
    int64_t nz = P->nnz;
    if (m <= 0) return ORC_OK;
    double **V = (double **)orc_xcalloc((size_t)m + 1, sizeof(double *));
    double *H = (double *)orc_xcalloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i*m+j] */
    double *cs = (double *)orc_xcalloc((size_t)m, sizeof(double));
    double *sn = (double *)orc_xcalloc((size_t)m, sizeof(double));
    double *g = (double *)orc_xcalloc((size_t)m + 1, sizeof(double));
    double *y = (double *)orc_xcalloc((size_t)m, sizeof(double));
    orc_csr W, Vm;
    orc_csr_copy(P, &W);
    Vm = *P;
    orc_masked_product(A, P, &W);
    orc_project_k(&W, rowtype, Bc, kc);
    V[0] = (double *)orc_xmalloc((size_t)nz * sizeof(double));
    for (int64_t q = 0; q < nz; q++) V[0][q] = -W.val[q];
    double beta = sqrt(frob_dot(P, V[0], V[0]));
    if (res_trace) for (int j = 0; j <= m; j++) res_trace[j] = beta;
    int k = 0;
    if (beta > 0.0) {
        for (int64_t q = 0; q < nz; q++) V[0][q] = V[0][q] / beta;
        g[0] = beta;
        for (int j = 0; j < m; j++) {
            Vm.val = V[j];
            orc_masked_product(A, &Vm, &W);
            orc_project_k(&W, rowtype, Bc, kc);
            for (int i = 0; i <= j; i++) {
                double hij = frob_dot(P, W.val, V[i]);
                H[i * m + j] = hij;
                for (int64_t q = 0; q < nz; q++) W.val[q] = W.val[q] - hij * V[i][q];
            }
            double hn = sqrt(frob_dot(P, W.val, W.val));
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; i++) {
                double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
            if (den == 0.0) break;
            cs[j] = H[j * m + j] / den;
            sn[j] = H[(j + 1) * m + j] / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            if (res_trace) for (int jj = j + 1; jj <= m; jj++) res_trace[jj] = fabs(g[j + 1]);
            if (hn <= ORC_GMRES_BREAK * beta) break;
            V[j + 1] = (double *)orc_xmalloc((size_t)nz * sizeof(double));
            for (int64_t q = 0; q < nz; q++) V[j + 1][q] = W.val[q] / hn;
        }
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int j = i + 1; j < k; j++) s -= H[i * m + j] * y[j];
            y[i] = s / H[i * m + i];
        }
        for (int j = 0; j < k; j++)
            for (int64_t q = 0; q < nz; q++) P->val[q] = P->val[q] + y[j] * V[j][q];
    }
    for (int j = 0; j <= m; j++) free(V[j]);
    free(V); free(H); free(cs); free(sn); free(g); free(y);
    orc_csr_free(&W);
    return ORC_OK;
}

/*
 * Post-filter (Sec. 3.7, Alg. 4 with drop tolerance theta): on free rows keep
 * |P_ij| >= theta * max_j |P_ij| (guard band) and always the row's own
 * aggregate; root rows keep their single entry; unaggregated rows stay empty.
 * near_ties counts dropped-or-kept entries within 1e-9 relative of the
 * threshold (P values agree with the GPU only to ~1e-12, so such entries
 * could decide differently).
 */
int orc_postfilter(const orc_csr *P, const int32_t *agg, const int32_t *rowtype, double theta,
                   orc_csr *Pf, int64_t *near_ties) {
    return orc_postfilter_m(P, agg, rowtype, theta, 1, Pf, near_ties);
}

/* m > 1: the row's own aggregate is the block of columns m agg .. m agg + m - 1 */
int orc_postfilter_m(const orc_csr *P, const int32_t *agg, const int32_t *rowtype, double theta, int mb,
                     orc_csr *Pf, int64_t *near_ties) {
    int32_t n = P->nrows;
    char *keep = (char *)orc_xcalloc((size_t)P->nnz, 1);
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    int64_t ties = 0;
    for (int32_t i = 0; i < n; i++) {
        int32_t cnt = 0;
        if (rowtype[i] == ORC_FREE) {
            double m = 0.0;
            for (int32_t e = P->rowptr[i]; e < P->rowptr[i + 1]; e++)
                if (fabs(P->val[e]) > m) m = fabs(P->val[e]);
            double thr = theta * m * (1.0 - ORC_GUARD);
            double ref = theta * m;
            for (int32_t e = P->rowptr[i]; e < P->rowptr[i + 1]; e++) {
                int own = (P->col[e] / mb == agg[i]);
                int k = (fabs(P->val[e]) >= thr) || own;
                if (!own && fabs(fabs(P->val[e]) - ref) < 1e-9 * ref) ties++;
                keep[e] = (char)k;
                cnt += k;
            }
        } else {
            for (int32_t e = P->rowptr[i]; e < P->rowptr[i + 1]; e++) { keep[e] = 1; cnt++; }
        }
        rowptr[i + 1] = rowptr[i] + cnt;
    }
    Pf->nrows = n;
    Pf->ncols = P->ncols;
    Pf->nnz = rowptr[n];
    Pf->rowptr = rowptr;
    Pf->col = (int32_t *)orc_xmalloc((size_t)Pf->nnz * sizeof(int32_t));
    Pf->val = (double *)orc_xmalloc((size_t)Pf->nnz * sizeof(double));
    int64_t dst = 0;
    for (int64_t e = 0; e < P->nnz; e++)
        if (keep[e]) { Pf->col[dst] = P->col[e]; Pf->val[dst] = P->val[e]; dst++; }
    free(keep);
    if (near_ties) *near_ties += ties;
    return ORC_OK;
}

/*
 * enforce (Alg. 3, eq. Tproj): minimal-norm least-squares update of each free
 * row on its pattern so that (t + u) Bc = B_i:  u = (B_i - t.b) b / (b.b).
 */
void orc_enforce(orc_csr *P, const int32_t *rowtype, const double *B, const double *Bc) {
    for (int32_t i = 0; i < P->nrows; i++) {
        if (rowtype[i] != ORC_FREE) continue;
        double tb = 0.0, bb = 0.0;
        for (int32_t e = P->rowptr[i]; e < P->rowptr[i + 1]; e++) {
            double b = Bc[P->col[e]];
            tb += P->val[e] * b;
            bb += b * b;
        }
        double c = (B[i] - tb) / bb;
        for (int32_t e = P->rowptr[i]; e < P->rowptr[i + 1]; e++)
            P->val[e] = P->val[e] + c * Bc[P->col[e]];
    }
}

/* ------------------------------------------------------------------------ */
/* Systems (Sec. 3.2 amalgamate, Sec. 3.4 unamalgamate, Sec. 3.6 eq.
 * root-nodeform for m > 1): unknowns node-major, m per node. */

/* S_m(I, J) = the largest entry of S's m x m block (I, J), over the entries
 * S stores; columns ascending. */
int orc_amalgamate(const orc_csr *S, int m, orc_csr *Sm) {
    int32_t nn = S->nrows / m;
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)nn + 1, sizeof(int32_t));
    double *acc = (double *)orc_xmalloc((size_t)nn * sizeof(double));
    char *seen = (char *)orc_xcalloc((size_t)nn, 1);
    int32_t *list = (int32_t *)orc_xmalloc((size_t)nn * sizeof(int32_t));
    /* pass 1: count */
    for (int32_t I = 0; I < nn; I++) {
        int32_t cnt = 0;
        for (int32_t i = I * m; i < I * m + m; i++)
            for (int32_t e = S->rowptr[i]; e < S->rowptr[i + 1]; e++) {
                int32_t J = S->col[e] / m;
                if (!seen[J]) { seen[J] = 1; list[cnt++] = J; }
            }
        for (int32_t q = 0; q < cnt; q++) seen[list[q]] = 0;
        rowptr[I + 1] = rowptr[I] + cnt;
    }
    Sm->nrows = Sm->ncols = nn;
    Sm->nnz = rowptr[nn];
    Sm->rowptr = rowptr;
    Sm->col = (int32_t *)orc_xmalloc((size_t)(Sm->nnz > 0 ? Sm->nnz : 1) * sizeof(int32_t));
    Sm->val = (double *)orc_xmalloc((size_t)(Sm->nnz > 0 ? Sm->nnz : 1) * sizeof(double));
    /* pass 2: block maxima, columns sorted */
    for (int32_t I = 0; I < nn; I++) {
        int32_t cnt = 0;
        for (int32_t i = I * m; i < I * m + m; i++)
            for (int32_t e = S->rowptr[i]; e < S->rowptr[i + 1]; e++) {
                int32_t J = S->col[e] / m;
                if (!seen[J]) { seen[J] = 1; acc[J] = S->val[e]; list[cnt++] = J; }
                else if (S->val[e] > acc[J]) acc[J] = S->val[e];
            }
        for (int32_t a = 1; a < cnt; a++) { /* insertion sort of the row's columns */
            int32_t x = list[a], b = a - 1;
            while (b >= 0 && list[b] > x) { list[b + 1] = list[b]; b--; }
            list[b + 1] = x;
        }
        for (int32_t q = 0; q < cnt; q++) {
            Sm->col[rowptr[I] + q] = list[q];
            Sm->val[rowptr[I] + q] = acc[list[q]];
            seen[list[q]] = 0;
        }
    }
    free(acc); free(seen); free(list);
    return ORC_OK;
}

/* N(i, m J + c) = N_m(floor(i/m), J) for c < m; root rows become identity
 * rows: root unknown i of aggregate a has the single entry (i, m a + i mod m). */
int orc_unamalgamate_pattern(const orc_csr *Nm, int m, const int32_t *agg, const int32_t *rowtype, orc_csr *N) {
    int32_t n = Nm->nrows * m;
    int32_t *rowptr = (int32_t *)orc_xcalloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t i = 0; i < n; i++) {
        int32_t I = i / m;
        int32_t cnt = rowtype[i] == ORC_ROOT ? 1 : m * (Nm->rowptr[I + 1] - Nm->rowptr[I]);
        rowptr[i + 1] = rowptr[i] + cnt;
    }
    N->nrows = n;
    N->ncols = Nm->ncols * m;
    N->nnz = rowptr[n];
    N->rowptr = rowptr;
    N->col = (int32_t *)orc_xmalloc((size_t)(N->nnz > 0 ? N->nnz : 1) * sizeof(int32_t));
    N->val = (double *)orc_xmalloc((size_t)(N->nnz > 0 ? N->nnz : 1) * sizeof(double));
    for (int32_t i = 0; i < n; i++) {
        int32_t I = i / m, dst = rowptr[i];
        if (rowtype[i] == ORC_ROOT) {
            N->col[dst] = m * agg[i] + i % m;
            N->val[dst] = 1.0;
            continue;
        }
        for (int32_t e = Nm->rowptr[I]; e < Nm->rowptr[I + 1]; e++)
            for (int c = 0; c < m; c++) {
                N->col[dst] = m * Nm->col[e] + c;
                N->val[dst++] = Nm->val[e];
            }
    }
    return ORC_OK;
}

/* T for block size m (eq. root-nodeform): Bc = B at the root unknowns; the
 * first m candidates are injected over each aggregate and normalised by the
 * root node's m x m block, T_i,(m a + .) = B_i,0:m Broot_a^{-1}, so root
 * rows are identity rows; candidates beyond m are then fitted row by row
 * (eq. Tproj).  agg is the node aggregate of every unknown, roots lists the
 * root unknowns (m per aggregate, m a + c at position m a + c). */
int orc_tentative_block(orc_csr *N, const int32_t *agg, const int32_t *roots, const int32_t *rowtype, const double *B,
                        int k, int m, double *Bc) {
    if (m > ORC_KMAX || k < m) return ORC_EINVAL;
    int32_t nc = N->ncols, na = nc / m;
    for (int32_t c = 0; c < nc; c++)
        for (int a = 0; a < k; a++) Bc[(size_t)c * k + a] = B[(size_t)roots[c] * k + a];
    double *Binv = (double *)orc_xmalloc((size_t)na * m * m * sizeof(double));
    for (int32_t a = 0; a < na; a++) { /* Gauss-Jordan with partial pivoting on the m x m root block */
        double M[ORC_KMAX * ORC_KMAX], X[ORC_KMAX * ORC_KMAX];
        double amax = 0.0;
        for (int r = 0; r < m; r++)
            for (int c = 0; c < m; c++) {
                M[r * m + c] = B[(size_t)roots[m * a + r] * k + c];
                X[r * m + c] = (r == c);
                if (fabs(M[r * m + c]) > amax) amax = fabs(M[r * m + c]);
            }
        for (int col = 0; col < m; col++) {
            int piv = col;
            for (int r = col + 1; r < m; r++) if (fabs(M[r * m + col]) > fabs(M[piv * m + col])) piv = r;
            if (!(fabs(M[piv * m + col]) > 1e-12 * amax)) { free(Binv); return ORC_EINVAL; }
            for (int c = 0; c < m; c++) {
                double t = M[col * m + c]; M[col * m + c] = M[piv * m + c]; M[piv * m + c] = t;
                t = X[col * m + c]; X[col * m + c] = X[piv * m + c]; X[piv * m + c] = t;
            }
            double d = M[col * m + col];
            for (int c = 0; c < m; c++) { M[col * m + c] = M[col * m + c] / d; X[col * m + c] = X[col * m + c] / d; }
            for (int r = 0; r < m; r++) {
                if (r == col) continue;
                double f = M[r * m + col];
                for (int c = 0; c < m; c++) {
                    M[r * m + c] = M[r * m + c] - f * M[col * m + c];
                    X[r * m + c] = X[r * m + c] - f * X[col * m + c];
                }
            }
        }
        memcpy(Binv + (size_t)a * m * m, X, (size_t)m * m * sizeof(double));
    }
    for (int32_t i = 0; i < N->nrows; i++) {
        int32_t s = N->rowptr[i], e = N->rowptr[i + 1];
        for (int32_t q = s; q < e; q++) N->val[q] = 0.0;
        if (agg[i] < 0) continue;
        int32_t a = agg[i];
        if (rowtype[i] == ORC_ROOT) {
            for (int32_t q = s; q < e; q++) N->val[q] = (N->col[q] == m * a + i % m) ? 1.0 : 0.0;
            continue;
        }
        const double *bi = B + (size_t)i * k, *Xi = Binv + (size_t)a * m * m;
        for (int32_t q = s; q < e; q++) {
            int32_t col = N->col[q];
            if (col / m != a) continue;
            int c = col % m;
            double t = 0.0;
            for (int r = 0; r < m; r++) t += bi[r] * Xi[r * m + c];
            N->val[q] = t;
        }
        if (k > m) row_fit_k(s, e, N->col, N->val, bi, Bc, k);
    }
    free(Binv);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Hierarchy */

int orc_hier_nlevels(const orc_hier *h) { return h->nlev; }
int64_t orc_hier_near_ties(const orc_hier *h) { return h->near_ties; }

const orc_csr *orc_hier_csr(const orc_hier *h, int lvl, int which) {
    if (lvl < 0 || lvl >= h->nlev) return NULL;
    const orc_level *L = &h->lev[lvl];
    switch (which) {
        case 0: return &L->A;
        case 1: return &L->S;
        case 2: return &L->N;
        case 3: return &L->T;
        case 4: return &L->P;
        case 5: return &L->R;
    }
    return NULL;
}

const int32_t *orc_hier_ivec(const orc_hier *h, int lvl, int which, int32_t *len) {
    if (lvl < 0 || lvl >= h->nlev) return NULL;
    const orc_level *L = &h->lev[lvl];
    switch (which) {
        case 0: *len = L->A.nrows; return L->agg;
        case 1: *len = L->nc; return L->roots;
        case 2: *len = L->A.nrows; return L->rowtype;
    }
    return NULL;
}

const double *orc_hier_dvec(const orc_hier *h, int lvl, int which, int32_t *len) {
    if (lvl < 0 || lvl >= h->nlev) return NULL;
    const orc_level *L = &h->lev[lvl];
    const int k = h->p.ncand > 0 ? h->p.ncand : 1;
    switch (which) {  /* row-major n x k / nc x k */
        case 0: *len = L->A.nrows * k; return L->B;
        case 1: *len = L->nc * k; return L->Bc;
        case 2: *len = L->A.nrows * k; return L->Bhat;
        case 3: *len = L->nc * k; return L->Bhatc;
    }
    return NULL;
}

static void level_free(orc_level *L) {
    orc_csr_free(&L->A); orc_csr_free(&L->S); orc_csr_free(&L->N); orc_csr_free(&L->T);
    orc_csr_free(&L->P); orc_csr_free(&L->R);
    free(L->agg); free(L->roots); free(L->rowtype);
    free(L->B); free(L->Bc); free(L->Bhat); free(L->Bhatc); free(L->diag);
    memset(L, 0, sizeof(*L));
}

void orc_hier_free(orc_hier *h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; l++) level_free(&h->lev[l]);
    free(h->lev);
    free(h->LU);
    free(h->piv);
    free(h);
}

/* energy minimisation of one operator (P for A, or R^T for A^T), steps of
 * Alg. 3: improve, then optionally filter, enforce, one more improve. */
static int build_transfer(const orc_csr *A, const orc_csr *N, const int32_t *agg, const int32_t *roots,
                          const int32_t *rowtype, const double *Bsm, const orc_params *p, orc_csr *Pout,
                          double *Bc, int64_t *near_ties) {
    const int k = p->ncand > 0 ? p->ncand : 1;
    const int mb = p->block_size > 0 ? p->block_size : 1;
    orc_csr P;
    orc_csr_copy(N, &P);
    int rc = mb > 1 ? orc_tentative_block(&P, agg, roots, rowtype, Bsm, k, mb, Bc)
                    : orc_tentative_k(&P, agg, roots, rowtype, Bsm, k, Bc);
    if (rc) { orc_csr_free(&P); return rc; }
    rc = (p->method == 0) ? orc_energy_min_cg_k(A, &P, rowtype, Bc, k, p->n_sweeps, p->precond, NULL)
                          : orc_energy_min_gmres_k(A, &P, rowtype, Bc, k, p->n_sweeps, NULL);
    if (rc) { orc_csr_free(&P); return rc; }
    if (p->postfilter > 0.0) {
        orc_csr Pf;
        orc_postfilter_m(&P, agg, rowtype, p->postfilter, mb, &Pf, near_ties);
        orc_csr_free(&P);
        orc_enforce_k(&Pf, rowtype, Bsm, Bc, k);
        rc = (p->method == 0) ? orc_energy_min_cg_k(A, &Pf, rowtype, Bc, k, 1, p->precond, NULL)
                              : orc_energy_min_gmres_k(A, &Pf, rowtype, Bc, k, 1, NULL);
        P = Pf;
    }
    *Pout = P;
    return rc;
}

#define ORC_MAX_DENSE 4096

/* Alg. 3 root_node_setup. */
int orc_setup(const orc_csr *A0, const double *B0, const double *Bhat0, const orc_params *p, orc_hier **out) {
    *out = NULL;
    if (A0->nrows != A0->ncols || A0->nrows <= 0) return ORC_EINVAL;
    if (!p->symmetric && !Bhat0) return ORC_EINVAL;
    orc_hier *h = (orc_hier *)orc_xcalloc(1, sizeof(orc_hier));
    h->p = *p;
    int cap = p->max_levels > 0 ? p->max_levels : 1;
    h->lev = (orc_level *)orc_xcalloc((size_t)cap, sizeof(orc_level));
    const int k = p->ncand > 0 ? p->ncand : 1;
    const int mb = p->block_size > 0 ? p->block_size : 1;
    if (k > ORC_KMAX || k < mb || A0->nrows % mb != 0) { free(h->lev); free(h); return ORC_EINVAL; }
    orc_level *L = &h->lev[0];
    orc_csr_copy(A0, &L->A);
    int32_t n = A0->nrows;
    L->B = (double *)orc_xmalloc((size_t)n * k * sizeof(double));
    memcpy(L->B, B0, (size_t)n * k * sizeof(double));
    if (!p->symmetric) {
        L->Bhat = (double *)orc_xmalloc((size_t)n * k * sizeof(double));
        memcpy(L->Bhat, Bhat0, (size_t)n * k * sizeof(double));
    }
    int lvl = 0;
    int rc = ORC_OK;
    while (h->lev[lvl].A.nrows > p->max_coarse && lvl < cap - 1) {
        L = &h->lev[lvl];
        n = L->A.nrows;
        L->diag = row_diag(&L->A);
        double theta = (lvl > 0 && p->soc_theta_coarse >= 0.0) ? p->soc_theta_coarse : p->soc_theta;
        rc = p->soc_kind == 1 ? orc_strength_classical(&L->A, theta, &L->S)     /* strength */
                              : orc_strength(&L->A, theta, &L->S);
        if (rc) break;
        L->agg = (int32_t *)orc_xmalloc((size_t)n * sizeof(int32_t));
        orc_csr Sm = {0};
        int32_t *aggm = NULL, *rootsm = NULL, ncm = 0;
        if (mb > 1) {                                                            /* amalgamate */
            orc_amalgamate(&L->S, mb, &Sm);
            aggm = (int32_t *)orc_xmalloc((size_t)(n / mb) * sizeof(int32_t));
            rc = orc_aggregate(&Sm, p->seed + (uint64_t)lvl, aggm, &rootsm, &ncm);
            if (rc) { orc_csr_free(&Sm); free(aggm); free(rootsm); break; }
            for (int32_t i = 0; i < n; i++) L->agg[i] = aggm[i / mb];          /* unamalgamate */
            L->nc = mb * ncm;
            L->roots = (int32_t *)orc_xmalloc((size_t)(L->nc > 0 ? L->nc : 1) * sizeof(int32_t));
            for (int32_t r = 0; r < ncm; r++)
                for (int c = 0; c < mb; c++) L->roots[mb * r + c] = mb * rootsm[r] + c;
        } else {
            rc = orc_aggregate(&L->S, p->seed + (uint64_t)lvl, L->agg, &L->roots, &L->nc); /* aggregate */
            if (rc) break;
        }
        if (L->nc == 0 || L->nc >= n) {                                          /* stalled */
            free(L->agg); free(L->roots); L->agg = L->roots = NULL; L->nc = 0;
            orc_csr_free(&L->S);
            if (mb > 1) { orc_csr_free(&Sm); free(aggm); free(rootsm); }
            break;
        }
        L->rowtype = (int32_t *)orc_xmalloc((size_t)n * sizeof(int32_t));
        orc_row_types(n, L->agg, L->roots, L->nc, L->rowtype);
        if (mb > 1) {                            /* N = S_m^d C on nodes, then on unknowns */
            orc_csr Nm;
            rc = orc_pattern(&Sm, aggm, rootsm, ncm, p->degree, p->prefilter, &Nm);
            orc_csr_free(&Sm); free(aggm); free(rootsm);
            if (rc) break;
            rc = orc_unamalgamate_pattern(&Nm, mb, L->agg, L->rowtype, &L->N);
            orc_csr_free(&Nm);
        } else {
            rc = orc_pattern(&L->S, L->agg, L->roots, L->nc, p->degree, p->prefilter, &L->N); /* N = S^d C */
        }
        if (rc) break;
        orc_smooth_candidates_k(&L->A, L->B, k, p->b_sweeps, p->omega);        /* smooth(A, B) */
        L->Bc = (double *)orc_xmalloc((size_t)L->nc * k * sizeof(double));
        orc_csr_copy(&L->N, &L->T);
        rc = mb > 1 ? orc_tentative_block(&L->T, L->agg, L->roots, L->rowtype, L->B, k, mb, L->Bc)
                    : orc_tentative_k(&L->T, L->agg, L->roots, L->rowtype, L->B, k, L->Bc); /* inject */
        if (rc) break;
        rc = build_transfer(&L->A, &L->N, L->agg, L->roots, L->rowtype, L->B, p, &L->P, L->Bc,
                            &h->near_ties);                                      /* improve (+filter) */
        if (rc) break;
        if (p->symmetric) {
            orc_transpose(&L->P, &L->R);                                         /* R = P^T */
        } else {
            orc_csr At, Rt;
            orc_transpose(&L->A, &At);
            orc_smooth_candidates_k(&At, L->Bhat, k, p->b_sweeps, p->omega);
            L->Bhatc = (double *)orc_xmalloc((size_t)L->nc * k * sizeof(double));
            rc = build_transfer(&At, &L->N, L->agg, L->roots, L->rowtype, L->Bhat, p, &Rt, L->Bhatc,
                                &h->near_ties);
            orc_csr_free(&At);
            if (rc) break;
            orc_transpose(&Rt, &L->R);
            orc_csr_free(&Rt);
        }
        orc_csr AP;                                                              /* A_c = R A P */
        rc = orc_spgemm(&L->A, &L->P, &AP);
        if (rc) break;
        orc_level *Lc = &h->lev[lvl + 1];
        rc = orc_spgemm(&L->R, &AP, &Lc->A);
        orc_csr_free(&AP);
        if (rc) break;
        Lc->B = (double *)orc_xmalloc((size_t)L->nc * k * sizeof(double));
        memcpy(Lc->B, L->Bc, (size_t)L->nc * k * sizeof(double));
        if (!p->symmetric) {
            Lc->Bhat = (double *)orc_xmalloc((size_t)L->nc * k * sizeof(double));
            memcpy(Lc->Bhat, L->Bhatc, (size_t)L->nc * k * sizeof(double));
        }
        lvl++;
    }
    if (rc) { h->nlev = lvl + 1; orc_hier_free(h); return rc; }
    h->nlev = lvl + 1;
    L = &h->lev[lvl];
    if (!L->diag) L->diag = row_diag(&L->A);
    int32_t nL = L->A.nrows;
    if (nL > ORC_MAX_DENSE) { orc_hier_free(h); return ORC_ESTALL; }
    h->ncoarse = nL;
    h->LU = (double *)orc_xcalloc((size_t)nL * (size_t)nL, sizeof(double));
    h->piv = (int32_t *)orc_xmalloc((size_t)(nL > 0 ? nL : 1) * sizeof(int32_t));
    for (int32_t i = 0; i < nL; i++)
        for (int32_t e = L->A.rowptr[i]; e < L->A.rowptr[i + 1]; e++)
            h->LU[(size_t)i * nL + L->A.col[e]] = L->A.val[e];
    rc = orc_lu_factor(nL, h->LU, h->piv);
    if (rc) { orc_hier_free(h); return rc; }
    *out = h;
    return ORC_OK;
}

