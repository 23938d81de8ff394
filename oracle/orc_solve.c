/*
 * orc_solve.c - coarsest-grid LU, V(nu_pre, nu_post) cycle and the outer
 * iterations of the CPU oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Cycle (Sec. 2, two-grid description and eq. twogrid, applied recursively):
 *   x <- x + omega D^{-1} (b - A x)       nu_pre times
 *   gamma times (V-cycle 1, W-cycle 2; once when the next level is the
 *   coarsest, whose exact solve leaves R (b - A x) = 0 for a second pass):
 *     r  = b - A x;  b_c = R r
 *     x_c = 0; recurse (coarsest: dense LU solve)
 *     x <- x + P x_c
 *   x <- x + omega D^{-1} (b - A x)       nu_post times
 * Outer: 0 stationary cycling, 1 CG preconditioned by one cycle, 2 GMRES(m)
 * right-preconditioned by one cycle (flexible form, Saad 1993, which equals
 * ordinary right preconditioning for a fixed cycle).  Stop on
 * ||b - A x|| / ||b|| < tol (Sec. 5 opening: relative residual 1e-8).
 */
#include <math.h>
#include <stdint.h>
#include "orc_internal.h"

/* Dense LU with partial pivoting (largest |pivot|, lowest row on ties),
 * row-major n x n in place.  A pivot below 1e-14 max|A| is singular. */
int orc_lu_factor(int n, double *LU, int32_t *piv) {
    double amax = 0.0;
    for (int64_t q = 0; q < (int64_t)n * n; q++)
        if (fabs(LU[q]) > amax) amax = fabs(LU[q]);
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(LU[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(LU[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best >= 1e-14 * amax) || best == 0.0) return ORC_ESINGULAR;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = LU[(size_t)k * n + j];
                LU[(size_t)k * n + j] = LU[(size_t)p * n + j];
                LU[(size_t)p * n + j] = t;
            }
        double d = LU[(size_t)k * n + k];
        for (int i = k + 1; i < n; i++) {
            double l = LU[(size_t)i * n + k] / d;
            LU[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++) LU[(size_t)i * n + j] = LU[(size_t)i * n + j] - l * LU[(size_t)k * n + j];
        }
    }
    return ORC_OK;
}

void orc_lu_solve(int n, const double *LU, const int32_t *piv, double *x) {
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < n; i++) {
        double s = x[i];
        for (int j = 0; j < i; j++) s = s - LU[(size_t)i * n + j] * x[j];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int j = i + 1; j < n; j++) s = s - LU[(size_t)i * n + j] * x[j];
        x[i] = s / LU[(size_t)i * n + i];
    }
}

static void jacobi(const orc_csr *A, const double *diag, const double *b, double *x, double omega, double *tmp) {
    orc_spmv(A, x, tmp);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < A->nrows; i++) x[i] = x[i] + omega * ((b[i] - tmp[i]) / diag[i]);
}

void orc_vcycle(const orc_hier *h, int lvl, const double *b, double *x) {
    const orc_level *L = &h->lev[lvl];
    int32_t n = L->A.nrows;
    if (lvl == h->nlev - 1) {
        memcpy(x, b, (size_t)n * sizeof(double));
        orc_lu_solve(n, h->LU, h->piv, x);
        return;
    }
    double *tmp = (double *)orc_xmalloc((size_t)n * sizeof(double));
    for (int s = 0; s < h->p.nu_pre; s++) jacobi(&L->A, L->diag, b, x, h->p.omega, tmp);
    int32_t nc = L->nc;
    double *bc = (double *)orc_xmalloc((size_t)nc * sizeof(double));
    double *xc = (double *)orc_xmalloc((size_t)nc * sizeof(double));
    const int passes = (lvl + 1 == h->nlev - 1 || h->p.gamma < 1) ? 1 : h->p.gamma;
    for (int c = 0; c < passes; c++) {
        orc_spmv(&L->A, x, tmp);
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; i++) tmp[i] = b[i] - tmp[i];
        orc_spmv(&L->R, tmp, bc);
        memset(xc, 0, (size_t)nc * sizeof(double));
        orc_vcycle(h, lvl + 1, bc, xc);
        orc_spmv(&L->P, xc, tmp);
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; i++) x[i] = x[i] + tmp[i];
    }
    for (int s = 0; s < h->p.nu_post; s++) jacobi(&L->A, L->diag, b, x, h->p.omega, tmp);
    free(bc);
    free(xc);
    free(tmp);
}

static double residual(const orc_csr *A, const double *b, const double *x, double *r) {
    orc_spmv(A, x, r);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < A->nrows; i++) r[i] = b[i] - r[i];
    return orc_nrm2(A->nrows, r);
}

int orc_solve(const orc_hier *h, const double *b, double *x, double tol, int maxit, int outer, int restart,
              orc_solve_info *info) {
    const orc_csr *A = &h->lev[0].A;
    int32_t n = A->nrows;
    double *r = (double *)orc_xmalloc((size_t)n * sizeof(double));
    double nb = orc_nrm2(n, b);
    if (nb == 0.0) nb = 1.0;
    double r0 = residual(A, b, x, r), rn = r0;
    int it = 0, status = ORC_ENOTCONV;
    if (r0 / nb < tol) status = ORC_OK;
    if (status != ORC_OK && outer == 0) {
        for (it = 1; it <= maxit; it++) {
            orc_vcycle(h, 0, b, x);
            rn = residual(A, b, x, r);
            if (rn / nb < tol) { status = ORC_OK; break; }
        }
        if (it > maxit) it = maxit;
    } else if (status != ORC_OK && outer == 1) {
        double *z = (double *)orc_xcalloc((size_t)n, sizeof(double));
        double *p = (double *)orc_xmalloc((size_t)n * sizeof(double));
        double *q = (double *)orc_xmalloc((size_t)n * sizeof(double));
        orc_vcycle(h, 0, r, z);
        memcpy(p, z, (size_t)n * sizeof(double));
        double rz = orc_dot(n, r, z);
        for (it = 1; it <= maxit; it++) {
            orc_spmv(A, p, q);
            double alpha = rz / orc_dot(n, p, q);
#pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; i++) {
                x[i] = x[i] + alpha * p[i];
                r[i] = r[i] - alpha * q[i];
            }
            rn = orc_nrm2(n, r);
            if (rn / nb < tol) { status = ORC_OK; break; }
            memset(z, 0, (size_t)n * sizeof(double));
            orc_vcycle(h, 0, r, z);
            double rz_new = orc_dot(n, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
#pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        if (it > maxit) it = maxit;
        rn = residual(A, b, x, r);
        free(z); free(p); free(q);
    } else if (status != ORC_OK && outer == 2) {
        int m = restart > 0 ? restart : 30;
        double *V = (double *)orc_xmalloc((size_t)(m + 1) * (size_t)n * sizeof(double));
        double *Z = (double *)orc_xmalloc((size_t)m * (size_t)n * sizeof(double));
        double *H = (double *)orc_xcalloc((size_t)(m + 1) * (size_t)m, sizeof(double));
        double *cs = (double *)orc_xmalloc((size_t)m * sizeof(double));
        double *sn = (double *)orc_xmalloc((size_t)m * sizeof(double));
        double *g = (double *)orc_xmalloc(((size_t)m + 1) * sizeof(double));
        double *y = (double *)orc_xmalloc((size_t)m * sizeof(double));
        double *w = (double *)orc_xmalloc((size_t)n * sizeof(double));
        it = 0;
        while (it < maxit && status != ORC_OK) {
            double beta = residual(A, b, x, r);
            rn = beta;
            if (beta / nb < tol) { status = ORC_OK; break; }
            for (int32_t i = 0; i < n; i++) V[i] = r[i] / beta;
            memset(g, 0, ((size_t)m + 1) * sizeof(double));
            g[0] = beta;
            int k = 0;
            for (int j = 0; j < m && it < maxit; j++) {
                double *zj = Z + (size_t)j * n, *vj = V + (size_t)j * n;
                memset(zj, 0, (size_t)n * sizeof(double));
                orc_vcycle(h, 0, vj, zj);
                orc_spmv(A, zj, w);
                for (int i = 0; i <= j; i++) {
                    double hij = orc_dot(n, w, V + (size_t)i * n);
                    H[i * m + j] = hij;
                    for (int32_t t = 0; t < n; t++) w[t] = w[t] - hij * V[(size_t)i * n + t];
                }
                double hn = orc_nrm2(n, w);
                H[(j + 1) * m + j] = hn;
                for (int i = 0; i < j; i++) {
                    double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                    H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                    H[i * m + j] = t;
                }
                double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
                cs[j] = H[j * m + j] / den;
                sn[j] = H[(j + 1) * m + j] / den;
                H[j * m + j] = den;
                H[(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                it++;
                k = j + 1;
                if (fabs(g[j + 1]) / nb < tol || hn == 0.0) break;
                for (int32_t t = 0; t < n; t++) V[(size_t)(j + 1) * n + t] = w[t] / hn;
            }
            for (int i = k - 1; i >= 0; i--) {
                double s = g[i];
                for (int j = i + 1; j < k; j++) s -= H[i * m + j] * y[j];
                y[i] = s / H[i * m + i];
            }
            for (int j = 0; j < k; j++)
                for (int32_t t = 0; t < n; t++) x[t] = x[t] + y[j] * Z[(size_t)j * n + t];
            rn = residual(A, b, x, r);
            if (rn / nb < tol) status = ORC_OK;
        }
        free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(w);
    } else if (status != ORC_OK) {
        free(r);
        return ORC_EINVAL;
    }
    if (info) {
        info->iters = it;
        info->rel_res = rn / nb;
        info->rho = (it > 0 && r0 > 0.0) ? pow(rn / r0, 1.0 / it) : 0.0;
        info->status = status;
    }
    free(r);
    return status;
}
