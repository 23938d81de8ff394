/*
 * orc.h - plain, slow FP64 CPU oracle for root-node AMG (Manteuffel, Olson,
 * Schroder, Southworth, "A Root-Node Based Algebraic Multigrid Method").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no source, header, table or helper with the CUDA path.
 *
 * Every routine follows the paper's algorithm steps in order (Alg. 3 and the
 * subsections of Sec. 3), written with the simplest data structures: CSR
 * matrices, a dense sparse-accumulator per row, sequential loops, and sums in
 * ascending index order.  Compiled with -ffp-contract=off so a*b+c is always
 * a rounded multiply followed by a rounded add.
 *
 * Readings of the paper (where it is silent or garbled) are stated beside the
 * routine that takes them.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

enum {
    ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ESINGULAR = 3, ORC_ESTALL = 4,
    ORC_ENOTCONV = 5, ORC_EINTERNAL = 8
};

/* CSR with int32 indices, sorted unique columns per row. */
typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;
    int32_t *rowptr; /* nrows+1 */
    int32_t *col;    /* nnz */
    double *val;     /* nnz (may be NULL for a pure pattern) */
} orc_csr;

typedef struct {
    double soc_theta;  /* symmetric strength drop tolerance theta */
    int degree;        /* d in N = S^d C */
    int n_sweeps;      /* energy-minimisation iterations */
    int method;        /* 0 = CG (SPD), 1 = GMRES (nonsymmetric) */
    double prefilter;  /* theta_pre (<= 0: off) */
    double postfilter; /* theta_post (<= 0: off) */
    int max_coarse;    /* stop coarsening at n <= max_coarse */
    int max_levels;
    int b_sweeps;      /* candidate relaxation sweeps */
    double omega;      /* weighted-Jacobi weight */
    uint64_t seed;     /* aggregation priority seed */
    int symmetric;     /* 1: R = P^T */
    int nu_pre, nu_post;
    int precond;       /* 1: Jacobi-preconditioned CG energy minimisation */
    double soc_theta_coarse; /* strength theta on levels >= 1 (< 0: same as soc_theta) */
    int gamma;         /* coarse-grid corrections per level: 1 V-cycle, 2 W-cycle */
    int soc_kind;      /* 0 symmetric strength, 1 classical strength */
    int ncand;         /* k, the number of candidate vectors (B is n x k, row-major) */
    int block_size;    /* m, unknowns per node (node-major; 1 = scalar problem) */
} orc_params;

/* Row classes of the interpolation pattern. */
enum { ORC_FREE = 0, ORC_ROOT = 1, ORC_UNAGG = 2 };

typedef struct orc_level orc_level;
typedef struct orc_hier orc_hier;

typedef struct {
    int iters;
    double rel_res;
    double rho;
    int status;
} orc_solve_info;

/* ---- memory ---- */
void orc_csr_free(orc_csr *a);
void orc_free(void *p);
/* OpenMP threads of the oracle's row loops (results do not depend on it) */
void orc_set_threads(int n);
int orc_get_threads(void);

/* ---- setup steps (each exported for pin tests) ---- */
int orc_strength(const orc_csr *A, double theta, orc_csr *S);
int orc_strength_classical(const orc_csr *A, double theta, orc_csr *S);
int orc_aggregate(const orc_csr *S, uint64_t seed, int32_t *agg, int32_t **roots, int32_t *nc);
uint64_t orc_splitmix64(uint64_t x);
void orc_smooth_candidates(const orc_csr *A, double *B, int sweeps, double omega);
int orc_pattern(const orc_csr *S, const int32_t *agg, const int32_t *roots, int32_t nc, int d,
                double theta_pre, orc_csr *N);
void orc_row_types(int32_t n, const int32_t *agg, const int32_t *roots, int32_t nc, int32_t *rowtype);
int orc_tentative(orc_csr *N, const int32_t *agg, const int32_t *roots, const double *B, double *Bc);
/* k candidates: B n x k, Bc nc x k (row-major) */
void orc_smooth_candidates_k(const orc_csr *A, double *B, int k, int sweeps, double omega);
int orc_tentative_k(orc_csr *N, const int32_t *agg, const int32_t *roots, const int32_t *rowtype, const double *B,
                    int k, double *Bc);
void orc_project_k(orc_csr *W, const int32_t *rowtype, const double *Bc, int k);
void orc_enforce_k(orc_csr *P, const int32_t *rowtype, const double *B, const double *Bc, int k);
int orc_energy_min_cg_k(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc, int k,
                        int sweeps, int precond, double *energy_trace);
int orc_energy_min_gmres_k(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc, int k,
                           int m, double *res_trace);
/* one-sided Jacobi SVD of a row's len x k Bc_J: U (len x k), V Sigma^+ (k x k); returns the rank kept */
int orc_row_svd(int len, int k, const double *M, double *U, double *VS);
/* systems (block size m > 1) */
int orc_amalgamate(const orc_csr *S, int m, orc_csr *Sm);
int orc_postfilter_m(const orc_csr *P, const int32_t *agg, const int32_t *rowtype, double theta, int mb,
                     orc_csr *Pf, int64_t *near_ties);
int orc_unamalgamate_pattern(const orc_csr *Nm, int m, const int32_t *agg, const int32_t *rowtype, orc_csr *N);
int orc_tentative_block(orc_csr *N, const int32_t *agg, const int32_t *roots, const int32_t *rowtype, const double *B,
                        int k, int m, double *Bc);
void orc_masked_product(const orc_csr *A, const orc_csr *X, orc_csr *W);
void orc_project(orc_csr *W, const int32_t *rowtype, const double *Bc);
int orc_energy_min_cg(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc,
                      int sweeps, int precond, double *energy_trace);
int orc_energy_min_gmres(const orc_csr *A, orc_csr *P, const int32_t *rowtype, const double *Bc,
                         int m, double *res_trace);
int orc_postfilter(const orc_csr *P, const int32_t *agg, const int32_t *rowtype, double theta,
                   orc_csr *Pf, int64_t *near_ties);
void orc_enforce(orc_csr *P, const int32_t *rowtype, const double *B, const double *Bc);
int orc_transpose(const orc_csr *A, orc_csr *At);
int orc_spgemm(const orc_csr *A, const orc_csr *B, orc_csr *C);
int orc_lu_factor(int n, double *LU, int32_t *piv);
void orc_lu_solve(int n, const double *LU, const int32_t *piv, double *x);

/* ---- full setup (Alg. 3) and solve ---- */
int orc_setup(const orc_csr *A, const double *B, const double *Bhat, const orc_params *p, orc_hier **out);
void orc_hier_free(orc_hier *h);
int orc_hier_nlevels(const orc_hier *h);
/* which: 0=A, 1=S, 2=N (pattern before energy-min, values of S^d C after pre-filter),
 *        3=T, 4=P, 5=R */
const orc_csr *orc_hier_csr(const orc_hier *h, int lvl, int which);
/* which: 0=agg (n), 1=roots (nc), 2=rowtype (n) */
const int32_t *orc_hier_ivec(const orc_hier *h, int lvl, int which, int32_t *len);
/* which: 0=B smoothed (n), 1=Bc (nc), 2=Bhat smoothed (n), 3=Bhat_c (nc) */
const double *orc_hier_dvec(const orc_hier *h, int lvl, int which, int32_t *len);
int64_t orc_hier_near_ties(const orc_hier *h);

void orc_vcycle(const orc_hier *h, int lvl, const double *b, double *x);
int orc_solve(const orc_hier *h, const double *b, double *x, double tol, int maxit, int outer, int restart,
              orc_solve_info *info);
#endif
