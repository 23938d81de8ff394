/*
 * rn.h - C ABI of the GB300 (sm_103a) root-node algebraic multigrid library.
 *
 * Method: Manteuffel, Olson, Schroder, Southworth, "A Root-Node Based
 * Algebraic Multigrid Method" (arXiv:1610.03154).  The library solves the
 * linear system A x = b of eq. linear-system (Sec. 1) with near-nullspace
 * candidates B (and B-hat for A^T when A is nonsymmetric, Sec. 3.1):
 *   rn_setup  builds the hierarchy of Alg. 3 (root_node_setup) on the GPU:
 *             strength (Sec. 3.2, eq. soc), seeded root-node aggregation
 *             (Sec. 3.3), pattern N = S^d C with pre-filter (Sec. 3.4-3.5,
 *             Alg. 4), tentative T (Sec. 3.6, eq. root-nodeform), constrained
 *             energy minimisation of P by CG or GMRES sweeps with the row-wise
 *             constraint projection (Sec. 3.6, eq. Tproj, Sec. 4 Lemma th:cg),
 *             post-filter + enforce + one re-sweep (Sec. 3.7), R = P^T or the
 *             same construction on A^T (Sec. 3.8), Galerkin A_c = R A P.
 *   rn_solve  runs V(nu_pre, nu_post) cycles with weighted Jacobi (Sec. 2,
 *             eq. twogrid) and a dense LU on the coarsest level, accelerated
 *             by CG or flexible GMRES, to a relative residual tolerance.
 *
 * Conventions (all entry points):
 *   - Status codes, never abort/exit.  rn_last_error() gives a thread-local
 *     message for the last failing call on the calling thread.
 *   - Matrices are CSR with int32 row pointers and column indices, columns
 *     sorted ascending and unique within each row, explicit nonzero diagonal,
 *     float64 values.  nnz must be < 2^31.
 *   - Location: pointers are device pointers when `location == RN_DEVICE`
 *     and ordinary host memory when `location == RN_HOST` (the library then
 *     copies the data in and the result out, inside the call).
 *   - Inputs are borrowed for the duration of the call only; rn_setup copies
 *     what it keeps.  The hierarchy is owned by the library until rn_free.
 *   - Device work runs on params.stream (a cudaStream_t; NULL means the
 *     legacy default stream).  Device memory comes from the caller's hooks
 *     (params.alloc / dealloc, e.g. torch's caching allocator) or, without
 *     them, from the stream-ordered allocator (cudaMallocAsync) on that
 *     stream.  rn_setup and rn_solve
 *     return after their last host read-back; outputs are complete when they
 *     return.
 *   - k (the number of candidates) is 1 <= k <= 4 (rn_setup); the batched
 *     and many-right-hand-side calls state their own limits.
 *   - One hierarchy must not be used by two threads at once.
 */
#ifndef RN_H
#define RN_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RN_OK = 0,
    RN_EINVAL = 1,      /* bad argument or malformed CSR (unsorted, no diagonal, zero root candidate) */
    RN_ENOMEM = 2,      /* device allocation failed */
    RN_ESINGULAR = 3,   /* coarsest-level LU met a pivot below 1e-14 max|A| */
    RN_ESTALL = 4,      /* coarsening stopped with more than 4096 rows left for the dense LU */
    RN_ENOTCONV = 5,    /* solve hit maxit before the tolerance (x holds the last iterate) */
    RN_ETIMEOUT = 6,    /* a bounded device loop (aggregation rounds) did not finish */
    RN_ECUDA = 7,       /* a CUDA runtime call failed */
    RN_EINTERNAL = 8    /* internal limit exceeded (e.g. a product row over 16384 distinct columns) */
} rn_status;

enum { RN_DEVICE = 0, RN_HOST = 1 };
enum { RN_ENERGY_CG = 0, RN_ENERGY_GMRES = 1 };
enum { RN_FP64 = 0, RN_MIXED = 1 };
enum { RN_OUTER_STATIONARY = 0, RN_OUTER_CG = 1, RN_OUTER_FGMRES = 2 };
/* Strength measures (Sec. 3.2): symmetric |a_ij| / sqrt(|a_ii a_jj|) >= theta;
 * classical (Ruge-Stueben) -a_ij >= theta max_{k != i} (-a_ik).  Both scaled by eq. soc. */
enum { RN_SOC_SYMMETRIC = 0, RN_SOC_CLASSICAL = 1 };

typedef struct {
    int32_t n_rows, n_cols;
    int64_t nnz;
    const int32_t *rowptr; /* n_rows + 1 */
    const int32_t *col;    /* nnz */
    const double *val;     /* nnz */
} rn_csr;

typedef struct {
    double soc_theta;        /* strength drop tolerance on the finest level (Sec. 3.2) */
    double soc_theta_coarse; /* on levels >= 1; < 0 means same as soc_theta */
    int degree;              /* d in N = S^d C (Sec. 3.4) */
    int n_sweeps;            /* energy-minimisation iterations (Sec. 3.6; paper: ceil(1.5 d)) */
    int energy_method;       /* RN_ENERGY_CG (SPD) or RN_ENERGY_GMRES */
    int energy_precond;      /* 1: Jacobi row scaling in CG energy minimisation */
    double prefilter;        /* theta_pre of Alg. 4 on N (<= 0: off) */
    double postfilter;       /* theta_post of Alg. 4 on P (<= 0: off) */
    int max_coarse;          /* coarsen while n > max_coarse */
    int max_levels;          /* <= 32 */
    int b_sweeps;            /* candidate relaxation sweeps (Sec. 3.1; paper: 4) */
    double omega;            /* weighted-Jacobi weight (cycle and candidate sweeps) */
    uint64_t seed;           /* aggregation priority seed (level l uses seed + l) */
    int symmetric;           /* 1: R = P^T;  0: R built from A^T and B-hat */
    int nu_pre, nu_post;     /* V-cycle relaxation counts */
    int precision;           /* RN_FP64, or RN_MIXED: FP32 cycle inside the FP64 outer iteration, and
                                FP32 energy-minimisation sweeps when k = 1 (FP64 sweeps for k > 1) */
    int outer;               /* RN_OUTER_STATIONARY / RN_OUTER_CG / RN_OUTER_FGMRES */
    int restart;             /* FGMRES restart length */
    int use_graphs;          /* 1: capture the preconditioner cycle in a CUDA graph */
    int keep_aux;            /* 1: keep S, N, T, agg, roots per level for rn_export_* */
    int coarse_cluster;      /* > 0: the cycle on the smallest levels (every operation taking at most
                                this many passes of one thread-block cluster's threads) runs as one
                                cluster launch; 0: one launch per operation on every level */
    int gamma;               /* coarse-grid corrections per level: 1 V-cycle, 2 W-cycle (Sec. 5.2's
                                W(1,1)); a level whose next level is the coarsest corrects once */
    int soc_kind;            /* strength measure (Sec. 3.2): RN_SOC_SYMMETRIC or RN_SOC_CLASSICAL */
    int block_size;          /* m, unknowns per node (node-major, m <= RN_MAX_BLOCK; 1: scalar problem).
                                m > 1 (systems, Sec. 3.2-3.6): S is amalgamated to nodes (largest entry of
                                each m x m block), aggregation and the pattern run on nodes and are
                                unamalgamated to unknowns, each root node carries m coarse unknowns, and
                                T injects the first m candidates normalised by the root node's block;
                                needs k >= m and n divisible by m */
    int autotune;            /* 1: the solve's SpMV schedule per matrix (lanes per row, hence rows per
                                staged tile, or the unstaged kernel) picked by timed trials on the
                                matrix, cached per matrix shape for the process; 0: the threshold rule
                                (the fewest lanes whose tile fits one shared-memory stage) */
    void *stream;            /* cudaStream_t */
    /* Device-memory hooks (both NULL: the stream-ordered pool, cudaMallocAsync;
     * one without the other is RN_EINVAL).  alloc(bytes, stream, ctx) returns
     * device memory for use in stream order on `stream`, or NULL, which fails
     * the call with RN_ENOMEM; dealloc(p, bytes, stream, ctx) takes it back in
     * stream order.  A hierarchy allocates and frees with the hooks of its
     * rn_setup call for its whole life (rn_solve and rn_free included), so they
     * and alloc_ctx must stay valid until rn_free.  Calls without an rn_params
     * argument (rn_energy_min, rn_adjoint_grad) use the pool. */
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*dealloc)(void *p, size_t bytes, void *stream, void *ctx);
    void *alloc_ctx;
} rn_params;

typedef struct {
    int iters;
    double rel_res;  /* ||b - A x|| / ||b|| in FP64 at exit */
    double rho;      /* average convergence factor (r_K / r_0)^(1/K) */
    double solve_ms; /* wall time of the call */
    int status;
} rn_solve_info;

#define RN_MAX_LEVELS 32
#define RN_MAX_CANDIDATES 4  /* k, the number of candidate vectors */
#define RN_MAX_BLOCK 3       /* m, unknowns per node */
typedef struct {
    int levels;
    int32_t n[RN_MAX_LEVELS];
    int64_t nnz_A[RN_MAX_LEVELS], nnz_P[RN_MAX_LEVELS], nnz_R[RN_MAX_LEVELS];
    double oc;        /* operator complexity, eq. oc */
    double cc;        /* cycle complexity, eq. cc */
    double setup_ms;  /* wall time of rn_setup */
    int agg_rounds;   /* aggregation rounds summed over levels */
} rn_stats;

typedef struct rn_hierarchy rn_hierarchy;

/* Fill *p with the defaults (theta 0.25, d 2, 4 CG sweeps, no filtering,
 * max_coarse 64, 4 candidate sweeps, omega 2/3, symmetric, V(1,1), FP64,
 * CG outer, graphs on, coarse_cluster 0).  Returns RN_EINVAL for
 * p == NULL. */
rn_status rn_default_params(rn_params *p);

/* Build the hierarchy (Alg. 3) for A with candidates B (n x k, row-major,
 * 1 <= k <= RN_MAX_CANDIDATES) and, when p->symmetric == 0, Bhat (candidates
 * for A^T, n x k).  Scalar problems (block size m = 1): the first candidate
 * is injected (root rows of P are identity rows) and the others are fitted
 * row by row on the pattern (eq. Tproj, Sec. 3.6), each row's k x k Gram
 * matrix inverted by its pseudo-inverse; every coarse level has k candidates.
 * `location` applies to A's arrays, B and Bhat.  On success *out owns the
 * hierarchy; on any error *out is NULL and nothing is leaked. */
rn_status rn_setup(const rn_csr *A, const double *B, const double *Bhat, int k, int location,
                   const rn_params *p, rn_hierarchy **out);

/* Solve A x = b to ||b - A x|| <= rtol ||b||: x holds x0 on entry and the
 * solution on exit (n entries each, `location` as in rn_setup).  info may be
 * NULL.  Returns RN_ENOTCONV when maxit outer iterations did not converge. */
rn_status rn_solve(rn_hierarchy *h, const double *b, double *x, int location, double rtol, int maxit,
                   rn_solve_info *info);

/* Solve A X = B for s right-hand sides at once (B and X: n x s, row-major;
 * X holds the initial guesses on entry and the solutions on exit).  The
 * stationary iteration X <- X + M(B - A X) applies the V-cycle to all s
 * columns together: every operator row is read once per operation for all
 * columns (SpMM in place of SpMV).  The cycle runs in the hierarchy's
 * precision (FP32 when mixed); residuals are FP64.  It stops when every
 * column satisfies ||b_c - A x_c|| < rtol ||b_c|| (a zero column when
 * ||b_c - A x_c|| < rtol).  info (may be NULL): iterations, the largest
 * column's relative residual, its average convergence factor, wall time.
 * Returns RN_EINVAL for s outside [1, 2048] or null arguments, RN_ENOTCONV
 * when a column is above the tolerance after maxit iterations. */
rn_status rn_solve_multi(rn_hierarchy *h, const double *B, double *X, int s, int location, double rtol, int maxit,
                         rn_solve_info *info);

/* Many independent problems (the paper has no batched form; a deployment
 * variant).  rn_setup_batched builds hierarchy i for (A[i], B[i], Bhat[i]),
 * all device data, k = 1, with the same params, whose stream must be NULL:
 * every problem gets a stream of its own and host threads (at most `threads`;
 * 0: one per hardware thread, at most 16) drive the setups, so they overlap
 * on the GPU.  Bhat may be NULL when p->symmetric.  out[i] receives problem
 * i's hierarchy; on any error every hierarchy is freed, out[] is all NULL and
 * the status of the first failing problem in index order is returned (its
 * message, prefixed with its index, is the last error).
 * rn_solve_batched solves A_i x_i = b_i (device vectors, x_i in/out) for all
 * i the same way, each on its hierarchy's stream; info (may be NULL) gets one
 * record per problem.  Results are those of rn_setup / rn_solve on each
 * problem alone. */
rn_status rn_setup_batched(int count, const rn_csr *A, const double *const *B, const double *const *Bhat,
                           const rn_params *p, int threads, rn_hierarchy **out);
/* Independent problems set up together (Alg. 3 on the block-diagonal union of
 * the problems; the paper sets up one operator).  rn_setup_merged builds
 * hierarchy i for (A[i], B[i]) (device data, one candidate each) in one pass:
 * every setup step is one set of launches for all problems, so many small
 * problems do not each pay the setup's launch and synchronisation latency.
 * Per problem are the aggregation priorities (a node's index within its own
 * problem), the energy minimisation's CG step lengths and stopping test
 * (reductions over chunks of one problem's pattern entries, in a fixed
 * order), and the end of coarsening (a problem leaves the merged operator at
 * its coarsest level).  So out[i] is the hierarchy rn_setup builds for
 * problem i: the same strength, aggregates, patterns and level sizes; values
 * agree to rounding (the CG sums run in another order).  out[i] owns its
 * memory and is used and freed like any hierarchy (rn_solve, rn_batch_merge,
 * rn_free); its stream is one of 64 streams the library keeps for the
 * process (problems i and i + 64 share one), each with a device pool of its
 * own, because a stream-ordered pool that holds blocks freed on many streams
 * is slow to allocate from.  Restrictions: params.stream NULL,
 * p->symmetric (R = P^T), energy_method RN_ENERGY_CG, block_size 1;
 * otherwise RN_EINVAL.  On any error every hierarchy is freed, out[] is all
 * NULL and the status is returned (the message names the problem where it
 * can).  Device memory comes from p's hooks (or the stream-ordered pool). */
rn_status rn_setup_merged(int count, const rn_csr *A, const double *const *B, const rn_params *p,
                          rn_hierarchy **out);
rn_status rn_solve_batched(int count, rn_hierarchy *const *h, const double *const *b, double *const *x, double rtol,
                           int maxit, int threads, rn_solve_info *info);

/* Independent problems solved as one (the same deployment variant; Sec. 2's
 * cycle and outer CG per problem).  rn_batch_merge copies the hierarchies
 * h[0..count) (set up with equal precision, omega, nu_pre, nu_post and
 * gamma = 1) into one block-diagonal hierarchy: problem p's operators on its
 * levels, and below its coarsest level identity transfers with relaxation
 * weight 0, which carry its right-hand side unchanged to the last level,
 * where every problem's coarsest block is solved with its own dense inverse.
 * So every cycle step, and every step of the outer CG (per-problem alpha,
 * beta and stopping, reduced over row chunks in a fixed order), is one launch
 * for all problems.  The h[i] are only read and may be freed afterwards.
 * stream: the batch's CUDA stream (NULL: a stream the library keeps for the
 * process, with a device pool of its own); the
 * solve and cycle read b[i] and write x[i] on it, and return after it has
 * finished with them.  Errors:
 * RN_EINVAL for count < 1, null arguments or differing cycle settings.
 * rn_batch_solve runs preconditioned CG on every problem (device vectors b[i],
 * x[i] of problem i's size; x[i] holds the initial guess and receives the
 * solution): a problem stops when ||b_i - A_i x_i|| < rtol ||b_i|| or after
 * maxit iterations; info (may be NULL) gets one record per problem (its
 * iterations, true relative residual, average convergence factor, the
 * call's wall time, status).  Returns RN_ENOTCONV when a problem did not
 * converge.  rn_batch_cycle applies one cycle to every problem: x[i] =
 * M_i^{-1} b[i].  rn_batch_free releases the batch (NULL: no-op). */
typedef struct rn_batch rn_batch;
rn_status rn_batch_merge(int count, rn_hierarchy *const *h, void *stream, rn_batch **out);
rn_status rn_batch_solve(rn_batch *b, const double *const *bvec, double *const *x, double rtol, int maxit,
                         rn_solve_info *info);
rn_status rn_batch_cycle(rn_batch *b, const double *const *bvec, double *const *x);
void rn_batch_free(rn_batch *b);

/* Apply one V-cycle to b with zero initial guess: x = M^{-1} b (device
 * pointers, FP64, level-0 size).  Used to check the cycle itself. */
rn_status rn_vcycle(rn_hierarchy *h, const double *b, double *x);

/* Release everything the hierarchy owns.  NULL is a no-op. */
void rn_free(rn_hierarchy *h);

/* Constrained energy minimisation of one transfer operator on a fixed pattern
 * (Alg. 3 'improve'; Sec. 3.6 with the row projection of eq. Tproj; Sec. 4,
 * Lemma th:cg): starting from the values P (in/out, nnz(N) entries on the
 * pattern of N), run `sweeps` iterations of CG (method RN_ENERGY_CG; Jacobi
 * row scaling when precond != 0) or GMRES (RN_ENERGY_GMRES) on the operator
 * X -> Proj(Mask_N(A X)), which keeps P on N, keeps root rows fixed and keeps
 * P Bc unchanged.
 *   A        n x n CSR (device), sorted columns, nonzero diagonal;
 *   N        n x n_c pattern (device CSR; N->val is ignored), sorted columns;
 *   rowtype  n entries (device): 0 free, 1 root (fixed), 2 unaggregated (fixed);
 *   Bc       n_c coarse candidates (device).
 * Work runs on `stream` (NULL: a stream the call creates); scratch comes from
 * the stream-ordered allocator.  Returns RN_EINVAL for bad sizes or a zero
 * diagonal; P is unchanged on error. */
rn_status rn_energy_min(const rn_csr *A, const rn_csr *N, const int32_t *rowtype, const double *Bc, double *P,
                        int sweeps, int method, int precond, void *stream);

/* rn_energy_min for callers that must not allocate device memory (the paper
 * has no counterpart; this is a deployment variant).  Examples: a host
 * framework whose caching allocator has reserved the GPU's memory, a
 * latency-critical loop that cannot afford an allocation's synchronisation,
 * a plugin host that forbids libraries to allocate.  Same arguments and result
 * as rn_energy_min with method RN_ENERGY_CG; the call makes no allocation: its
 * scratch is one statically allocated device array of about 16 MB, which every
 * GPU that loads this library keeps until the process exits.
 *   Limits: A->n_rows <= 262144 and N->nnz <= 524288; larger inputs return
 *   RN_EINVAL with a message naming the limit.
 *   The first call on a device resolves the array's device address
 *   (cudaGetSymbolAddress).
 *   stream NULL means the legacy default stream.
 *   All calls share the array: calls whose GPU work overlaps (other streams,
 *   other threads) race on it and must be serialised by the caller.
 *   The call reads one flag back to the host and synchronises its stream
 *   before it returns, so it cannot be captured into a CUDA graph.
 *   rn_allocation_count() is unchanged across the call. */
rn_status rn_energy_min_noalloc(const rn_csr *A, const rn_csr *N, const int32_t *rowtype, const double *Bc,
                                double *P, int sweeps, int precond, void *stream);

/* Level sizes and the complexities of Sec. 2.4 (eq. oc, eq. cc). */
rn_status rn_hierarchy_stats(const rn_hierarchy *h, rn_stats *s);

/* Copy one matrix of level `lvl` to host buffers.
 * which: 0 A, 1 S, 2 N (pattern after pre-filter and root pattern, values of
 * S^d C), 3 T, 4 P, 5 R.  S, N and T need keep_aux.  Call once with NULL
 * arrays to get n_rows, n_cols and nnz, then with buffers of rowptr[n_rows+1],
 * col[nnz], val[nnz].  Returns RN_EINVAL when the matrix does not exist. */
rn_status rn_export_csr(const rn_hierarchy *h, int lvl, int which, int32_t *n_rows, int32_t *n_cols, int64_t *nnz,
                        int32_t *rowptr, int32_t *col, double *val);

/* Copy one vector of level `lvl` to host.  which: 0 agg (int32, n), 1 roots
 * (int32, n_c), 2 row types (int32, n: 0 free, 1 root, 2 unaggregated),
 * 3 smoothed B (double, n), 4 Bc (double, n_c), 5 smoothed B-hat, 6 B-hat_c.
 * out == NULL only returns *len. */
rn_status rn_export_vec(const rn_hierarchy *h, int lvl, int which, int64_t *len, void *out);

/* Per-kernel device timing.  While enabled, every library kernel launch is
 * bracketed by CUDA events on its stream; rn_profile_read returns, per kernel
 * name, the launch count, summed device milliseconds and the algorithmic
 * bytes the launches moved (the traffic model of each kernel: every input
 * and output array touched once).  Process-wide, not thread-safe. */
typedef struct {
    char name[48];
    int64_t launches;
    double ms;
    double bytes;
} rn_kernel_stat;
rn_status rn_profile_enable(int on);
rn_status rn_profile_reset(void);
rn_status rn_profile_read(rn_kernel_stat *out, int max, int *count);

/* Number of library kernels launched by this process so far (kernels inside
 * a replayed CUDA graph are counted one by one). */
int64_t rn_kernel_launches(void);

/* Number of memory allocations the library has made in this process so far:
 * device buffers (from the caller's hooks or the stream-ordered allocator)
 * and page-locked host scratch.  No counterpart in the paper; it lets a caller
 * check that a call made no allocation (rn_energy_min_noalloc). */
int64_t rn_allocation_count(void);

/* Differentiation through a solve (x = A^{-1} b): given lambda = A^{-T} dL/dx,
 * the gradient with respect to A's stored values is dL/dA_ij = -lambda_i x_j.
 * Writes grad[e] = -lambda[row(e)] * x[col[e]] for every stored entry e of A,
 * in A's CSR order (A->val is not read and may be NULL).
 *   A        n_rows x n_cols CSR pattern (device), nnz entries;
 *   lambda   n_rows adjoint values (device); x  n_cols solution values (device);
 *   grad     nnz outputs (device, written).
 * Work runs on `stream` (NULL: a stream the call creates); the call returns
 * when it is done.  Returns RN_EINVAL for null arguments or bad sizes. */
rn_status rn_adjoint_grad(const rn_csr *A, const double *lambda, const double *x, double *grad, void *stream);

/* Measurement hook (no counterpart in the paper): time one level-0 launch of
 * the solve in isolation.  The operation is enqueued `reps` times on the
 * hierarchy's stream exactly as rn_solve issues it (kernel, launch shape,
 * buffers), each launch bracketed by CUDA events and preceded by a read of
 * `flush_bytes` bytes from a buffer the call allocates (0: no flush), so that
 * every launch starts with a cold L2 holding no dirty lines and the GPU is
 * busy while the launch is enqueued.  Outputs: *us the mean device time of one launch in microseconds,
 * *bytes its algorithmic bytes (0 for RN_OP_COARSE_CLUSTER), name (>= 48
 * chars, may be NULL) the launch's name.  The solve workspaces are left in an
 * unspecified state; the hierarchy stays valid (rn_solve and rn_vcycle
 * initialise them).  Returns RN_EINVAL for an operation this hierarchy does
 * not run (a one-level hierarchy, RN_OP_COARSE_CLUSTER with the cluster path
 * off) or reps outside [1, 100000]. */
enum {
    RN_OP_OUTER_SPMV = 0,      /* q = A p with <p, q> (FP64) */
    RN_OP_RELAX0_RESIDUAL = 1, /* level 0: residual after the first sweep from zero (the sweep's
                                  x0 = omega D^{-1} r is formed by RN_OP_CG_XR) */
    RN_OP_JACOBI_OUT = 2,      /* level 0: last post-sweep, writing the FP64 preconditioned vector z,
                                  fused with the outer CG's <r, z> (and <z, r_old>) */
    RN_OP_RESTRICT = 3,        /* b_1 = R_0 r_0 */
    RN_OP_PROLONG = 4,         /* x_0 += P_0 x_1 */
    RN_OP_CG_XR = 5,           /* x += alpha p, r -= alpha q, ||r||^2, and the cycle's level-0 x0 */
    RN_OP_CG_RZ = 6,           /* <r, z> (and <z, r_old>) on its own: used only when the cycle has no
                                  level-0 post-sweep */
    RN_OP_CG_P = 7,            /* p = z + beta p */
    RN_OP_COARSE_CLUSTER = 8,  /* the cycle on the smallest levels, one cluster launch */
    RN_OP_COUNT = 9
};
rn_status rn_time_op(rn_hierarchy *h, int op, int reps, int64_t flush_bytes, double *us, double *bytes, char *name);

/* Measurement hook for the setup (no counterpart in the paper): time one
 * level-0 operation of Alg. 3 in isolation, with the flush, events and
 * outputs of rn_time_op.  The energy-minimisation operations run on level 0's
 * minimisation pattern N (after the pre-filter) from its tentative T, in the
 * hierarchy's setup precision (FP32 sweeps when precision is RN_MIXED and k = 1); every
 * run starts from the CG state after the first sweep, restored before it
 * outside the timed region, so it times a general sweep.  They need a
 * hierarchy built with keep_aux and energy_method RN_ENERGY_CG.  The Galerkin
 * operations form A_0 P_0 and R_0 (A_0 P_0) as the setup does (symbolic and
 * numeric passes, with the products' host synchronisations), and the
 * transpose forms P_0^T.  Algorithmic bytes: the sweep 12 nnz(A) + 4 nnz(N)
 * + 64 nnz(N) + 8 n + 8 k n_c in FP64 (8, 4, 32, 4 and 4 k in place of 12,
 * 4, 64, 8 and 8 k for FP32 sweeps); A P: 12 (nnz(A) + nnz(P)) + 12 nnz(AP);
 * R (A P): 12 (nnz(R) + nnz(AP)) + 12 nnz(A_1); P^T: 24 nnz(P).  Returns
 * RN_EINVAL for an unknown operation, a one-level hierarchy or a hierarchy
 * without what the operation needs. */
enum {
    RN_SOP_ENERGY_SWEEP = 0,     /* one CG sweep: direction, masked product with <D, W>, update with rho */
    RN_SOP_ENERGY_DIRECTION = 1, /* D = D^{-1} R + beta D */
    RN_SOP_ENERGY_PRODUCT = 2,   /* W = Proj(Mask_N(A D)) with <D, W> and alpha */
    RN_SOP_ENERGY_UPDATE = 3,    /* P += alpha D, R -= alpha W, rho and beta */
    RN_SOP_GALERKIN_AP = 4,      /* A_0 P_0 */
    RN_SOP_GALERKIN_RAP = 5,     /* R_0 (A_0 P_0) = A_1 */
    RN_SOP_TRANSPOSE = 6,        /* P_0^T */
    RN_SOP_COUNT = 7
};
rn_status rn_time_setup_op(rn_hierarchy *h, int op, int reps, int64_t flush_bytes, double *us, double *bytes,
                           char *name);

const char *rn_last_error(void);
const char *rn_status_string(rn_status s);

#ifdef __cplusplus
}
#endif
#endif
