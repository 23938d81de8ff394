// rn_hier.cuh - the device hierarchy {A_l, P_l, R_l} of Alg. 3 plus solve
// workspaces.  HBM layout per level: CSR int32 row pointers / columns and
// FP64 values (plus FP32 value shadows for the mixed-precision cycle), the
// diagonal, and the level vectors; the coarsest level keeps a dense FP64
// inverse formed from its partially pivoted LU factors.
#pragma once
#include <functional>
#include <memory>

#include "rn_internal.cuh"

namespace rn {
struct MergedSetup;  // independent problems set up together (rn_setup.cu)
}

struct rn_level {
    rn::DCsr A, P, R;                       // operator, interpolation, restriction
    rn::DCsr S, N, T;                       // kept only with keep_aux
    rn::DVec<double> diag;                  // a_ii
    rn::DVec<double> wd;                    // omega / a_ii (the cycle's relaxation weights)
    rn::DVec<float> wd32;
    rn::DVec<int32_t> agg, roots, rowtype;  // aggregation (agg/roots kept with keep_aux)
    int32_t nc = 0;
    rn::DVec<double> B, Bc, Bhat, Bhatc;    // smoothed candidates and their injections
    // cycle workspaces (FP64 and FP32): right-hand side, iterate, scratch
    rn::DVec<double> b, x, t, r;
    rn::DVec<float> b32, x32, t32, r32;
    int spmv_group = 4;                     // lanes per row for A's SpMV
    int p_group = 4, r_group = 4;
};

struct rn_hierarchy {
    rn_params p{};
    int k = 1;                 // candidate vectors: B is n x k, Bc nc x k (row-major) on every level
    int mb = 1;                // unknowns per node (block size m); nodes are m consecutive unknowns
    cudaStream_t s = nullptr;  // params.stream, or a stream the hierarchy created (own_stream)
    bool own_stream = false;
    std::vector<std::unique_ptr<rn_level>> lev;  // lev.back() is the coarsest
    int32_t nL = 0;
    rn::DVec<double> Ainv;                        // coarsest inverse, row-major nL x nL
    // merged independent problems: the coarsest level is block diagonal, block
    // p on rows [cblk_row[p], cblk_row[p+1]) with its inverse at Ainv + cblk_inv[p]
    rn::DVec<int32_t> cblk_row;
    rn::DVec<int64_t> cblk_inv;
    int ncblk = 0;
    rn::DVec<double> partial;                     // block partial sums (2 x kReduceBlocks)
    rn::DVec<unsigned> counters;                  // arrival counter of the grid reductions (kept at 0)
    rn::DVec<double> scal;                        // device scalars
    rn::DVec<int32_t> iflags;                     // device int flags
    // outer-iteration vectors (level-0 size)
    rn::DVec<double> r, z, pv, q, w, rold, xs;     // xs: the CG solve graph's iterate
    rn::DVec<double> V, Z, H, gv;                 // FGMRES basis, preconditioned basis, Hessenberg, rhs
    // CUDA graph of one preconditioner application (FP64 or FP32 cycle)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    const double *graph_in = nullptr;
    double *graph_out = nullptr;
    int64_t graph_kernels = 0;                    // kernel nodes in the captured cycle
    // CUDA graph of the whole outer CG loop (conditional WHILE / IF nodes)
    cudaGraph_t cg_graph = nullptr;
    cudaGraphExec_t cg_exec = nullptr;
    int64_t cg_kernels[2] = {0, 0};               // kernel nodes of the two halves of an iteration
    // cycle below level sub_k run by one thread-block cluster (sub_k < 0: off)
    rn::DVec<unsigned char> sub_desc;             // SubPhase<T>[sub_nph]
    int sub_k = -1, sub_cs = 0, sub_nph = 0;
    // solve-path kernels launched with programmatic dependent launch
    bool pdl = true;
    // statistics
    double setup_ms = 0.0;
    int agg_rounds = 0;
    // set while this hierarchy is the working copy of a merged setup
    rn::MergedSetup *merged = nullptr;
    rn::DVec<int32_t> maxlen;  // longest rows per level and matrix, between prepare_solve_begin and _end
    int pool = -1;             // the library device pool its buffers come from without hooks (-1: default)
    ~rn_hierarchy();
};

// Independent problems merged into one block-diagonal hierarchy (rn_batch.cu):
// the merged hierarchy, the level-0 row offsets of every problem, the
// reduction chunks and the per-problem CG state.
struct rn_batch {
    std::unique_ptr<rn_hierarchy> M;
    bool own_stream = false;
    int np = 0, nch = 0;
    std::vector<int32_t> off0;                     // level-0 rows of problem p: [off0[p], off0[p+1])
    rn::DVec<int32_t> ch_lo, ch_hi, ch_pid, pc;    // chunk rows, problem; first chunk of each problem
    rn::DVec<double> part;                         // chunk partial sums
    rn::DVec<unsigned> counter;
    rn::DVec<double> d;                            // per-problem CG scalars
    rn::DVec<int32_t> iv;                          // per-problem counters and flags, then the active count
    rn::DVec<double> bm, xm;                       // merged right-hand side and iterate
    rn::DVec<int32_t> offs;                        // every level's problem row offsets (levels x (np + 1))
    rn::DVec<unsigned char> lists;                 // tile-list descriptors of the merged matrices
    int nlists = 0;
    bool flexible = false;                         // mixed precision: flexible (Polak-Ribiere) beta
    double rtol = 0.0, graph_rtol = -1.0;
    int maxit = 0, graph_maxit = -1;
    cudaGraph_t it_graph = nullptr;                // one CG iteration
    cudaGraphExec_t it_exec = nullptr;
    int64_t it_kernels = 0;
    ~rn_batch();
};

namespace rn {
rn_batch *batch_merge(int count, rn_hierarchy *const *hs, cudaStream_t s);
void batch_cycle(rn_batch &b, const double *const *rhs, double *const *out);
rn_status batch_solve(rn_batch &b, const double *const *rhs, double *const *x, double rtol, int maxit,
                      rn_solve_info *info);
// Smallest coarse levels in one cluster launch (rn_cluster.cu)
constexpr int32_t kSubMaxCoarse = 1024;  // coarsest size the cluster solves densely
constexpr int kSubMaxPhases = 96;        // longest phase list the kernel stages
enum SubOp { SUB_SPMV = 0, SUB_SPMV_ADD = 1, SUB_RESID = 2, SUB_JACOBI = 3, SUB_JZ_RESID = 4, SUB_SCALE = 5,
             SUB_COARSE = 6 };
template <typename T>
struct SubMat {  // CSR view with the lanes per row the cluster kernel uses (trivial type: staged in shared memory)
    int32_t n;
    int g;
    const int32_t *rp, *col;
    const T *val;
};
// One phase: y = op(M, x, b) with relaxation weights d (omega / a_ii); xz is
// the second output of SUB_JZ_RESID; SUB_COARSE reads the dense inverse.
template <typename T>
struct SubPhase {
    int op;
    SubMat<T> M;
    const T *x, *b, *d;
    T *y, *xz;
};
void prepare_subcycle(rn_hierarchy &h);
template <typename T>
void launch_subcycle(rn_hierarchy &h, T *cur_k, const char *name);
// setup (rn_setup.cu)
void build_hierarchy(rn_hierarchy &h, const CsrView &A0, const double *B0, const double *Bhat0);
// Independent problems set up together: out[t] receives problem t's hierarchy
// (each already holding params, stream and scratch as rn_setup makes them).
void build_hierarchies_merged(std::vector<rn_hierarchy *> &out, const std::vector<CsrView> &A,
                              const std::vector<const double *> &B, cudaStream_t s);

struct Pattern {  // borrowed view of a fixed interpolation pattern
    int32_t n, nc;
    int64_t nnz;
    const int32_t *rp, *col;
};
// Independent problems set up together: at the current level problem t of
// the merged matrix owns rows [ro[t], ro[t + 1]) (host and device copies).
struct SegRows {
    int np = 0;
    std::vector<int32_t> ro;
    const int32_t *ro_d = nullptr;
};
// Context of one energy minimisation: stream, reduction scratch, scalar block
// (>= 8 doubles), flags (>= 2 ints), settings, and optional workspaces
// (CG: nnz(N) doubles each; rs2: n doubles; allocated internally when null).
struct EmCtx {
    cudaStream_t s = nullptr;
    double *partial = nullptr;
    unsigned *counter = nullptr;
    double *sc = nullptr;
    int32_t *fl = nullptr;
    int precond = 1;
    int method = RN_ENERGY_CG;
    double *R = nullptr, *Dd = nullptr, *W = nullptr;
    double *rs2 = nullptr;  // n rows: the row projection's scales (allocated internally when null)
    bool fp32 = false;      // CG sweeps in FP32 (mixed precision); workspaces then allocated internally
    int k = 1;              // candidates (Bc is nc x k); k > 1 projects with per-row Gram pseudo-inverses
    const double *u64 = nullptr;      // k > 1: U of every row's Bc_J already formed on N (else formed inside)
    const int32_t *zero_row = nullptr;
    // true: every product scans the pattern rows (energy_product_kernel) and
    // no gather map is built; with R, Dd, W, rs2 supplied, k = 1 and FP64
    // sweeps the minimisation then allocates nothing (same results)
    bool scan_only = false;
    // independent problems set up together: per-problem CG scalars (CG, k = 1)
    const SegRows *seg = nullptr;
};
// dinv: the inverted diagonal of A (CG's preconditioner D^{-1} when c.precond)
void energy_min(const EmCtx &c, const CsrView &A, const Pattern &N, double *X, const int32_t *rowtype,
                const double *Bc, const double *dinv, int sweeps);
// solve (rn_solve.cu)
void prepare_solve(rn_hierarchy &h);  // prepare_solve_begin then prepare_solve_end
void prepare_solve_begin(rn_hierarchy &h);
void prepare_solve_end(rn_hierarchy &h);
rn_status solve(rn_hierarchy &h, const double *b, double *x, double rtol, int maxit, rn_solve_info *info);
void apply_cycle(rn_hierarchy &h, const double *rhs, double *out);
void cycle_launches(rn_hierarchy &h, const double *rhs, double *out);  // the cycle's launches, no graph
void outer_spmv(rn_hierarchy &h, const double *x, double *y);          // y = A_0 x
void outer_residual(rn_hierarchy &h, const double *x, const double *b, double *r);  // r = b - A_0 x
void cycle_checked(rn_hierarchy &h, const double *rhs, double *out);  // + staging-error check
void time_op(rn_hierarchy &h, int op, int reps, int64_t flush_bytes, double *us, double *bytes, std::string &name);
// Mean device time (us) of `timed`, run reps times on stream s, each run
// preceded by `before` (untimed; may be empty) and a read of flush_bytes
// that leaves L2 cold and keeps the GPU busy while the work is enqueued.
double time_launches(cudaStream_t s, int reps, int64_t flush_bytes, const std::function<void()> &before,
                     const std::function<void()> &timed);
// One setup operation of level 0 timed the same way (rn_time_setup_op).
void time_setup_op(rn_hierarchy &h, int op, int reps, int64_t flush_bytes, double *us, double *bytes,
                   std::string &name);
// many right-hand sides (rn_multi.cu)
rn_status solve_multi(rn_hierarchy &h, const double *B, double *X, int ns, double rtol, int maxit,
                      rn_solve_info *info);
template <typename T>
T *pre_smoothed(rn_level &L, int nu_pre);
}  // namespace rn
