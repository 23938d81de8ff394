// rn_hier.cuh - the device hierarchy {A_l, P_l, R_l} of Alg. 3 plus solve
// workspaces.  HBM layout per level: CSR int32 row pointers / columns and
// FP64 values (plus FP32 value shadows for the mixed-precision cycle), the
// diagonal, and the level vectors; the coarsest level keeps a dense FP64
// inverse formed from its partially pivoted LU factors.
#pragma once
#include <memory>

#include "rn_internal.cuh"

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
    cudaStream_t s = nullptr;  // params.stream, or a stream the hierarchy created (own_stream)
    bool own_stream = false;
    std::vector<std::unique_ptr<rn_level>> lev;  // lev.back() is the coarsest
    int32_t nL = 0;
    rn::DVec<double> Ainv;                        // coarsest inverse, row-major nL x nL
    rn::DVec<double> partial;                     // block partial sums (2 x kReduceBlocks)
    rn::DVec<unsigned> counters;                  // arrival counter of the grid reductions (kept at 0)
    rn::DVec<double> scal;                        // device scalars
    rn::DVec<int32_t> iflags;                     // device int flags
    // outer-iteration vectors (level-0 size)
    rn::DVec<double> r, z, pv, q, w, rold;
    rn::DVec<double> V, Z, H, gv;                 // FGMRES basis, preconditioned basis, Hessenberg, rhs
    // CUDA graph of one preconditioner application (FP64 or FP32 cycle)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    const double *graph_in = nullptr;
    double *graph_out = nullptr;
    int64_t graph_kernels = 0;                    // kernel nodes in the captured cycle
    // statistics
    double setup_ms = 0.0;
    int agg_rounds = 0;
    ~rn_hierarchy();
};

namespace rn {
// setup (rn_setup.cu)
void build_hierarchy(rn_hierarchy &h, const CsrView &A0, const double *B0, const double *Bhat0);

struct Pattern {  // borrowed view of a fixed interpolation pattern
    int32_t n, nc;
    int64_t nnz;
    const int32_t *rp, *col;
};
// Context of one energy minimisation: stream, reduction scratch, scalar block
// (>= 8 doubles), flags (>= 2 ints), settings, and optional CG workspaces
// (nnz(N) doubles each; allocated internally when null).
struct EmCtx {
    cudaStream_t s = nullptr;
    double *partial = nullptr;
    unsigned *counter = nullptr;
    double *sc = nullptr;
    int32_t *fl = nullptr;
    int precond = 1;
    int method = RN_ENERGY_CG;
    double *R = nullptr, *Dd = nullptr, *W = nullptr;
};
void energy_min(const EmCtx &c, const CsrView &A, const Pattern &N, double *X, const int32_t *rowtype,
                const double *Bc, const double *diag, int sweeps);
// solve (rn_solve.cu)
void prepare_solve(rn_hierarchy &h);
rn_status solve(rn_hierarchy &h, const double *b, double *x, double rtol, int maxit, rn_solve_info *info);
void apply_cycle(rn_hierarchy &h, const double *rhs, double *out);
void cycle_checked(rn_hierarchy &h, const double *rhs, double *out);  // + staging-error check
}  // namespace rn
