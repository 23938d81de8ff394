// rn_solve.cu - V(nu_pre, nu_post) cycle (Sec. 2, eq. twogrid applied
// recursively) and the outer iterations.
//
// The cycle is a fixed sequence of launches per level - weighted Jacobi,
// residual, restriction R r, recursion, prolongation x += P x_c, weighted
// Jacobi - ending in a dense solve x = A_L^{-1} b on the coarsest level.  All
// sizes are fixed after setup, so one application of the cycle is captured
// in a CUDA graph and replayed.  In mixed precision the cycle runs on FP32
// shadows of A, P, R and the diagonal; the outer iteration (residual, Krylov
// vectors, dot products) and the coarsest solve stay FP64.
#include <algorithm>
#include <cmath>

#include "rn_hier.cuh"

namespace rn {

constexpr int kS = 256;  // threads per block, SpMV family

enum SpOp { OP_SPMV = 0, OP_SPMV_ADD = 1, OP_RESID = 2, OP_JACOBI = 3 };

// Row-group SpMV family: G lanes per row, rows contiguous per block.
//   OP_SPMV      y = A x
//   OP_SPMV_ADD  y += A x            (prolongation: A = P)
//   OP_RESID     y = b - A x         (+ sum y^2 into partial)
//   OP_JACOBI    y = x + omega (b - A x) / diag
template <typename T, int G, int OP>
__global__ void __launch_bounds__(kS)
spmv_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col, const T *__restrict__ val,
            const T *__restrict__ x, const T *__restrict__ b, const T *__restrict__ diag, T omega, T *__restrict__ y,
            double *__restrict__ partial) {
    __shared__ double sm[32];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    double nrm = 0.0;
    for (int32_t i = blockIdx.x * (kS / G) + g; i < n; i += gridDim.x * (kS / G)) {
        T acc = T(0);
        const int32_t e1 = rp[i + 1];
        for (int32_t e = rp[i] + lane; e < e1; e += G) acc = fma(val[e], x[col[e]], acc);
        if (G > 1) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, G);
        }
        if (lane == 0) {
            if (OP == OP_SPMV) y[i] = acc;
            else if (OP == OP_SPMV_ADD) y[i] += acc;
            else if (OP == OP_RESID) {
                const T r = b[i] - acc;
                y[i] = r;
                nrm += (double)r * (double)r;
            } else {
                y[i] = x[i] + omega * (b[i] - acc) / diag[i];
            }
        }
    }
    if (OP == OP_RESID && partial) {
        const double t = block_sum<kS>(nrm, sm);
        if (threadIdx.x == 0) partial[blockIdx.x] = t;
    }
}

template <typename T>
__global__ void jacobi_zero_kernel(int32_t n, const T *__restrict__ b, const T *__restrict__ diag, T omega,
                                   T *__restrict__ y) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = omega * b[i] / diag[i];
}

// x = A_L^{-1} b on the coarsest level (FP64 arithmetic, T in/out), warp per row
template <typename T>
__global__ void coarse_solve_kernel(int32_t n, const double *__restrict__ Ainv, const T *__restrict__ b,
                                    T *__restrict__ x) {
    const int lane = threadIdx.x & 31;
    for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        double acc = 0.0;
        for (int32_t j = lane; j < n; j += 32) acc = fma(Ainv[(int64_t)i * n + j], (double)b[j], acc);
        acc = warp_sum(acc);
        if (lane == 0) x[i] = (T)acc;
    }
}

__global__ void d2f_kernel(int64_t n, const double *__restrict__ x, float *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
__global__ void f2d_kernel(int64_t n, const float *__restrict__ x, double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// ------------------------------------------------------------------ outer-iteration vector kernels
// sc: device scalars.  Layout used by the outer solvers:
//   sc[8] ||r||^2, sc[9] <r,z>, sc[10] <p,q>, sc[11] <z, r_old>, sc[12] alpha, sc[13] beta, sc[14] rz_prev
__global__ void axpy_kernel(int64_t n, double *__restrict__ x, const double *__restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += z[i];
}

__global__ void cg_alpha_kernel(double *sc) { sc[12] = sc[9] / sc[10]; }

// x += alpha p; r_old = r (optional); r -= alpha q; partial ||r||^2
__global__ void __launch_bounds__(kS)
cg_xr_kernel(int64_t n, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
             const double *__restrict__ q, double *__restrict__ rold, const double *__restrict__ sc,
             double *__restrict__ partial) {
    __shared__ double sm[32];
    const double a = sc[12];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = x[i] + a * p[i];
        const double ri = r[i];
        if (rold) rold[i] = ri;
        const double rn = ri - a * q[i];
        r[i] = rn;
        acc = fma(rn, rn, acc);
    }
    const double t = block_sum<kS>(acc, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// <r,z> and (flexible) <z, r_old>
__global__ void __launch_bounds__(kS)
cg_rz_kernel(int64_t n, const double *__restrict__ r, const double *__restrict__ z, const double *__restrict__ rold,
             double *__restrict__ partial) {
    __shared__ double sm[32];
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a = fma(r[i], z[i], a);
        if (rold) b = fma(z[i], rold[i], b);
    }
    const double ta = block_sum<kS>(a, sm);
    const double tb = block_sum<kS>(b, sm);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = ta;
        partial[kReduceBlocks + blockIdx.x] = tb;
    }
}

// beta = <z,r> / rz_prev  (standard)  or  (<z,r> - <z,r_old>) / rz_prev  (flexible)
__global__ void cg_beta_kernel(double *sc, int flexible) {
    const double rz = sc[9];
    sc[13] = (flexible ? (rz - sc[11]) : rz) / sc[14];
    sc[14] = rz;
}

__global__ void cg_p_kernel(int64_t n, double *__restrict__ p, const double *__restrict__ z,
                            const double *__restrict__ sc, int first) {
    const double b = first ? 0.0 : sc[13];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : z[i] + b * p[i];
}

__global__ void scale_copy_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ den,
                                  double *__restrict__ y, int sqrt_den) {
    const double d = sqrt_den ? sqrt(*den) : *den;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] / d;
}

__global__ void axpy_dev_kernel(int64_t n, double *__restrict__ w, const double *__restrict__ v,
                                const double *__restrict__ h) {
    const double c = *h;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = w[i] - c * v[i];
}

// FGMRES Givens step on column j (H row-major (m+1) x m); g rhs; res -> sc[15]
__global__ void fg_givens_kernel(int m, int j, double *H, double *cs, double *sn, double *g, double *sc) {
    const double hn = sqrt(sc[8]);
    H[(j + 1) * m + j] = hn;
    for (int i = 0; i < j; i++) {
        double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
    }
    const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
    cs[j] = den > 0.0 ? H[j * m + j] / den : 1.0;
    sn[j] = den > 0.0 ? H[(j + 1) * m + j] / den : 0.0;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    sc[15] = fabs(g[j + 1]);
    sc[16] = hn;
}

__global__ void fg_start_kernel(double *g, int m, double *sc) {
    const double beta = sqrt(sc[8]);
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
}

__global__ void fg_backsolve_kernel(int m, int k, const double *H, const double *g, double *y) {
    for (int i = k - 1; i >= 0; i--) {
        double s = g[i];
        for (int j = i + 1; j < k; j++) s -= H[i * m + j] * y[j];
        y[i] = s / H[i * m + i];
    }
}

__global__ void fg_update_kernel(int64_t n, int k, double *__restrict__ x, const double *__restrict__ Z,
                                 const double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = x[i];
        for (int j = 0; j < k; j++) v = v + y[j] * Z[(int64_t)j * n + i];
        x[i] = v;
    }
}

// ================================================================== host side
static int pick_spmv_g(double avg) {
    if (avg <= 3.0) return 2;
    if (avg <= 12.0) return 4;
    if (avg <= 24.0) return 8;
    if (avg <= 48.0) return 16;
    return 32;
}

template <typename T>
static const T *vals_of(const DCsr &A);
template <>
const double *vals_of<double>(const DCsr &A) { return A.val.p; }
template <>
const float *vals_of<float>(const DCsr &A) { return A.val32.p; }

template <typename T, int OP>
static void spmv_launch(const char *name, const DCsr &A, int G, const T *x, const T *b, const T *diag, T omega, T *y,
                        double *partial, int *grid_out, cudaStream_t s) {
    const int32_t n = A.n;
    if (n == 0) return;
    int grid = grid_for(n, kS / G, 8);
    if (grid > kReduceBlocks) grid = kReduceBlocks;
    if (grid_out) *grid_out = grid;
    const double vb = sizeof(T);
    // algorithmic bytes: matrix (index + value), row pointers, x gathered once,
    // output (and b, diag, x_i where used) once
    double bytes = (4.0 + vb) * A.nnz + 4.0 * (n + 1) + vb * A.m + vb * n;
    if (OP == OP_SPMV_ADD) bytes += vb * n;
    if (OP == OP_RESID) bytes += vb * n;
    if (OP == OP_JACOBI) bytes += 2.0 * vb * n;
    const T *val = vals_of<T>(A);
#define RN_SPMV_CASE(GG)                                                                                   \
    case GG:                                                                                               \
        RN_LAUNCH(name, bytes, s, (spmv_kernel<T, GG, OP>), grid, kS, 0, n, A.rowptr.p, A.col.p, val, x, b, \
                  diag, omega, y, partial);                                                                \
        break;
    switch (G) {
        RN_SPMV_CASE(2)
        RN_SPMV_CASE(4)
        RN_SPMV_CASE(8)
        RN_SPMV_CASE(16)
        RN_SPMV_CASE(32)
        default: fail(RN_EINTERNAL, "bad spmv group");
    }
#undef RN_SPMV_CASE
}

template <typename T>
struct LevelBufs;
template <>
struct LevelBufs<double> {
    static double *b(rn_level &L) { return L.b.p; }
    static double *x(rn_level &L) { return L.x.p; }
    static double *t(rn_level &L) { return L.t.p; }
    static double *r(rn_level &L) { return L.r.p; }
    static const double *d(rn_level &L) { return L.diag.p; }
};
template <>
struct LevelBufs<float> {
    static float *b(rn_level &L) { return L.b32.p; }
    static float *x(rn_level &L) { return L.x32.p; }
    static float *t(rn_level &L) { return L.t32.p; }
    static float *r(rn_level &L) { return L.r32.p; }
    static const float *d(rn_level &L) { return L.diag32.p; }
};

static const char *kJacobiName[2] = {"cycle_jacobi_f64", "cycle_jacobi_f32"};
static const char *kResidName[2] = {"cycle_residual_f64", "cycle_residual_f32"};
static const char *kRestrictName[2] = {"cycle_restrict_f64", "cycle_restrict_f32"};
static const char *kProlongName[2] = {"cycle_prolong_f64", "cycle_prolong_f32"};

// One cycle on level l with zero initial guess: b_l must hold the right-hand
// side.  Returns the buffer with the result; when `out` is given (level 0)
// the last relaxation writes there.
template <typename T>
static T *vcycle(rn_hierarchy &h, int l, T *out) {
    using LB = LevelBufs<T>;
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[l];
    const int prec = (sizeof(T) == 4);
    const int32_t n = L.A.n;
    T *b = LB::b(L);
    if (l == (int)h.lev.size() - 1) {
        T *x = out ? out : LB::x(L);
        RN_LAUNCH("cycle_coarse_solve", 8.0 * n * n + 2.0 * sizeof(T) * n, s, coarse_solve_kernel<T>,
                  grid_for((int64_t)n * 32, 256, 4), 256, 0, n, h.Ainv.p, b, x);
        return x;
    }
    const T omega = (T)h.p.omega;
    const T *d = LB::d(L);
    T *cur = LB::x(L), *oth = LB::t(L);
    const int npre = h.p.nu_pre, npost = h.p.nu_post;
    for (int k = 0; k < npre; k++) {
        if (k == 0) {
            RN_LAUNCH(kJacobiName[prec], 3.0 * sizeof(T) * n, s, jacobi_zero_kernel<T>, grid_for(n, 1024), 256, 0, n,
                      b, d, omega, cur);
        } else {
            spmv_launch<T, OP_JACOBI>(kJacobiName[prec], L.A, L.spmv_group, cur, b, d, omega, oth, nullptr, nullptr, s);
            std::swap(cur, oth);
        }
    }
    if (npre == 0) RN_CUDA_CHECK(cudaMemsetAsync(cur, 0, sizeof(T) * n, s));
    T *r = LB::r(L);
    spmv_launch<T, OP_RESID>(kResidName[prec], L.A, L.spmv_group, cur, b, nullptr, T(0), r, nullptr, nullptr, s);
    rn_level &Lc = *h.lev[l + 1];
    spmv_launch<T, OP_SPMV>(kRestrictName[prec], L.R, L.r_group, r, nullptr, nullptr, T(0), LB::b(Lc), nullptr,
                            nullptr, s);
    T *xc = vcycle<T>(h, l + 1, nullptr);
    spmv_launch<T, OP_SPMV_ADD>(kProlongName[prec], L.P, L.p_group, xc, nullptr, nullptr, T(0), cur, nullptr, nullptr,
                                s);
    for (int k = 0; k < npost; k++) {
        T *dst = (out && k == npost - 1) ? out : oth;
        spmv_launch<T, OP_JACOBI>(kJacobiName[prec], L.A, L.spmv_group, cur, b, d, omega, dst, nullptr, nullptr, s);
        if (dst == out) return out;
        std::swap(cur, oth);
    }
    if (out) {
        d2d(out, cur, n, s);
        return out;
    }
    return cur;
}

// out = M rhs (FP64 in/out; level-0 size), without the graph
static void cycle_direct(rn_hierarchy &h, const double *rhs, double *out) {
    cudaStream_t s = h.s;
    rn_level &L0 = *h.lev[0];
    const int64_t n = L0.A.n;
    if (h.p.precision == RN_MIXED) {
        RN_LAUNCH("convert", 12.0 * n, s, d2f_kernel, grid_for(n, 1024), 256, 0, n, rhs, L0.b32.p);
        float *res = vcycle<float>(h, 0, nullptr);
        RN_LAUNCH("convert", 12.0 * n, s, f2d_kernel, grid_for(n, 1024), 256, 0, n, res, out);
    } else {
        d2d(L0.b.p, rhs, n, s);
        vcycle<double>(h, 0, out);
    }
}

void apply_cycle(rn_hierarchy &h, const double *rhs, double *out) {
    cudaStream_t s = h.s;
    if (!h.p.use_graphs || profiling_enabled()) {
        cycle_direct(h, rhs, out);
        return;
    }
    rn_level &L0 = *h.lev[0];
    const int64_t n = L0.A.n;
    if (!h.graph_exec) {
        const int64_t before = launches_so_far();
        RN_CUDA_CHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            cycle_direct(h, h.graph_in, h.graph_out);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        RN_CUDA_CHECK(cudaStreamEndCapture(s, &h.graph));
        RN_CUDA_CHECK(cudaGraphInstantiate(&h.graph_exec, h.graph, 0));
        h.graph_kernels = launches_so_far() - before;
        add_launches(-h.graph_kernels);  // captured, not launched
    }
    if (rhs != h.graph_in) d2d(const_cast<double *>(h.graph_in), rhs, n, s);
    RN_CUDA_CHECK(cudaGraphLaunch(h.graph_exec, s));
    add_launches(h.graph_kernels);
    if (out != h.graph_out) d2d(out, h.graph_out, n, s);
}

void prepare_solve(rn_hierarchy &h) {
    cudaStream_t s = h.s;
    const bool mixed = h.p.precision == RN_MIXED;
    for (size_t l = 0; l < h.lev.size(); l++) {
        rn_level &L = *h.lev[l];
        const int32_t n = L.A.n;
        L.b.alloc(n, s);
        L.x.alloc(n, s);
        L.t.alloc(n, s);
        L.r.alloc(n, s);
        L.spmv_group = pick_spmv_g(n ? (double)L.A.nnz / n : 1.0);
        if (L.P.n) L.p_group = pick_spmv_g((double)L.P.nnz / L.P.n);
        if (L.R.n) L.r_group = pick_spmv_g((double)L.R.nnz / L.R.n);
        if (mixed) {
            L.b32.alloc(n, s);
            L.x32.alloc(n, s);
            L.t32.alloc(n, s);
            L.r32.alloc(n, s);
            L.A.val32.alloc(L.A.nnz, s);
            to_float(L.A.val.p, L.A.val32.p, L.A.nnz, s);
            L.diag32.alloc(n, s);
            to_float(L.diag.p, L.diag32.p, n, s);
            if (L.P.nnz) {
                L.P.val32.alloc(L.P.nnz, s);
                to_float(L.P.val.p, L.P.val32.p, L.P.nnz, s);
            }
            if (L.R.nnz) {
                L.R.val32.alloc(L.R.nnz, s);
                to_float(L.R.val.p, L.R.val32.p, L.R.nnz, s);
            }
        }
    }
    const int64_t n0 = h.lev[0]->A.n;
    h.r.alloc(n0, s);
    h.z.alloc(n0, s);
    h.pv.alloc(n0, s);
    h.q.alloc(n0, s);
    h.w.alloc(n0, s);
    h.rold.alloc(n0, s);
    // the partial-sum buffer needs room for two reductions at once
    h.partial.alloc(2 * kReduceBlocks, s);
    h.graph_in = h.r.p;
    h.graph_out = h.z.p;
    if (h.p.outer == RN_OUTER_FGMRES) {
        const int m = std::max(1, h.p.restart);
        h.V.alloc((size_t)(m + 1) * n0, s);
        h.Z.alloc((size_t)m * n0, s);
        h.H.alloc((size_t)(m + 1) * m + 4 * (m + 1), s);
    }
}

static double norm_from(double *sc_slot, cudaStream_t s) { return std::sqrt(read_scalar(sc_slot, s)); }

rn_status solve(rn_hierarchy &h, const double *b, double *x, double rtol, int maxit, rn_solve_info *info) {
    cudaStream_t s = h.s;
    rn_level &L0 = *h.lev[0];
    const int64_t n = L0.A.n;
    double *sc = h.scal.p;
    double *part = h.partial.p;
    int grid = 1;
    const double t0 = now_ms();
    // ||b||
    dot(b, b, n, sc + 17, s, part);
    double nb = norm_from(sc + 17, s);
    if (nb == 0.0) nb = 1.0;
    // r = b - A x
    spmv_launch<double, OP_RESID>("outer_residual", L0.A, L0.spmv_group, x, b, nullptr, 0.0, h.r.p, part, &grid, s);
    reduce_partials(part, grid, sc + 8, s);
    const double r0 = norm_from(sc + 8, s);
    double rn = r0;
    int it = 0;
    rn_status st = RN_ENOTCONV;
    const int eg = grid_for(n, 1024);
    const int rg = std::min(grid_for(n, kS * 4, 8), kReduceBlocks);
    if (rn / nb < rtol) st = RN_OK;
    if (st != RN_OK && h.p.outer == RN_OUTER_STATIONARY) {
        // x <- x + M (b - A x): the cycle applied to the current iterate
        for (it = 1; it <= maxit; it++) {
            apply_cycle(h, h.r.p, h.z.p);
            RN_LAUNCH("outer_axpy", 24.0 * n, s, axpy_kernel, eg, 256, 0, n, x, h.z.p);
            spmv_launch<double, OP_RESID>("outer_residual", L0.A, L0.spmv_group, x, b, nullptr, 0.0, h.r.p, part,
                                          &grid, s);
            reduce_partials(part, grid, sc + 8, s);
            rn = norm_from(sc + 8, s);
            if (rn / nb < rtol) { st = RN_OK; break; }
        }
        if (it > maxit) it = maxit;
    } else if (st != RN_OK && h.p.outer == RN_OUTER_CG) {
        const bool flexible = h.p.precision == RN_MIXED;
        apply_cycle(h, h.r.p, h.z.p);
        RN_LAUNCH("outer_cg_vec", 16.0 * n, s, cg_rz_kernel, rg, kS, 0, n, h.r.p, h.z.p, nullptr, part);
        reduce_partials(part, rg, sc + 9, s);
        RN_LAUNCH("outer_cg_vec", 24.0 * n, s, cg_p_kernel, eg, 256, 0, n, h.pv.p, h.z.p, sc, 1);
        d2d(sc + 14, sc + 9, 1, s);
        for (it = 1; it <= maxit; it++) {
            // q = A p, <p, q>
            spmv_launch<double, OP_SPMV>("outer_spmv", L0.A, L0.spmv_group, h.pv.p, nullptr, nullptr, 0.0, h.q.p,
                                         nullptr, nullptr, s);
            dot(h.pv.p, h.q.p, n, sc + 10, s, part);
            RN_LAUNCH("outer_cg_scalar", 0, s, cg_alpha_kernel, 1, 1, 0, sc);
            RN_LAUNCH("outer_cg_vec", 56.0 * n, s, cg_xr_kernel, rg, kS, 0, n, x, h.r.p, h.pv.p, h.q.p,
                      flexible ? h.rold.p : nullptr, sc, part);
            reduce_partials(part, rg, sc + 8, s);
            rn = norm_from(sc + 8, s);
            if (rn / nb < rtol) { st = RN_OK; break; }
            apply_cycle(h, h.r.p, h.z.p);
            RN_LAUNCH("outer_cg_vec", 24.0 * n, s, cg_rz_kernel, rg, kS, 0, n, h.r.p, h.z.p,
                      flexible ? h.rold.p : nullptr, part);
            reduce_partials(part, rg, sc + 9, s);
            if (flexible) reduce_partials(part + kReduceBlocks, rg, sc + 11, s);
            RN_LAUNCH("outer_cg_scalar", 0, s, cg_beta_kernel, 1, 1, 0, sc, flexible ? 1 : 0);
            RN_LAUNCH("outer_cg_vec", 24.0 * n, s, cg_p_kernel, eg, 256, 0, n, h.pv.p, h.z.p, sc, 0);
        }
        if (it > maxit) it = maxit;
        spmv_launch<double, OP_RESID>("outer_residual", L0.A, L0.spmv_group, x, b, nullptr, 0.0, h.r.p, part, &grid,
                                      s);
        reduce_partials(part, grid, sc + 8, s);
        rn = norm_from(sc + 8, s);
        st = (rn / nb < rtol) ? RN_OK : RN_ENOTCONV;
    } else if (st != RN_OK && h.p.outer == RN_OUTER_FGMRES) {
        const int m = std::max(1, h.p.restart);
        double *H = h.H.p, *cs = H + (m + 1) * m, *sn = cs + (m + 1), *g = sn + (m + 1), *y = g + (m + 1);
        it = 0;
        while (it < maxit && st != RN_OK) {
            // r = b - A x, V0 = r / ||r||
            spmv_launch<double, OP_RESID>("outer_residual", L0.A, L0.spmv_group, x, b, nullptr, 0.0, h.r.p, part,
                                          &grid, s);
            reduce_partials(part, grid, sc + 8, s);
            rn = norm_from(sc + 8, s);
            if (rn / nb < rtol) { st = RN_OK; break; }
            RN_LAUNCH("outer_gmres_scalar", 0, s, fg_start_kernel, 1, 1, 0, g, m, sc);
            RN_LAUNCH("outer_gmres_vec", 16.0 * n, s, scale_copy_kernel, eg, 256, 0, n, h.r.p, sc + 8, h.V.p, 1);
            int k = 0;
            for (int j = 0; j < m && it < maxit; j++) {
                double *vj = h.V.p + (int64_t)j * n, *zj = h.Z.p + (int64_t)j * n;
                apply_cycle(h, vj, zj);
                spmv_launch<double, OP_SPMV>("outer_spmv", L0.A, L0.spmv_group, zj, nullptr, nullptr, 0.0, h.w.p,
                                             nullptr, nullptr, s);
                for (int i = 0; i <= j; i++) {
                    double *vi = h.V.p + (int64_t)i * n;
                    dot(h.w.p, vi, n, H + i * m + j, s, part);
                    RN_LAUNCH("outer_gmres_vec", 24.0 * n, s, axpy_dev_kernel, eg, 256, 0, n, h.w.p, vi,
                              H + i * m + j);
                }
                dot(h.w.p, h.w.p, n, sc + 8, s, part);
                RN_LAUNCH("outer_gmres_scalar", 0, s, fg_givens_kernel, 1, 1, 0, m, j, H, cs, sn, g, sc);
                it++;
                k = j + 1;
                double res[2];
                RN_CUDA_CHECK(cudaMemcpyAsync(res, sc + 15, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
                RN_CUDA_CHECK(cudaStreamSynchronize(s));
                if (res[0] / nb < rtol || res[1] == 0.0) break;
                RN_LAUNCH("outer_gmres_vec", 16.0 * n, s, scale_copy_kernel, eg, 256, 0, n, h.w.p, sc + 16,
                          h.V.p + (int64_t)(j + 1) * n, 0);
            }
            RN_LAUNCH("outer_gmres_scalar", 0, s, fg_backsolve_kernel, 1, 1, 0, m, k, H, g, y);
            RN_LAUNCH("outer_gmres_vec", (8.0 * k + 16.0) * n, s, fg_update_kernel, eg, 256, 0, n, k, x, h.Z.p, y);
            spmv_launch<double, OP_RESID>("outer_residual", L0.A, L0.spmv_group, x, b, nullptr, 0.0, h.r.p, part,
                                          &grid, s);
            reduce_partials(part, grid, sc + 8, s);
            rn = norm_from(sc + 8, s);
            if (rn / nb < rtol) st = RN_OK;
        }
    } else if (st != RN_OK) {
        fail(RN_EINVAL, "unknown outer iteration");
    }
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    if (info) {
        info->iters = it;
        info->rel_res = rn / nb;
        info->rho = (it > 0 && r0 > 0.0) ? std::pow(rn / r0, 1.0 / it) : 0.0;
        info->solve_ms = now_ms() - t0;
        info->status = st;
    }
    return st;
}

}  // namespace rn
