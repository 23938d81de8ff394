// rn_solve.cu - V(nu_pre, nu_post) cycle (Sec. 2, eq. twogrid applied
// recursively) and the outer iterations.
//
// The cycle is a fixed sequence of launches per level - weighted Jacobi,
// residual, restriction R r, recursion, prolongation x += P x_c, weighted
// Jacobi - ending in a dense solve x = A_L^{-1} b on the coarsest level.  All
// sizes are fixed after setup, so one application of the cycle is captured
// in a CUDA graph and replayed.  In mixed precision the cycle runs on FP32
// shadows of A, P, R and the diagonal; the outer iteration (residual, Krylov
// vectors, dot products) and the coarsest solve stay FP64, and the level-0
// kernels read the FP64 right-hand side and write the FP64 result directly.
//
// The SpMV family (TMA-staged tiles) is in rn_spmv.cuh.
#include <algorithm>
#include <cmath>

#include <functional>
#include <tuple>
#include <mutex>
#include <map>

#include "rn_hier.cuh"
#include "rn_spmv.cuh"

namespace rn {

template <typename T, typename TB>
__global__ void jacobi_zero_kernel(int32_t n, const TB *__restrict__ b, const T *__restrict__ diag, T omega,
                                   T *__restrict__ y) {
    pdl_wait();
    pdl_trigger();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = diag[i] * (T)b[i];  // diag holds omega / a_ii
}

// x = A_L^{-1} b on the coarsest level (FP64 arithmetic), warp per row
template <typename TB, typename TO>
__global__ void coarse_solve_kernel(int32_t n, const double *__restrict__ Ainv, const TB *__restrict__ b,
                                    TO *__restrict__ x) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        double acc = 0.0;
        for (int32_t j = lane; j < n; j += 32) acc = fma(Ainv[(int64_t)i * n + j], (double)b[j], acc);
        acc = warp_sum(acc);
        if (lane == 0) x[i] = (TO)acc;
    }
}

// x = blockdiag(A_p^{-1}) b for independent problems merged into one
// hierarchy: block p holds rows [ro[p], ro[p+1]) and its row-major inverse at
// Ainv + ao[p]; warp per row with the lane order of coarse_solve_kernel, so
// each block's result is bit-identical to solving that problem alone.
template <typename TB, typename TO>
__global__ void coarse_solve_blocks_kernel(int nblk, const int32_t *__restrict__ ro, const int64_t *__restrict__ ao,
                                           const double *__restrict__ Ainv, const TB *__restrict__ b,
                                           TO *__restrict__ x) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int32_t ntot = ro[nblk];
    for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < ntot; i += (gridDim.x * blockDim.x) >> 5) {
        int lo = 0, hi = nblk - 1;  // the block of row i: the largest p with ro[p] <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ro[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int32_t r0 = ro[lo], n = ro[lo + 1] - r0;
        const double *Ai = Ainv + ao[lo] + (int64_t)(i - r0) * n;
        double acc = 0.0;
        for (int32_t j = lane; j < n; j += 32) acc = fma(Ai[j], (double)b[r0 + j], acc);
        acc = warp_sum(acc);
        if (lane == 0) x[i] = (TO)acc;
    }
}

__global__ void f2d_kernel(int64_t n, const float *__restrict__ x, double *__restrict__ y) {
    pdl_wait();
    pdl_trigger();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

__global__ void row_maxlen_kernel(int32_t n, const int32_t *__restrict__ rp, int32_t *__restrict__ out) {
    pdl_wait();
    int32_t m = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, rp[i + 1] - rp[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ------------------------------------------------------------------ outer-iteration vector kernels
// Scalars live on the device (see Fin); alpha and beta are formed once by the
// finisher of the reduction that completes them, not per thread (FP64 division
// is a long sequence on this part's narrow FP64 pipe).  The level-0 vector
// kernels give each thread kVecU elements a grid stride apart, loaded before
// any is used.
constexpr int kVecU = 4;

__global__ void axpy_kernel(int64_t n, double *__restrict__ x, const double *__restrict__ z) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += z[i];
}

// x += alpha p; r_old = r (flexible); r -= alpha q; ||r||^2 (FIN_XR: stopping test);
// and, when x0 is given, the next cycle's first-sweep iterate x0 = w (XT) r
// (w = omega / a_ii on level 0), exactly as jacobi_zero_kernel forms it.
template <typename XT>
__global__ void __launch_bounds__(kS)
cg_xr_kernel(int64_t n, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
             const double *__restrict__ q, double *__restrict__ rold, const double *__restrict__ sc,
             const XT *__restrict__ w, XT *__restrict__ x0, Fin fin) {
    __shared__ double sm[32];
    pdl_wait();
    pdl_trigger();
    const double a = sc[12];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc[1] = {0.0};
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecU * stride) {
        double xv[kVecU], pv[kVecU], rv[kVecU], qv[kVecU];
#pragma unroll
        for (int u = 0; u < kVecU; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                xv[u] = x[i];
                pv[u] = p[i];
                rv[u] = r[i];
                qv[u] = q[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVecU; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                x[i] = xv[u] + a * pv[u];
                if (rold) rold[i] = rv[u];
                const double rn = rv[u] - a * qv[u];
                r[i] = rn;
                if (x0) x0[i] = w[i] * (XT)rn;
                acc[0] = fma(rn, rn, acc[0]);
            }
        }
    }
    grid_finish<kS, 1>(acc, fin, sm);
}

// <r,z> and (flexible) <z, r_old>; the finisher keeps the previous <r,z> and forms beta
__global__ void __launch_bounds__(kS)
cg_rz_kernel(int64_t n, const double *__restrict__ r, const double *__restrict__ z, const double *__restrict__ rold,
             Fin fin) {
    __shared__ double sm[32];
    pdl_wait();
    pdl_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc[2] = {0.0, 0.0};
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecU * stride) {
        double rv[kVecU], zv[kVecU], ov[kVecU];
#pragma unroll
        for (int u = 0; u < kVecU; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                rv[u] = r[i];
                zv[u] = z[i];
                ov[u] = rold ? rold[i] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < kVecU; u++) {
            if (i0 + u * stride < n) {
                acc[0] = fma(rv[u], zv[u], acc[0]);
                if (rold) acc[1] = fma(zv[u], ov[u], acc[1]);
            }
        }
    }
    grid_finish<kS, 2>(acc, fin, sm);
}

// p = z (first) or z + beta p, beta = sc[13]
__global__ void __launch_bounds__(kS)
cg_p_kernel(int64_t n, double *__restrict__ p, const double *__restrict__ z, const double *__restrict__ sc,
            int first) {
    pdl_wait();
    pdl_trigger();
    const double beta = sc[13];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecU * stride) {
        double zv[kVecU], pv[kVecU];
#pragma unroll
        for (int u = 0; u < kVecU; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                zv[u] = z[i];
                pv[u] = first ? 0.0 : p[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVecU; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) p[i] = first ? zv[u] : zv[u] + beta * pv[u];
        }
    }
}

// Solve-path launches: with programmatic dependent launch when the hierarchy
// uses it (every kernel launched this way calls pdl_wait first).
#define RN_SLAUNCH(h, name, bytes, stream, kernel, grid, block, smem, ...)              \
    do {                                                                                 \
        if ((h).pdl) RN_LAUNCH_PDL(name, bytes, stream, kernel, grid, block, smem, __VA_ARGS__); \
        else RN_LAUNCH(name, bytes, stream, kernel, grid, block, smem, __VA_ARGS__);     \
    } while (0)

// one wave of resident blocks for the level-0 vector kernels
static int vec_grid(const void *k, int64_t n) {
    const int64_t need = (n + (int64_t)kS * kVecU - 1) / ((int64_t)kS * kVecU);
    const int64_t wave = (int64_t)resident_blocks(k, kS, 0) * num_sms();
    return (int)std::max<int64_t>(1, std::min<int64_t>({need, wave, (int64_t)kReduceBlocks}));
}

#define VG(kernel) vec_grid((const void *)(kernel), n)

// loop state of the outer CG: ||b||, rtol, iteration count and limit
__global__ void cg_loop_init_kernel(double *sc, int32_t *fl, double nb, double rtol, int maxit) {
    pdl_wait();
    sc[18] = nb;
    sc[19] = rtol;
    fl[9] = 0;
    fl[10] = maxit;
    fl[11] = 0;
}

__global__ void scale_copy_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ den,
                                  double *__restrict__ y, int sqrt_den) {
    pdl_wait();
    const double d = sqrt_den ? sqrt(*den) : *den;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] / d;
}

// FGMRES Givens step on column j (H row-major (m+1) x m); g rhs; |g_{j+1}| -> sc[15]
__global__ void fg_givens_kernel(int m, int j, double *H, double *cs, double *sn, double *g, double *sc) {
    pdl_wait();
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
    pdl_wait();
    const double beta = sqrt(sc[8]);
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
}

__global__ void fg_backsolve_kernel(int m, int k, const double *H, const double *g, double *y) {
    pdl_wait();
    for (int i = k - 1; i >= 0; i--) {
        double s = g[i];
        for (int j = i + 1; j < k; j++) s -= H[i * m + j] * y[j];
        y[i] = s / H[i * m + i];
    }
}

__global__ void fg_update_kernel(int64_t n, int k, double *__restrict__ x, const double *__restrict__ Z,
                                 const double *__restrict__ y) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = x[i];
        for (int j = 0; j < k; j++) v = v + y[j] * Z[(int64_t)j * n + i];
        x[i] = v;
    }
}

// ================================================================== host side
static Fin make_fin(rn_hierarchy &h, int mode, double *out = nullptr) {
    Fin f;
    f.mode = mode;
    f.partial = h.partial.p;
    f.counter = h.counters.p;
    f.out = out;
    f.sc = h.scal.p;
    f.fl = h.iflags.p;
    return f;
}

// lanes per row so that a tile (256/G rows) fits one stage; 0 = rows too long
static int tile_group(int32_t maxlen, int nnz_per_stage) {
    for (int G = 1; G <= 32; G *= 2)
        if ((int64_t)(kS / G) * maxlen <= nnz_per_stage) return G;
    return 0;
}
static int fallback_group(double avg) {
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

template <typename T, typename TB, typename TO, int G, int OP, bool TL>
static void launch_tile_t(const char *name, double bytes, const DCsr &M, const T *x, const TB *b, const T *diag,
                          T omega, TO *y, T *xz, const double *aux, const Fin &fin, int32_t *err, cudaStream_t s,
                          bool pdl, const int32_t *tlist, const int32_t *tcount) {
    constexpr int SL = tile_nnz<T>() + kTileSlack;
    constexpr int RL = kS / G + 8;
    const size_t smem = (2 * SL + 2 * RL) * sizeof(int32_t) + 2 * SL * sizeof(T);
    static const bool configured = [&] {  // once per instantiation (thread-safe static initialisation)
        RN_CUDA_CHECK(cudaFuncSetAttribute(spmv_tile_kernel<T, TB, TO, G, OP, TL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return true;
    }();
    (void)configured;
    const int32_t ntiles = (M.n + (kS / G) - 1) / (kS / G);
    const int per_sm = sizeof(T) == 8 ? 3 : 4;  // CTAs that fit one SM's shared memory
    int grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * per_sm);
    grid = std::max(1, std::min(grid, kReduceBlocks));
    struct {
        bool pdl;
    } hh{pdl};
    RN_SLAUNCH(hh, name, bytes, s, (spmv_tile_kernel<T, TB, TO, G, OP, TL>), grid, kS, smem, M.n, ntiles,
               M.rowptr.p, M.col.p, vals_of<T>(M), x, b, diag, omega, y, xz, aux, fin, err, tlist, tcount);
}

// Merged independent problems list the tiles that hold rows of problems still
// iterating; the other matrices (and the fused-reduction operations, which
// the merged solve does not use) run every tile.
template <typename T, typename TB, typename TO, int G, int OP>
static void launch_tile(const char *name, double bytes, const DCsr &M, const T *x, const TB *b, const T *diag,
                        T omega, TO *y, T *xz, const double *aux, const Fin &fin, int32_t *err, cudaStream_t s,
                        bool pdl) {
    constexpr bool f64 = sizeof(T) == 8;
    const int32_t *tlist = f64 ? M.tl64.p : M.tl32.p;
    if constexpr (OP != OP_SPMV_DOT && OP != OP_JACOBI_RZ) {
        if (tlist) {
            launch_tile_t<T, TB, TO, G, OP, true>(name, bytes, M, x, b, diag, omega, y, xz, aux, fin, err, s, pdl,
                                                  tlist, M.tcnt.p + (f64 ? 1 : 0));
            return;
        }
    } else {
        if (tlist) fail(RN_EINTERNAL, "tile lists are not used with fused reductions");
    }
    launch_tile_t<T, TB, TO, G, OP, false>(name, bytes, M, x, b, diag, omega, y, xz, aux, fin, err, s, pdl, nullptr,
                                           nullptr);
}

template <typename T, typename TB, typename TO, int G, int OP>
static void launch_group(const char *name, double bytes, const DCsr &M, const T *x, const TB *b, const T *diag,
                         T omega, TO *y, T *xz, const double *aux, const Fin &fin, cudaStream_t s, bool pdl) {
    int grid = grid_for(M.n, kS / G, 8);
    grid = std::min(grid, kReduceBlocks);
    struct {
        bool pdl;
    } hh{pdl};
    RN_SLAUNCH(hh, name, bytes, s, (spmv_group_kernel<T, TB, TO, G, OP>), grid, kS, 0, M.n, M.rowptr.p, M.col.p,
               vals_of<T>(M), x, b, diag, omega, y, xz, aux, fin);
}

// Algorithmic bytes of one SpMV-family launch: the matrix (index + value) and
// row pointers once, x gathered once, the output (and b, diag, x_i where
// read) once.
template <typename T, typename TB, typename TO, int OP>
static double spmv_bytes(const DCsr &M) {
    const double vb = sizeof(T);
    double bytes = (4.0 + vb) * M.nnz + 4.0 * (M.n + 1) + vb * M.m + (double)sizeof(TO) * M.n;
    if (OP == OP_SPMV_ADD) bytes += sizeof(TO) * (double)M.n;
    if (OP == OP_RESID) bytes += sizeof(TB) * (double)M.n;
    if (OP == OP_JACOBI) bytes += (sizeof(TB) + vb) * (double)M.n;
    if (OP == OP_JACOBI_RZ) bytes += (sizeof(TB) + vb) * (double)M.n;  // + r_old when flexible (not counted)
    if (OP == OP_JZ_RESID) bytes += (sizeof(TB) + 2.0 * vb) * (double)M.n - vb * M.m;  // b, d read; x written
    return bytes;
}

// y = op(M, x, b): picks the staged tile kernel when the rows fit a stage.
// xz: second output of OP_JZ_RESID (the relaxed iterate).
template <typename T, typename TB, typename TO, int OP>
static void spmv(rn_hierarchy &h, const char *name, const DCsr &M, const T *x, const TB *b, const T *diag, T omega,
                 TO *y, const Fin &fin, T *xz = nullptr, const double *aux = nullptr) {
    cudaStream_t s = h.s;
    if (M.n == 0) return;
    const double bytes = spmv_bytes<T, TB, TO, OP>(M);
    int32_t *err = h.iflags.p + 8;
    const int G = sizeof(T) == 8 ? M.tile_group64 : M.tile_group;
#define RN_TILE_CASE(GG) \
    case GG: launch_tile<T, TB, TO, GG, OP>(name, bytes, M, x, b, diag, omega, y, xz, aux, fin, err, s, h.pdl); return;
#define RN_GROUP_CASE(GG) \
    case GG: launch_group<T, TB, TO, GG, OP>(name, bytes, M, x, b, diag, omega, y, xz, aux, fin, s, h.pdl); return;
    switch (G) {
        RN_TILE_CASE(1)
        RN_TILE_CASE(2)
        RN_TILE_CASE(4)
        RN_TILE_CASE(8)
        RN_TILE_CASE(16)
        RN_TILE_CASE(32)
        default: break;
    }
    switch (fallback_group(M.n ? (double)M.nnz / M.n : 1.0)) {
        RN_GROUP_CASE(2)
        RN_GROUP_CASE(4)
        RN_GROUP_CASE(8)
        RN_GROUP_CASE(16)
        default: launch_group<T, TB, TO, 32, OP>(name, bytes, M, x, b, diag, omega, y, xz, aux, fin, s, h.pdl); return;
    }
#undef RN_TILE_CASE
#undef RN_GROUP_CASE
}

template <typename T>
struct LevelBufs;
template <>
struct LevelBufs<double> {
    static double *b(rn_level &L) { return L.b.p; }
    static double *x(rn_level &L) { return L.x.p; }
    static double *t(rn_level &L) { return L.t.p; }
    static double *r(rn_level &L) { return L.r.p; }
    static const double *d(rn_level &L) { return L.wd.p; }  // omega / a_ii
};
template <>
struct LevelBufs<float> {
    static float *b(rn_level &L) { return L.b32.p; }
    static float *x(rn_level &L) { return L.x32.p; }
    static float *t(rn_level &L) { return L.t32.p; }
    static float *r(rn_level &L) { return L.r32.p; }
    static const float *d(rn_level &L) { return L.wd32.p; }  // omega / a_ii
};

struct CycleNames {
    const char *jacobi, *jacobi0, *resid, *jzresid, *restr, *prolong, *coarse;
};
static const CycleNames kNames[2][2] = {
    // [precision: 0 f64, 1 f32][level: 0 finest, 1 coarser]
    {{"cycle_jacobi_f64_L0", "cycle_jacobi0_f64_L0", "cycle_residual_f64_L0", "cycle_relax0_residual_f64_L0",
      "cycle_restrict_f64_L0", "cycle_prolong_f64_L0", "cycle_coarse_solve"},
     {"cycle_jacobi_f64_Lc", "cycle_jacobi0_f64_Lc", "cycle_residual_f64_Lc", "cycle_relax0_residual_f64_Lc",
      "cycle_restrict_f64_Lc", "cycle_prolong_f64_Lc", "cycle_coarse_solve"}},
    {{"cycle_jacobi_f32_L0", "cycle_jacobi0_f32_L0", "cycle_residual_f32_L0", "cycle_relax0_residual_f32_L0",
      "cycle_restrict_f32_L0", "cycle_prolong_f32_L0", "cycle_coarse_solve"},
     {"cycle_jacobi_f32_Lc", "cycle_jacobi0_f32_Lc", "cycle_residual_f32_Lc", "cycle_relax0_residual_f32_Lc",
      "cycle_restrict_f32_Lc", "cycle_prolong_f32_Lc", "cycle_coarse_solve"}}};

// Pre-relaxation from a zero guess followed by the residual on one level:
// returns the iterate buffer; r receives b - A x.  With one pre-sweep both
// happen in one fused pass.
template <typename T, typename TB>
static T *relax0_and_residual(rn_hierarchy &h, const CycleNames &nm, rn_level &L, const TB *b, T *r,
                               bool x0_ready = false) {
    using LB = LevelBufs<T>;
    cudaStream_t s = h.s;
    const int32_t n = L.A.n;
    const T omega = (T)h.p.omega;
    const T *d = LB::d(L);
    T *cur = LB::x(L), *oth = LB::t(L);
    const Fin none;
    if (h.p.nu_pre == 1) {
        if (sizeof(TB) == 8) {
            // level 0 (FP64 right-hand side): x = (omega / a_ii) b is formed once per row (by the
            // outer CG's update when x0_ready), so the residual gathers plain T values - no
            // FP64 conversion or product per gathered entry on the narrow FP64 pipe
            if (!x0_ready)
                RN_SLAUNCH(h, nm.jacobi0, (sizeof(TB) + 2.0 * sizeof(T)) * n, s, (jacobi_zero_kernel<T, TB>),
                           grid_for(n, 1024), 256, 0, n, b, d, omega, cur);
            spmv<T, TB, T, OP_RESID>(h, nm.resid, L.A, cur, b, nullptr, T(0), r, none);
            return cur;
        }
        spmv<T, TB, T, OP_JZ_RESID>(h, nm.jzresid, L.A, (const T *)nullptr, b, d, omega, r, none, cur);
        return cur;
    }
    for (int k = 0; k < h.p.nu_pre; k++) {
        if (k == 0) {
            RN_SLAUNCH(h, nm.jacobi0, (sizeof(TB) + 2.0 * sizeof(T)) * n, s, (jacobi_zero_kernel<T, TB>),
                      grid_for(n, 1024), 256, 0, n, b, d, omega, cur);
        } else {
            spmv<T, TB, T, OP_JACOBI>(h, nm.jacobi, L.A, cur, b, d, omega, oth, none);
            std::swap(cur, oth);
        }
    }
    if (h.p.nu_pre == 0) RN_CUDA_CHECK(cudaMemsetAsync(cur, 0, sizeof(T) * n, s));
    spmv<T, TB, T, OP_RESID>(h, nm.resid, L.A, cur, b, nullptr, T(0), r, none);
    return cur;
}

template <typename T>
static T *vcycle_level(rn_hierarchy &h, int l);

// Coarse-grid corrections on level l: gamma (1 V-cycle, 2 W-cycle), but one
// when level l+1 is the coarsest: its exact solve leaves R (b - A x) = 0.
static int corrections(const rn_hierarchy &h, int l) {
    return l + 2 >= (int)h.lev.size() ? 1 : h.p.gamma;
}

// Coarse-grid correction of level l: b_{l+1} = R_l r, the cycle on level
// l+1, cur += P_l x_{l+1}.  From the cluster's level on, all of it (transfers
// included) is one cluster launch.
template <typename T>
static void coarse_correction(rn_hierarchy &h, int l, const T *r, T *cur) {
    using LB = LevelBufs<T>;
    rn_level &L = *h.lev[l];
    rn_level &Lc = *h.lev[l + 1];
    const CycleNames &nm = kNames[sizeof(T) == 4][l > 0];
    const Fin none;
    if (h.sub_k == l) {
        launch_subcycle<T>(h, cur, sizeof(T) == 4 ? "cycle_coarse_cluster_f32" : "cycle_coarse_cluster_f64");
        return;
    }
    spmv<T, T, T, OP_SPMV>(h, nm.restr, L.R, r, (const T *)nullptr, nullptr, T(0), LB::b(Lc), none);
    T *xc = vcycle_level<T>(h, l + 1);
    spmv<T, T, T, OP_SPMV_ADD>(h, nm.prolong, L.P, xc, (const T *)nullptr, nullptr, T(0), cur, none);
}

// One cycle on level l >= 1 with zero initial guess; b_l holds the right-hand
// side.  Returns the buffer holding the result.
template <typename T>
static T *vcycle_level(rn_hierarchy &h, int l) {
    using LB = LevelBufs<T>;
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[l];
    const CycleNames &nm = kNames[sizeof(T) == 4][1];
    const int32_t n = L.A.n;
    T *b = LB::b(L);
    const Fin none;
    if (l == (int)h.lev.size() - 1) {
        T *x = LB::x(L);
        if (h.ncblk > 0)
            RN_SLAUNCH(h, nm.coarse, 8.0 * h.Ainv.n + 2.0 * sizeof(T) * n, s, (coarse_solve_blocks_kernel<T, T>),
                       grid_for((int64_t)n * 32, 256, 4), 256, 0, h.ncblk, h.cblk_row.p, h.cblk_inv.p, h.Ainv.p, b, x);
        else
            RN_SLAUNCH(h, nm.coarse, 8.0 * n * n + 2.0 * sizeof(T) * n, s, (coarse_solve_kernel<T, T>),
                       grid_for((int64_t)n * 32, 256, 4), 256, 0, n, h.Ainv.p, b, x);
        return x;
    }
    const T omega = (T)h.p.omega;
    const T *d = LB::d(L);
    T *r = LB::r(L);
    T *cur = relax0_and_residual<T, T>(h, nm, L, b, r);
    T *oth = (cur == LB::x(L)) ? LB::t(L) : LB::x(L);
    coarse_correction<T>(h, l, r, cur);
    for (int c = 1; c < corrections(h, l); c++) {  // W-cycle: correct again from the new residual
        spmv<T, T, T, OP_RESID>(h, nm.resid, L.A, cur, b, nullptr, T(0), r, none);
        coarse_correction<T>(h, l, r, cur);
    }
    for (int k = 0; k < h.p.nu_post; k++) {
        spmv<T, T, T, OP_JACOBI>(h, nm.jacobi, L.A, cur, b, d, omega, oth, none);
        std::swap(cur, oth);
    }
    return cur;
}

// out = M rhs on level 0 (FP64 in/out); the cycle itself runs in T.  With rz
// set, the last post-sweep also reduces the outer CG's <rhs, out> and
// <out, rz_rold> into *rz (FIN_RZ); returns whether it did (it cannot without
// a post-sweep on a multilevel hierarchy).
template <typename T>
static bool vcycle_top(rn_hierarchy &h, const double *rhs, double *out, const Fin *rz, const double *rz_rold,
                       bool x0_ready) {
    using LB = LevelBufs<T>;
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[0];
    const CycleNames &nm = kNames[sizeof(T) == 4][0];
    const int32_t n = L.A.n;
    const Fin none;
    if (h.lev.size() == 1) {
        if (h.ncblk > 0)
            RN_SLAUNCH(h, nm.coarse, 8.0 * h.Ainv.n + 16.0 * n, s, (coarse_solve_blocks_kernel<double, double>),
                       grid_for((int64_t)n * 32, 256, 4), 256, 0, h.ncblk, h.cblk_row.p, h.cblk_inv.p, h.Ainv.p,
                       rhs, out);
        else
            RN_SLAUNCH(h, nm.coarse, 8.0 * n * n + 16.0 * n, s, (coarse_solve_kernel<double, double>),
                       grid_for((int64_t)n * 32, 256, 4), 256, 0, n, h.Ainv.p, rhs, out);
        return false;
    }
    const T omega = (T)h.p.omega;
    const T *d = LB::d(L);
    T *r = LB::r(L);
    T *cur = relax0_and_residual<T, double>(h, nm, L, rhs, r, x0_ready);
    T *oth = (cur == LB::x(L)) ? LB::t(L) : LB::x(L);
    coarse_correction<T>(h, 0, r, cur);
    for (int c = 1; c < corrections(h, 0); c++) {
        spmv<T, double, T, OP_RESID>(h, nm.resid, L.A, cur, rhs, nullptr, T(0), r, none);
        coarse_correction<T>(h, 0, r, cur);
    }
    const int npost = h.p.nu_post;
    for (int k = 0; k < npost; k++) {
        if (k == npost - 1) {
            if (rz) {
                spmv<T, double, double, OP_JACOBI_RZ>(h, nm.jacobi, L.A, cur, rhs, d, omega, out, *rz, nullptr,
                                                      rz_rold);
                return true;
            }
            spmv<T, double, double, OP_JACOBI>(h, nm.jacobi, L.A, cur, rhs, d, omega, out, none);
            return false;
        }
        spmv<T, double, T, OP_JACOBI>(h, nm.jacobi, L.A, cur, rhs, d, omega, oth, none);
        std::swap(cur, oth);
    }
    // no post-smoothing: copy the iterate out
    if (sizeof(T) == 8) d2d(out, reinterpret_cast<const double *>(cur), n, s);
    else RN_SLAUNCH(h, "convert", 12.0 * n, s, f2d_kernel, grid_for(n, 1024), 256, 0, (int64_t)n,
                   reinterpret_cast<const float *>(cur), out);
    return false;
}

// x0_ready: level 0's first-sweep iterate (omega / a_ii) rhs is already in its
// buffer (written by the outer CG's update of rhs).
static bool cycle_direct(rn_hierarchy &h, const double *rhs, double *out, const Fin *rz = nullptr,
                         const double *rz_rold = nullptr, bool x0_ready = false) {
    if (h.p.precision == RN_MIXED) return vcycle_top<float>(h, rhs, out, rz, rz_rold, x0_ready);
    return vcycle_top<double>(h, rhs, out, rz, rz_rold, x0_ready);
}

// Whether the outer CG's update forms level 0's first-sweep iterate.
static bool cg_forms_x0(const rn_hierarchy &h) { return h.p.nu_pre == 1 && h.lev.size() > 1; }

void cycle_launches(rn_hierarchy &h, const double *rhs, double *out) { cycle_direct(h, rhs, out); }

void outer_spmv(rn_hierarchy &h, const double *x, double *y) {
    spmv<double, double, double, OP_SPMV>(h, "outer_spmv", h.lev[0]->A, x, (const double *)nullptr, nullptr, 0.0, y,
                                          Fin());
}

void outer_residual(rn_hierarchy &h, const double *x, const double *b, double *r) {
    spmv<double, double, double, OP_RESID>(h, "outer_residual", h.lev[0]->A, x, b, nullptr, 0.0, r, Fin());
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

// Longest row of M into *slot (one launch; the caller reads all slots at once).
static void launch_maxlen(rn_hierarchy &h, const DCsr &M, int32_t *slot) {
    if (M.n == 0) return;
    RN_LAUNCH("prepare", 4.0 * M.n, h.s, row_maxlen_kernel, grid_for(M.n, 1024), 256, 0, M.n, M.rowptr.p, slot);
}

static void set_tile_group(DCsr &M, int32_t maxlen) {
    if (M.n == 0) return;
    M.maxlen = maxlen;
    M.tile_group = tile_group(M.maxlen, tile_nnz<float>());
    M.tile_group64 = tile_group(M.maxlen, tile_nnz<double>());
}

__global__ void omega_over_diag_kernel(int64_t n, double omega, const double *__restrict__ d,
                                       double *__restrict__ wd, float *__restrict__ wd32) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = omega / d[i];
        wd[i] = w;
        if (wd32) wd32[i] = (float)w;
    }
}

// ------------------------------------------------------------------ schedule autotuner
// The staged SpMV's schedule for a matrix is its lanes per row G (a tile is
// 256/G rows): the threshold rule takes the smallest G whose tile fits one
// shared-memory stage (set_tile_group).  With params.autotune the candidates
// - that G, every larger power of two up to 32, and the unstaged group kernel
// (0; not for a merged batch, whose staged tiles carry the lists that skip
// converged problems) - are timed on the matrix itself (y = M x on the level's
// vectors: one untimed launch, then five timed by CUDA events, the fastest
// kept) and a candidate replaces the threshold's G only when it is at least 5%
// faster; the choice is cached for the process per (rows, columns, entries,
// longest row, value type, merged or not), so later hierarchies of the same
// shapes take it without trials.
static void check_tile_error(rn_hierarchy &h);

using TuneKey = std::tuple<int32_t, int32_t, int64_t, int32_t, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;

template <typename T>
static void tune_matrix(rn_hierarchy &h, DCsr &M, const T *x, T *y) {
    if (M.n == 0 || M.nnz == 0) return;
    int &group = sizeof(T) == 8 ? M.tile_group64 : M.tile_group;
    const bool merged = h.ncblk > 0;
    const TuneKey key{M.n, M.m, M.nnz, M.maxlen, (int)sizeof(T), merged ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            group = it->second;
            return;
        }
    }
    std::vector<int> cand;
    if (group > 0)
        for (int G = group; G <= 32; G *= 2) cand.push_back(G);
    if (!merged || group == 0) cand.push_back(0);  // the unstaged kernel
    cudaStream_t s = h.s;
    cudaEvent_t ev[2];
    RN_CUDA_CHECK(cudaEventCreate(&ev[0]));
    RN_CUDA_CHECK(cudaEventCreate(&ev[1]));
    const int thr = group;
    int best = group;
    float best_ms = 1e30f, thr_ms = 1e30f;
    try {
        for (int G : cand) {
            group = G;
            spmv<T, T, T, OP_SPMV>(h, "autotune", M, x, (const T *)nullptr, nullptr, T(0), y, Fin());
            float tmin = 1e30f;
            for (int r = 0; r < 5; r++) {
                float t = 0.f;
                RN_CUDA_CHECK(cudaEventRecord(ev[0], s));
                spmv<T, T, T, OP_SPMV>(h, "autotune", M, x, (const T *)nullptr, nullptr, T(0), y, Fin());
                RN_CUDA_CHECK(cudaEventRecord(ev[1], s));
                RN_CUDA_CHECK(cudaEventSynchronize(ev[1]));
                RN_CUDA_CHECK(cudaEventElapsedTime(&t, ev[0], ev[1]));
                tmin = std::min(tmin, t);
            }
            if (G == thr) thr_ms = tmin;
            if (tmin < best_ms) {
                best_ms = tmin;
                best = G;
            }
        }
        if (best != thr && !(best_ms < 0.95f * thr_ms)) best = thr;  // only a clear win replaces the rule
    } catch (...) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        throw;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    check_tile_error(h);
    group = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
}

// every level's A, P and R in the cycle's value type, and level 0's A in FP64
// (the outer iteration's SpMV)
static void autotune_schedules(rn_hierarchy &h) {
    const bool mixed = h.p.precision == RN_MIXED;
    for (size_t l = 0; l < h.lev.size(); l++) {
        rn_level &L = *h.lev[l];
        const bool last = l + 1 == h.lev.size();
        if (mixed) {
            tune_matrix<float>(h, L.A, L.x32.p, L.t32.p);
            if (!last) {
                tune_matrix<float>(h, L.P, h.lev[l + 1]->x32.p, L.t32.p);
                tune_matrix<float>(h, L.R, L.t32.p, h.lev[l + 1]->b32.p);
            }
        }
        if (!mixed || l == 0) tune_matrix<double>(h, L.A, L.x.p, L.t.p);
        if (!mixed && !last) {
            tune_matrix<double>(h, L.P, h.lev[l + 1]->x.p, L.t.p);
            tune_matrix<double>(h, L.R, L.t.p, h.lev[l + 1]->b.p);
        }
    }
}

// The solve's preparation in two halves, so that many hierarchies can enqueue
// the first before any of them waits for its read-back: the longest rows of
// every level's A, P and R (begin), then their read and the rest (end).
void prepare_solve_begin(rn_hierarchy &h) {
    cudaStream_t s = h.s;
    const size_t nmat = 3 * h.lev.size();
    h.maxlen.alloc(nmat, s);
    RN_CUDA_CHECK(cudaMemsetAsync(h.maxlen.p, 0, h.maxlen.bytes(), s));
    for (size_t l = 0; l < h.lev.size(); l++) {
        launch_maxlen(h, h.lev[l]->A, h.maxlen.p + 3 * l);
        launch_maxlen(h, h.lev[l]->P, h.maxlen.p + 3 * l + 1);
        launch_maxlen(h, h.lev[l]->R, h.maxlen.p + 3 * l + 2);
    }
}

void prepare_solve(rn_hierarchy &h) {
    prepare_solve_begin(h);
    prepare_solve_end(h);
}

void prepare_solve_end(rn_hierarchy &h) {
    cudaStream_t s = h.s;
    const bool mixed = h.p.precision == RN_MIXED;
    const size_t nmat = 3 * h.lev.size();
    if (h.maxlen.n != nmat) fail(RN_EINTERNAL, "prepare_solve_end without prepare_solve_begin");
    std::vector<int32_t> mlh(nmat);
    read_small(mlh.data(), h.maxlen.p, nmat, s);  // at most 3 x 32 levels: one read-back for all
    h.maxlen.release();
    for (size_t l = 0; l < h.lev.size(); l++) {
        rn_level &L = *h.lev[l];
        const int32_t n = L.A.n;
        L.b.alloc(n, s);
        L.x.alloc(n, s);
        L.t.alloc(n, s);
        L.r.alloc(n, s);
        set_tile_group(L.A, mlh[3 * l]);
        set_tile_group(L.P, mlh[3 * l + 1]);
        set_tile_group(L.R, mlh[3 * l + 2]);
        if (mixed) {
            L.b32.alloc(n, s);
            L.x32.alloc(n, s);
            L.t32.alloc(n, s);
            L.r32.alloc(n, s);
        }
        // relaxation weights omega / a_ii (a multiply in the sweeps instead of
        // a divide: FP64 division is slow on this part's reduced FP64 pipe)
        L.wd.alloc(n, s);
        if (mixed) L.wd32.alloc(n, s);
        RN_LAUNCH("prepare", 20.0 * n, s, omega_over_diag_kernel, grid_for(n, 1024), 256, 0, (int64_t)n, h.p.omega,
                  L.diag.p, L.wd.p, mixed ? L.wd32.p : nullptr);
        if (mixed) {
            L.A.val32.alloc(L.A.nnz, s);
            to_float(L.A.val.p, L.A.val32.p, L.A.nnz, s);
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
    if (h.p.autotune) autotune_schedules(h);
    const int64_t n0 = h.lev[0]->A.n;
    h.r.alloc(n0, s);
    h.z.alloc(n0, s);
    h.pv.alloc(n0, s);
    h.q.alloc(n0, s);
    h.w.alloc(n0, s);
    h.rold.alloc(n0, s);
    h.xs.alloc(n0, s);
    h.graph_in = h.r.p;
    h.graph_out = h.z.p;
    prepare_subcycle(h);
    if (h.p.outer == RN_OUTER_FGMRES) {
        const int m = std::max(1, h.p.restart);
        h.V.alloc((size_t)(m + 1) * n0, s);
        h.Z.alloc((size_t)m * n0, s);
        h.H.alloc((size_t)(m + 1) * m + 4 * (m + 1), s);
    }
}

static void check_tile_error(rn_hierarchy &h) {
    if (read_scalar(h.iflags.p + 8, h.s)) {
        RN_CUDA_CHECK(cudaMemsetAsync(h.iflags.p + 8, 0, sizeof(int32_t), h.s));
        fail(RN_ETIMEOUT, "a shared-memory staging wait gave up (bulk copy did not complete)");
    }
}

void cycle_checked(rn_hierarchy &h, const double *rhs, double *out) {
    apply_cycle(h, rhs, out);
    check_tile_error(h);
}

// Outer CG (Sec. 2: the cycle as preconditioner), one iteration in two halves:
// q = A p with <p,q> and alpha, then x, r and the stopping test; after the
// preconditioner z = M r, <r,z> (and <z,r_old>) with beta, then p.
static void cg_iteration_first_half(rn_hierarchy &h, double *x, const Fin &cond) {
    rn_level &L0 = *h.lev[0];
    const int64_t n = L0.A.n;
    double *sc = h.scal.p;
    const bool flexible = h.p.precision == RN_MIXED;
    spmv<double, double, double, OP_SPMV_DOT>(h, "outer_spmv", L0.A, h.pv.p, (const double *)nullptr, nullptr, 0.0,
                                              h.q.p, make_fin(h, FIN_PQ));
    Fin fx = make_fin(h, FIN_XR);
    fx.cond_loop = cond.cond_loop;
    fx.cond_body = cond.cond_body;
    rn_level &L0r = *h.lev[0];
    const bool fx0 = cg_forms_x0(h);
    if (h.p.precision == RN_MIXED)
        RN_SLAUNCH(h, "outer_cg_vec", 48.0 * n + 8.0 * n + (fx0 ? 8.0 * n : 0.0), h.s, cg_xr_kernel<float>,
                   VG(cg_xr_kernel<float>), kS, 0, n, x, h.r.p, h.pv.p, h.q.p, h.rold.p, sc,
                   (const float *)L0r.wd32.p, fx0 ? L0r.x32.p : nullptr, fx);
    else
        RN_SLAUNCH(h, "outer_cg_vec", 48.0 * n + (fx0 ? 16.0 * n : 0.0), h.s, cg_xr_kernel<double>,
                   VG(cg_xr_kernel<double>), kS, 0, n, x, h.r.p, h.pv.p, h.q.p, (double *)nullptr, sc,
                   (const double *)L0r.wd.p, fx0 ? L0r.x.p : nullptr, fx);
}

// z = M r, <r,z> (and <z,r_old>) with beta, then p.  The reductions ride on
// the cycle's last level-0 sweep when it has one.
static void cg_iteration_second_half(rn_hierarchy &h, bool flexible) {
    const int64_t n = h.lev[0]->A.n;
    Fin fr = make_fin(h, FIN_RZ);
    fr.it = flexible ? 2 : 0;
    const double *rold = flexible ? h.rold.p : nullptr;
    if (!cycle_direct(h, h.r.p, h.z.p, &fr, rold, cg_forms_x0(h)))
        RN_SLAUNCH(h, "outer_cg_vec", (flexible ? 24.0 : 16.0) * n, h.s, cg_rz_kernel, VG(cg_rz_kernel), kS, 0, n,
                  h.r.p, h.z.p, rold, fr);
    RN_SLAUNCH(h, "outer_cg_vec", 24.0 * n, h.s, cg_p_kernel, VG(cg_p_kernel), kS, 0, n, h.pv.p, h.z.p, h.scal.p, 0);
}

// Capture stream work into a standalone graph.
template <typename F>
static cudaGraph_t capture(rn_hierarchy &h, F &&work) {
    cudaGraph_t g = nullptr;
    RN_CUDA_CHECK(cudaStreamBeginCapture(h.s, cudaStreamCaptureModeThreadLocal));
    try {
        work();
    } catch (...) {
        cudaStreamEndCapture(h.s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    RN_CUDA_CHECK(cudaStreamEndCapture(h.s, &g));
    return g;
}

// The solve graph: kCgGraphIters iterations, each
//   IF(a_j) { first half }  ->  IF(b_j) { cycle; second half }
// The first half's reduction finisher sets b_j and a_{j+1} (iterate while not
// converged and below the iteration limit), so the host only relaunches the
// graph, and reads the loop state, once per kCgGraphIters iterations.  The
// graph holds no loop: whatever the conditions, one launch ends.
constexpr int kCgGraphIters = 8;

static void build_cg_graph(rn_hierarchy &h) {
    const bool flexible = h.p.precision == RN_MIXED;
    cudaGraph_t g = nullptr;
    RN_CUDA_CHECK(cudaGraphCreate(&g, 0));
    struct GraphGuard {
        cudaGraph_t *g;
        ~GraphGuard() {
            if (*g) cudaGraphDestroy(*g);
        }
    } guard{&g};
    cudaGraphConditionalHandle ha[kCgGraphIters + 1] = {}, hb[kCgGraphIters] = {};
    for (int j = 0; j < kCgGraphIters; j++) {
        RN_CUDA_CHECK(cudaGraphConditionalHandleCreate(&ha[j], g, j == 0 ? 1u : 0u, cudaGraphCondAssignDefault));
        RN_CUDA_CHECK(cudaGraphConditionalHandleCreate(&hb[j], g, 0u, cudaGraphCondAssignDefault));
    }
    const int64_t k0 = launches_so_far();
    cudaGraph_t g2 = capture(h, [&] { cg_iteration_second_half(h, flexible); });
    const int64_t k1 = launches_so_far();
    cudaGraphNode_t prev = nullptr;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < kCgGraphIters && e == cudaSuccess; j++) {
        Fin cond;
        cond.cond_loop = ha[j + 1];  // 0 after the last copy: nothing to set
        cond.cond_body = hb[j];
        cudaGraph_t g1 = nullptr;
        try {
            g1 = capture(h, [&] { cg_iteration_first_half(h, h.xs.p, cond); });
        } catch (...) {
            cudaGraphDestroy(g2);
            throw;
        }
        cudaGraphNodeParams pa = {};
        pa.type = cudaGraphNodeTypeConditional;
        pa.conditional.handle = ha[j];
        pa.conditional.type = cudaGraphCondTypeIf;
        pa.conditional.size = 1;
        cudaGraphNode_t na = nullptr, nb = nullptr, c1 = nullptr, c2 = nullptr;
        e = cudaGraphAddNode(&na, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &pa);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&c1, pa.conditional.phGraph_out[0], nullptr, 0, g1);
        cudaGraphDestroy(g1);
        cudaGraphNodeParams pb = {};
        pb.type = cudaGraphNodeTypeConditional;
        pb.conditional.handle = hb[j];
        pb.conditional.type = cudaGraphCondTypeIf;
        pb.conditional.size = 1;
        if (e == cudaSuccess) e = cudaGraphAddNode(&nb, g, &na, nullptr, 1, &pb);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&c2, pb.conditional.phGraph_out[0], nullptr, 0, g2);
        prev = nb;
    }
    const int64_t k2 = launches_so_far();
    h.cg_kernels[0] = (k2 - k1) / kCgGraphIters;
    h.cg_kernels[1] = k1 - k0;
    add_launches(k0 - k2);  // captured, not launched
    cudaGraphDestroy(g2);
    RN_CUDA_CHECK(e);
    e = cudaGraphInstantiate(&h.cg_exec, g, 0);
    if (e != cudaSuccess && h.pdl) {
        // programmatic edges inside conditional bodies not accepted here: plain edges
        cudaGetLastError();
        h.cg_exec = nullptr;
        h.pdl = false;
        if (h.graph_exec) {  // keep the cycle graph consistent with the launches
            cudaGraphExecDestroy(h.graph_exec);
            cudaGraphDestroy(h.graph);
            h.graph_exec = nullptr;
            h.graph = nullptr;
        }
        cudaGraphDestroy(g);
        g = nullptr;
        build_cg_graph(h);
        return;
    }
    RN_CUDA_CHECK(e);
    h.cg_graph = g;
    g = nullptr;
}

rn_status solve(rn_hierarchy &h, const double *b, double *x, double rtol, int maxit, rn_solve_info *info) {
    cudaStream_t s = h.s;
    rn_level &L0 = *h.lev[0];
    const int64_t n = L0.A.n;
    double *sc = h.scal.p;
    const double t0 = now_ms();
    const Fin none;
    const int eg = grid_for(n, 1024);
    auto residual = [&]() {  // r = b - A x, sc[8] = ||r||^2
        spmv<double, double, double, OP_RESID>(h, "outer_residual", L0.A, x, b, nullptr, 0.0, h.r.p,
                                               make_fin(h, FIN_STORE, sc + 8));
        return std::sqrt(read_scalar(sc + 8, s));
    };
    dot(b, b, n, sc + 17, s, h.partial.p, h.counters.p);
    double nb = std::sqrt(read_scalar(sc + 17, s));
    if (nb == 0.0) nb = 1.0;
    const double r0 = residual();
    double rn = r0;
    int it = 0;
    rn_status st = RN_ENOTCONV;
    if (rn / nb < rtol) st = RN_OK;
    if (st != RN_OK && h.p.outer == RN_OUTER_STATIONARY) {
        // x <- x + M (b - A x): the cycle applied to the current iterate
        for (it = 1; it <= maxit; it++) {
            apply_cycle(h, h.r.p, h.z.p);
            RN_LAUNCH("outer_axpy", 24.0 * n, s, axpy_kernel, eg, 256, 0, n, x, h.z.p);
            rn = residual();
            if (rn / nb < rtol) { st = RN_OK; break; }
        }
        if (it > maxit) it = maxit;
    } else if (st != RN_OK && h.p.outer == RN_OUTER_CG) {
        const bool flexible = h.p.precision == RN_MIXED;
        apply_cycle(h, h.r.p, h.z.p);
        Fin f0 = make_fin(h, FIN_RZ);
        f0.it = 1;  // first: beta = 0
        RN_LAUNCH("outer_cg_vec", 16.0 * n, s, cg_rz_kernel, VG(cg_rz_kernel), kS, 0, n, h.r.p, h.z.p, nullptr, f0);
        RN_LAUNCH("outer_cg_vec", 16.0 * n, s, cg_p_kernel, VG(cg_p_kernel), kS, 0, n, h.pv.p, h.z.p, sc, 1);
        RN_LAUNCH("outer_cg_state", 0, s, cg_loop_init_kernel, 1, 1, 0, sc, h.iflags.p, nb, rtol, maxit);
        if (maxit <= 0) {
            it = 0;
        } else if (h.p.use_graphs && !profiling_enabled()) {
            // iterations run in graph launches of kCgGraphIters; the device decides when to stop
            d2d(h.xs.p, x, n, s);
            if (!h.cg_exec) build_cg_graph(h);
            it = 0;
            for (;;) {
                RN_CUDA_CHECK(cudaGraphLaunch(h.cg_exec, s));
                int32_t fl[3];  // iterations done, limit, converged
                read_small(fl, h.iflags.p + 9, 3, s);
                const int done = fl[0] - it;
                const bool stopped = fl[2] != 0 || fl[0] >= maxit;
                // the second half runs in every iteration but a stopping one
                add_launches((int64_t)done * h.cg_kernels[0] + (int64_t)(done - (stopped ? 1 : 0)) * h.cg_kernels[1]);
                it = fl[0];
                if (stopped) break;
                if (done != kCgGraphIters) fail(RN_EINTERNAL, "solve graph: conditional nodes were not honoured");
            }
            d2d(x, h.xs.p, n, s);
        } else {
            for (it = 1; it <= maxit; it++) {
                cg_iteration_first_half(h, x, Fin());
                rn = std::sqrt(read_scalar(sc + 8, s));
                if (rn / nb < rtol) break;
                cg_iteration_second_half(h, flexible);
            }
            if (it > maxit) it = maxit;
        }
        rn = residual();
        st = (rn / nb < rtol) ? RN_OK : RN_ENOTCONV;
    } else if (st != RN_OK && h.p.outer == RN_OUTER_FGMRES) {
        const int m = std::max(1, h.p.restart);
        double *H = h.H.p, *cs = H + (m + 1) * m, *sn = cs + (m + 1), *g = sn + (m + 1), *y = g + (m + 1);
        it = 0;
        while (it < maxit && st != RN_OK) {
            // V0 = r / ||r|| (r and ||r||^2 are current)
            RN_LAUNCH("outer_gmres_scalar", 0, s, fg_start_kernel, 1, 1, 0, g, m, sc);
            RN_LAUNCH("outer_gmres_vec", 16.0 * n, s, scale_copy_kernel, eg, 256, 0, n, h.r.p, sc + 8, h.V.p, 1);
            int k = 0;
            for (int j = 0; j < m && it < maxit; j++) {
                double *vj = h.V.p + (int64_t)j * n, *zj = h.Z.p + (int64_t)j * n;
                apply_cycle(h, vj, zj);
                spmv<double, double, double, OP_SPMV>(h, "outer_spmv", L0.A, zj, (const double *)nullptr, nullptr,
                                                      0.0, h.w.p, none);
                // modified Gram-Schmidt: each update w -= h_ij v_i is fused with
                // the next projection <w, v_{i+1}> (the last with ||w||^2), the
                // same operations in the same order as separate launches
                dot(h.w.p, h.V.p, n, H + j, s, h.partial.p, h.counters.p);
                for (int i = 0; i <= j; i++) {
                    const double *vi = h.V.p + (int64_t)i * n;
                    if (i < j)
                        axpy_dot(h.w.p, vi, H + i * m + j, vi + n, n, H + (i + 1) * m + j, s, h.partial.p,
                                 h.counters.p);
                    else
                        axpy_dot(h.w.p, vi, H + i * m + j, nullptr, n, sc + 8, s, h.partial.p, h.counters.p);
                }
                RN_LAUNCH("outer_gmres_scalar", 0, s, fg_givens_kernel, 1, 1, 0, m, j, H, cs, sn, g, sc);
                it++;
                k = j + 1;
                double res[2];
                read_small(res, sc + 15, 2, s);
                if (res[0] / nb < rtol || res[1] == 0.0) break;
                RN_LAUNCH("outer_gmres_vec", 16.0 * n, s, scale_copy_kernel, eg, 256, 0, n, h.w.p, sc + 16,
                          h.V.p + (int64_t)(j + 1) * n, 0);
            }
            RN_LAUNCH("outer_gmres_scalar", 0, s, fg_backsolve_kernel, 1, 1, 0, m, k, H, g, y);
            RN_LAUNCH("outer_gmres_vec", (8.0 * k + 16.0) * n, s, fg_update_kernel, eg, 256, 0, n, k, x, h.Z.p, y);
            rn = residual();
            if (rn / nb < rtol) st = RN_OK;
        }
    } else if (st != RN_OK) {
        fail(RN_EINVAL, "unknown outer iteration");
    }
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    check_tile_error(h);
    if (info) {
        info->iters = it;
        info->rel_res = rn / nb;
        info->rho = (it > 0 && r0 > 0.0) ? std::pow(rn / r0, 1.0 / it) : 0.0;
        info->solve_ms = now_ms() - t0;
        info->status = st;
    }
    return st;
}

// ------------------------------------------------------------------ measurement
// One level-0 launch of the solve, as the solve issues it (kernel, launch
// shape, buffers), for timing in isolation.  Returns its algorithmic bytes.
template <typename T>
static double enqueue_op(rn_hierarchy &h, int op, std::string &name) {
    using LB = LevelBufs<T>;
    rn_level &L0 = *h.lev[0];
    const int64_t n = L0.A.n;
    const bool mixed = sizeof(T) == 4;
    const CycleNames &nm = kNames[mixed][0];
    const Fin none;
    double *sc = h.scal.p;
    const bool multi = h.lev.size() > 1;
    if (op >= RN_OP_RELAX0_RESIDUAL && op <= RN_OP_PROLONG && !multi) fail(RN_EINVAL, "operation needs two levels");
    const T omega = (T)h.p.omega;
    switch (op) {
        case RN_OP_OUTER_SPMV:
            name = "outer_spmv";
            spmv<double, double, double, OP_SPMV_DOT>(h, "outer_spmv", L0.A, h.pv.p, (const double *)nullptr, nullptr,
                                                      0.0, h.q.p, make_fin(h, FIN_STORE, sc + 20));
            return spmv_bytes<double, double, double, OP_SPMV_DOT>(L0.A);
        case RN_OP_RELAX0_RESIDUAL:  // x0 = (omega / a_ii) r formed by the outer CG's update
            name = nm.resid;
            spmv<T, double, T, OP_RESID>(h, nm.resid, L0.A, LB::x(L0), h.r.p, nullptr, T(0), LB::r(L0), none);
            return spmv_bytes<T, double, T, OP_RESID>(L0.A);
        case RN_OP_JACOBI_OUT:  // as the CG solve issues it: fused with <r,z> (and <z,r_old>)
            name = nm.jacobi;
            spmv<T, double, double, OP_JACOBI_RZ>(h, nm.jacobi, L0.A, LB::x(L0), h.r.p, LB::d(L0), omega, h.z.p,
                                                  make_fin(h, FIN_STORE, sc + 20), nullptr,
                                                  mixed ? h.rold.p : nullptr);
            return spmv_bytes<T, double, double, OP_JACOBI_RZ>(L0.A) + (mixed ? 8.0 * n : 0.0);
        case RN_OP_RESTRICT:
            name = nm.restr;
            spmv<T, T, T, OP_SPMV>(h, nm.restr, L0.R, LB::r(L0), (const T *)nullptr, nullptr, T(0),
                                   LB::b(*h.lev[1]), none);
            return spmv_bytes<T, T, T, OP_SPMV>(L0.R);
        case RN_OP_PROLONG:
            name = nm.prolong;
            spmv<T, T, T, OP_SPMV_ADD>(h, nm.prolong, L0.P, LB::x(*h.lev[1]), (const T *)nullptr, nullptr, T(0),
                                       LB::x(L0), none);
            return spmv_bytes<T, T, T, OP_SPMV_ADD>(L0.P);
        case RN_OP_CG_XR: {
            name = "outer_cg_xr";
            const bool fx0 = cg_forms_x0(h);
            const double b = 48.0 * n + (mixed ? 8.0 * n : 0.0) + (fx0 ? (mixed ? 8.0 : 16.0) * n : 0.0);
            T *x0 = fx0 ? LB::x(L0) : nullptr;
            RN_LAUNCH("outer_cg_vec", b, h.s, cg_xr_kernel<T>, VG(cg_xr_kernel<T>), kS, 0, n, h.xs.p, h.r.p, h.pv.p,
                      h.q.p, mixed ? h.rold.p : nullptr, sc, LB::d(L0), x0, make_fin(h, FIN_STORE, sc + 20));
            return b;
        }
        case RN_OP_CG_RZ: {  // runs only when the cycle has no level-0 post-sweep to carry it
            name = "outer_cg_rz";
            const double b = (mixed ? 24.0 : 16.0) * n;
            RN_LAUNCH("outer_cg_vec", b, h.s, cg_rz_kernel, VG(cg_rz_kernel), kS, 0, n, h.r.p, h.z.p,
                      mixed ? h.rold.p : nullptr, make_fin(h, FIN_STORE, sc + 20));
            return b;
        }
        case RN_OP_CG_P: {
            name = "outer_cg_p";
            const double b = 24.0 * n;
            RN_LAUNCH("outer_cg_vec", b, h.s, cg_p_kernel, VG(cg_p_kernel), kS, 0, n, h.pv.p, h.z.p, sc, 0);
            return b;
        }
        case RN_OP_COARSE_CLUSTER: {
            if (h.sub_k < 0) fail(RN_EINVAL, "this hierarchy runs no cluster cycle");
            name = mixed ? "cycle_coarse_cluster_f32" : "cycle_coarse_cluster_f64";
            launch_subcycle<T>(h, pre_smoothed<T>(*h.lev[h.sub_k], h.p.nu_pre), name.c_str());
            return 0.0;  // latency-bound: no bandwidth claim
        }
        default: fail(RN_EINVAL, "unknown operation");
    }
    return 0.0;
}

// Reads the flush buffer (16-byte words) so that L2 ends up holding only its
// clean lines: a write flush would leave up to 129 MB of dirty lines whose
// write-back the timed kernel would pay for.  One word per block is stored so
// the loads are not dead.
__global__ void flush_read_kernel(const uint4 *__restrict__ p, int64_t n16, uint32_t *__restrict__ sink) {
    pdl_wait();
    uint32_t a = 0u;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n16; k += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = p[k];  // default policy: the lines displace what L2 held
        a ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    a = __reduce_xor_sync(0xffffffffu, a);
    if ((threadIdx.x & 31) == 0) atomicXor(sink + blockIdx.x, a);
}

double time_launches(cudaStream_t s, int reps, int64_t flush_bytes, const std::function<void()> &before,
                     const std::function<void()> &timed) {
    if (reps < 1 || reps > 100000) fail(RN_EINVAL, "reps must be in [1, 100000]");
    if (flush_bytes < 0) fail(RN_EINVAL, "flush_bytes must be >= 0");
    const int64_t n16 = flush_bytes / 16;
    DVec<uint4> fl(n16 > 0 ? (size_t)n16 : 0, s);
    const int fgrid = 4 * num_sms();
    DVec<uint32_t> sink(fgrid, s);
    if (n16 > 0) RN_CUDA_CHECK(cudaMemsetAsync(fl.p, 0x5a, (size_t)n16 * 16, s));
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    struct EvGuard {
        std::vector<cudaEvent_t> &ev;
        ~EvGuard() {
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
        }
    } guard{ev};
    for (auto &e : ev) RN_CUDA_CHECK(cudaEventCreate(&e));
    for (int r = 0; r < reps; r++) {
        if (before) before();
        if (n16 > 0) {
            flush_read_kernel<<<fgrid, 512, 0, s>>>(fl.p, n16, sink.p);
            RN_CUDA_CHECK(cudaGetLastError());
        }
        RN_CUDA_CHECK(cudaEventRecord(ev[2 * r], s));
        timed();
        RN_CUDA_CHECK(cudaEventRecord(ev[2 * r + 1], s));
    }
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    double tot = 0.0;
    for (int r = 0; r < reps; r++) {
        float ms = 0.f;
        RN_CUDA_CHECK(cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]));
        tot += ms;
    }
    return tot * 1e3 / reps;
}

void time_op(rn_hierarchy &h, int op, int reps, int64_t flush_bytes, double *us, double *bytes, std::string &name) {
    cudaStream_t s = h.s;
    if (reps < 1 || reps > 100000) fail(RN_EINVAL, "reps must be in [1, 100000]");
    if (flush_bytes < 0) fail(RN_EINVAL, "flush_bytes must be >= 0");
    const int64_t n16 = flush_bytes / 16;
    DVec<uint4> fl(n16 > 0 ? (size_t)n16 : 0, s);
    const int fgrid = 4 * num_sms();
    DVec<uint32_t> sink(fgrid, s);
    if (n16 > 0) RN_CUDA_CHECK(cudaMemsetAsync(fl.p, 0x5a, (size_t)n16 * 16, s));
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    struct EvGuard {
        std::vector<cudaEvent_t> &ev;
        ~EvGuard() {
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
        }
    } guard{ev};
    for (auto &e : ev) RN_CUDA_CHECK(cudaEventCreate(&e));
    const bool mixed = h.p.precision == RN_MIXED;
    double b = 0.0;
    for (int r = 0; r < reps; r++) {
        // the flush keeps the GPU busy while the launch is enqueued and leaves L2 cold and clean
        if (n16 > 0) {
            flush_read_kernel<<<fgrid, 512, 0, s>>>(fl.p, n16, sink.p);
            RN_CUDA_CHECK(cudaGetLastError());
        }
        RN_CUDA_CHECK(cudaEventRecord(ev[2 * r], s));
        b = mixed ? enqueue_op<float>(h, op, name) : enqueue_op<double>(h, op, name);
        RN_CUDA_CHECK(cudaEventRecord(ev[2 * r + 1], s));
    }
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    check_tile_error(h);
    double tot = 0.0;
    for (int r = 0; r < reps; r++) {
        float ms = 0.f;
        RN_CUDA_CHECK(cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]));
        tot += ms;
    }
    *us = tot * 1e3 / reps;
    *bytes = b;
}

}  // namespace rn
