// rn_multi.cu - many right-hand sides at once: the V-cycle (Sec. 2, eq.
// twogrid applied recursively) on n x s row-major multivectors, with SpMM in
// place of SpMV, inside the stationary outer iteration X <- X + M(B - A X)
// with a stopping test per column.
//
// Each operator row is read once per operation for all s columns: a warp
// takes a row, broadcasts each stored entry and streams the s-wide rows of
// the operand (coalesced, s/32 values per lane), so the matrix traffic of one
// cycle is shared by every right-hand side.  In mixed precision the cycle's
// multivectors are FP32 and the outer residual FP64, as in the single solve.
// Column norms are reduced per block and then per column in block order
// (deterministic).
#include "rn_hier.cuh"

namespace rn {

constexpr int kMT = 256;  // threads per block: 8 warps, a warp per row
constexpr int kCPL = 8;   // columns per lane per pass (256 columns per warp pass)

enum MOp { M_SPMM = 0, M_SPMM_ADD = 1, M_RESID = 2, M_JACOBI = 3, M_JZ_RESID = 4 };

// Y = op(M, X, B) on s columns.  M_JZ_RESID: XZ = D B, Y = B - M (D B), with D
// (omega / a_ii) applied to the gathered rows of B.  With nrm, the squares of
// Y's entries (M_RESID) are summed per column into nrm[block * s + c].
// A warp takes (row, column chunk) tasks: CPL columns per lane, 32 * CPL per
// chunk; few rows take narrow chunks (CPL = 2) so that more warps share them.
template <typename T, typename TB, typename TO, int OP, int CPL>
__global__ void __launch_bounds__(kMT)
spmm_kernel(int32_t n, int s, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
            const T *__restrict__ val, const T *__restrict__ X, const TB *__restrict__ B, const T *__restrict__ d,
            TO *__restrict__ Y, T *__restrict__ XZ, double *__restrict__ nrm) {
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = kMT / 32;
    extern __shared__ double snrm[];  // [wpb][s] when nrm
    if (nrm)
        for (int c = threadIdx.x; c < wpb * s; c += kMT) snrm[c] = 0.0;
    __syncthreads();
    const int nck = (s + 32 * CPL - 1) / (32 * CPL);
    const int64_t ntask = (int64_t)n * nck;
    for (int64_t task = (int64_t)blockIdx.x * wpb + warp; task < ntask; task += (int64_t)gridDim.x * wpb) {
        const int32_t i = (int32_t)(task / nck);
        const int c0 = (int)(task % nck) * 32 * CPL;
        const int32_t e0 = rp[i], e1 = rp[i + 1];
        const T di = (OP == M_JACOBI || OP == M_JZ_RESID) ? d[i] : T(0);
        {
            T acc[CPL];
#pragma unroll
            for (int u = 0; u < CPL; u++) acc[u] = T(0);
            // the row's entries 32 at a time: one coalesced load of columns and
            // values across the lanes, then each entry broadcast by a shuffle, so
            // the operand rows of several entries are gathered at once instead of
            // each gather waiting for its entry's column index
            for (int32_t eb = e0; eb < e1; eb += 32) {
                const int cnt = min(32, e1 - eb);
                int32_t jl = 0;
                T al = T(0), dl = T(1);
                if (lane < cnt) {
                    jl = col[eb + lane];
                    al = val[eb + lane];
                    if (OP == M_JZ_RESID) dl = d[jl];
                }
#pragma unroll 4
                for (int k = 0; k < cnt; k++) {
                    const int32_t j = __shfl_sync(0xffffffffu, jl, k);
                    const T a = __shfl_sync(0xffffffffu, al, k);
                    const T dj = OP == M_JZ_RESID ? __shfl_sync(0xffffffffu, dl, k) : T(1);
#pragma unroll
                    for (int u = 0; u < CPL; u++) {
                        const int c = c0 + lane + 32 * u;
                        if (c < s) {
                            const int64_t o = (int64_t)j * s + c;
                            const T xv = OP == M_JZ_RESID ? dj * (T)B[o] : X[o];
                            acc[u] = fma(a, xv, acc[u]);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CPL; u++) {
                const int c = c0 + lane + 32 * u;
                if (c >= s) continue;
                const int64_t o = (int64_t)i * s + c;
                if (OP == M_SPMM) {
                    Y[o] = (TO)acc[u];
                } else if (OP == M_SPMM_ADD) {
                    Y[o] = (TO)((T)Y[o] + acc[u]);
                } else if (OP == M_RESID) {
                    const TO r = (TO)((T)B[o] - acc[u]);
                    Y[o] = r;
                    if (nrm) snrm[warp * s + c] += (double)r * (double)r;
                } else if (OP == M_JACOBI) {
                    Y[o] = (TO)(X[o] + di * ((T)B[o] - acc[u]));
                } else {  // M_JZ_RESID
                    const T bi = (T)B[o];
                    XZ[o] = di * bi;
                    Y[o] = (TO)(bi - acc[u]);
                }
            }
        }
    }
    if (nrm) {
        __syncthreads();
        for (int c = threadIdx.x; c < s; c += kMT) {
            double t = 0.0;
            for (int w = 0; w < wpb; w++) t += snrm[w * s + c];
            nrm[(int64_t)blockIdx.x * s + c] = t;
        }
    }
}

// column sums of the per-block partials: a block per 32 columns, lane =
// column; warp w sums partials w, w + 8, ... (four chains), and the eight warp
// sums are added in warp order (a fixed order: reproducible run to run)
constexpr int kColWarps = 8;
__global__ void __launch_bounds__(32 * kColWarps)
col_norms_kernel(int nb, int s, const double *__restrict__ part, double *__restrict__ out) {
    pdl_wait();
    __shared__ double ws[kColWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    if (c < s) {
        int b = w;
        for (; b + 3 * kColWarps < nb; b += 4 * kColWarps) {
#pragma unroll
            for (int u = 0; u < 4; u++) t[u] += part[(int64_t)(b + u * kColWarps) * s + c];
        }
        for (; b < nb; b += kColWarps) t[0] += part[(int64_t)b * s + c];
    }
    ws[w][lane] = (t[0] + t[1]) + (t[2] + t[3]);
    __syncthreads();
    if (w == 0 && c < s) {
        double a = 0.0;
#pragma unroll
        for (int k = 0; k < kColWarps; k++) a += ws[k][lane];
        out[c] = a;
    }
}

// Y = D B (first sweep from a zero guess, row-local)
template <typename T, typename TB>
__global__ void jz_multi_kernel(int32_t n, int s, const TB *__restrict__ B, const T *__restrict__ d,
                                T *__restrict__ Y) {
    pdl_wait();
    const int64_t total = (int64_t)n * s;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x)
        Y[o] = d[o / s] * (T)B[o];
}

// coarsest level: Y = A_L^{-1} B in FP64 arithmetic; a warp per row, lanes
// over columns, kCPL columns per lane summed side by side (each column's sum
// in ascending j), so every step of j issues kCPL independent loads
template <typename TB, typename TO>
__global__ void coarse_multi_kernel(int32_t n, int s, const double *__restrict__ Ainv, const TB *__restrict__ B,
                                    TO *__restrict__ Y) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5)
        for (int c0 = 0; c0 < s; c0 += 32 * kCPL) {
            double acc[kCPL];
#pragma unroll
            for (int u = 0; u < kCPL; u++) acc[u] = 0.0;
#pragma unroll 4
            for (int32_t j = 0; j < n; j++) {
                const double aij = Ainv[(int64_t)i * n + j];
#pragma unroll
                for (int u = 0; u < kCPL; u++) {
                    const int c = c0 + lane + 32 * u;
                    if (c < s) acc[u] = fma(aij, (double)B[(int64_t)j * s + c], acc[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < kCPL; u++) {
                const int c = c0 + lane + 32 * u;
                if (c < s) Y[(int64_t)i * s + c] = (TO)acc[u];
            }
        }
}

template <typename T>
__global__ void cvt_multi_kernel(int64_t total, const T *__restrict__ x, double *__restrict__ y) {
    pdl_wait();
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x)
        y[o] = (double)x[o];
}

__global__ void add_multi_kernel(int64_t total, double *__restrict__ X, const double *__restrict__ Z) {
    pdl_wait();
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x)
        X[o] += Z[o];
}

// ------------------------------------------------------------------ host side
template <typename T>
static const T *mvals(const DCsr &M) {
    if constexpr (sizeof(T) == 4) return M.val32.p;
    else return M.val.p;
}
template <typename T>
static const T *mweights(rn_level &L) {
    if constexpr (sizeof(T) == 4) return L.wd32.p;
    else return L.wd.p;
}

static int multi_grid(int32_t n) { return std::max(1, std::min<int>((n + 7) / 8, num_sms() * 8)); }

constexpr int32_t kMultiFewRows = 2048;  // below: 2 columns per lane, 4x the warps per row

template <typename T, typename TB, typename TO, int OP, int CPL>
static void spmm_t(cudaStream_t s, const char *name, const DCsr &M, int ns, const T *X, const TB *B, const T *d,
                   TO *Y, T *XZ, double *nrm, int grid) {
    const int nck = (ns + 32 * CPL - 1) / (32 * CPL);
    if (!grid) grid = std::max(1, (int)std::min<int64_t>(((int64_t)M.n * nck + 7) / 8, (int64_t)num_sms() * 8));
    const double bytes =
        (4.0 + sizeof(T)) * M.nnz + 4.0 * (M.n + 1) + (double)ns * (sizeof(T) * M.m + sizeof(TO) * M.n);
    const size_t smem = nrm ? sizeof(double) * (kMT / 32) * ns : 0;
    if (smem > 48 * 1024) {
        RN_CUDA_CHECK(cudaFuncSetAttribute(spmm_kernel<T, TB, TO, OP, CPL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    RN_LAUNCH(name, bytes, s, (spmm_kernel<T, TB, TO, OP, CPL>), grid, kMT, smem, M.n, ns, M.rowptr.p, M.col.p,
              mvals<T>(M), X, B, d, Y, XZ, nrm);
}
// grid: given only for the outer residual, whose per-block column partials
// the caller sizes (it keeps 8 columns per lane)
template <typename T, typename TB, typename TO, int OP>
static void spmm(cudaStream_t s, const char *name, const DCsr &M, int ns, const T *X, const TB *B, const T *d, TO *Y,
                 T *XZ = nullptr, double *nrm = nullptr, int grid = 0) {
    if (M.n == 0) return;
    if (grid || M.n >= kMultiFewRows) spmm_t<T, TB, TO, OP, kCPL>(s, name, M, ns, X, B, d, Y, XZ, nrm, grid);
    else spmm_t<T, TB, TO, OP, 2>(s, name, M, ns, X, B, d, Y, XZ, nrm, grid);
}

// multivector workspaces of one cycle, per level: b, x, t, r (n_l x s each)
template <typename T>
struct MultiBufs {
    std::vector<DVec<T>> b, x, t, r;
};

// One cycle on level l >= 1 (zero initial guess, right-hand side in W.b[l]);
// returns the buffer with the result.
template <typename T>
static T *mcycle_level(rn_hierarchy &h, MultiBufs<T> &W, int l, int ns) {
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[l];
    const int32_t n = L.A.n;
    if (l == (int)h.lev.size() - 1) {
        // a warp per block: the rows' FP64 multiply-adds spread over as many SMs as rows
        RN_LAUNCH("multi_coarse_solve", 8.0 * n * n + 2.0 * sizeof(T) * n * ns, s, (coarse_multi_kernel<T, T>),
                  grid_for((int64_t)n * 32, 32, 16), 32, 0, n, ns, h.Ainv.p, W.b[l].p, W.x[l].p);
        return W.x[l].p;
    }
    const T *d = mweights<T>(L);
    T *cur = W.x[l].p, *oth = W.t[l].p, *b = W.b[l].p, *r = W.r[l].p;
    if (h.p.nu_pre == 1) {
        spmm<T, T, T, M_JZ_RESID>(s, "multi_relax0_residual", L.A, ns, (const T *)nullptr, b, d, r, cur);
    } else {
        const int64_t tot = (int64_t)n * ns;
        if (h.p.nu_pre == 0) RN_CUDA_CHECK(cudaMemsetAsync(cur, 0, sizeof(T) * tot, s));
        else RN_LAUNCH("multi_jacobi0", 3.0 * sizeof(T) * tot, s, (jz_multi_kernel<T, T>), grid_for(tot, 1024), 256, 0,
                       n, ns, (const T *)b, d, cur);
        for (int k = 1; k < h.p.nu_pre; k++) {
            spmm<T, T, T, M_JACOBI>(s, "multi_jacobi", L.A, ns, cur, b, d, oth);
            std::swap(cur, oth);
        }
        spmm<T, T, T, M_RESID>(s, "multi_residual", L.A, ns, cur, b, (const T *)nullptr, r);
    }
    spmm<T, T, T, M_SPMM>(s, "multi_restrict", L.R, ns, r, (const T *)nullptr, (const T *)nullptr, W.b[l + 1].p);
    T *xc = mcycle_level<T>(h, W, l + 1, ns);
    spmm<T, T, T, M_SPMM_ADD>(s, "multi_prolong", L.P, ns, xc, (const T *)nullptr, (const T *)nullptr, cur);
    for (int k = 0; k < h.p.nu_post; k++) {
        spmm<T, T, T, M_JACOBI>(s, "multi_jacobi", L.A, ns, cur, b, d, oth);
        std::swap(cur, oth);
    }
    return cur;
}

// Z = M R on level 0 (FP64 in and out; the cycle in T)
template <typename T>
static void mcycle_top(rn_hierarchy &h, MultiBufs<T> &W, const double *R, double *Z, int ns) {
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[0];
    const int32_t n = L.A.n;
    const int64_t tot = (int64_t)n * ns;
    if (h.lev.size() == 1) {
        RN_LAUNCH("multi_coarse_solve", 8.0 * n * n + 16.0 * tot, s, (coarse_multi_kernel<double, double>),
                  grid_for((int64_t)n * 32, 32, 16), 32, 0, n, ns, h.Ainv.p, R, Z);
        return;
    }
    const T *d = mweights<T>(L);
    T *cur = W.x[0].p, *oth = W.t[0].p, *r = W.r[0].p;
    // first sweep from zero: x = D R formed row-locally, then the residual
    if (h.p.nu_pre == 0) RN_CUDA_CHECK(cudaMemsetAsync(cur, 0, sizeof(T) * tot, s));
    else RN_LAUNCH("multi_jacobi0", (8.0 + 2.0 * sizeof(T)) * tot, s, (jz_multi_kernel<T, double>),
                   grid_for(tot, 1024), 256, 0, n, ns, R, d, cur);
    for (int k = 1; k < h.p.nu_pre; k++) {
        spmm<T, double, T, M_JACOBI>(s, "multi_jacobi_L0", L.A, ns, cur, R, d, oth);
        std::swap(cur, oth);
    }
    spmm<T, double, T, M_RESID>(s, "multi_residual_L0", L.A, ns, cur, R, (const T *)nullptr, r);
    spmm<T, T, T, M_SPMM>(s, "multi_restrict_L0", L.R, ns, r, (const T *)nullptr, (const T *)nullptr, W.b[1].p);
    T *xc = mcycle_level<T>(h, W, 1, ns);
    spmm<T, T, T, M_SPMM_ADD>(s, "multi_prolong_L0", L.P, ns, xc, (const T *)nullptr, (const T *)nullptr, cur);
    for (int k = 0; k < h.p.nu_post; k++) {
        if (k == h.p.nu_post - 1) {
            spmm<T, double, double, M_JACOBI>(s, "multi_jacobi_L0", L.A, ns, cur, R, d, Z);
            return;
        }
        spmm<T, double, T, M_JACOBI>(s, "multi_jacobi_L0", L.A, ns, cur, R, d, oth);
        std::swap(cur, oth);
    }
    // no post-smoothing: the iterate itself, in FP64
    RN_LAUNCH("multi_convert", (8.0 + sizeof(T)) * tot, s, (cvt_multi_kernel<T>), grid_for(tot, 1024), 256, 0, tot,
              (const T *)cur, Z);
}

template <typename T>
static rn_status solve_multi_t(rn_hierarchy &h, const double *B, double *X, int ns, double rtol, int maxit,
                               rn_solve_info *info) {
    cudaStream_t s = h.s;
    rn_level &L0 = *h.lev[0];
    const int32_t n = L0.A.n;
    const int64_t tot = (int64_t)n * ns;
    MultiBufs<T> W;
    const int nl = (int)h.lev.size();
    W.b.resize(nl); W.x.resize(nl); W.t.resize(nl); W.r.resize(nl);
    for (int l = 0; l < nl; l++) {
        const size_t m = (size_t)h.lev[l]->A.n * ns;
        W.b[l].alloc(m, s); W.x[l].alloc(m, s); W.t[l].alloc(m, s); W.r[l].alloc(m, s);
    }
    DVec<double> R(tot, s), Z(tot, s);
    const int grid = multi_grid(n);
    DVec<double> part((size_t)grid * ns, s), nb2(ns, s), nr2(ns, s);
    std::vector<double> hb(ns), hr(ns);
    auto residual = [&](double *out) {  // R = B - A X, out = per-column ||r||^2
        spmm<double, double, double, M_RESID>(s, "multi_outer_residual", L0.A, ns, X, B, (const double *)nullptr,
                                              R.p, (double *)nullptr, part.p, grid);
        RN_LAUNCH("multi_col_norms", 8.0 * grid * ns, s, col_norms_kernel, (ns + 31) / 32, 32 * kColWarps, 0, grid, ns,
                  part.p, out);
    };
    // ||b_c||^2 from the same reduction with X = 0
    {
        DVec<double> zero(tot, s);
        RN_CUDA_CHECK(cudaMemsetAsync(zero.p, 0, sizeof(double) * tot, s));
        spmm<double, double, double, M_RESID>(s, "multi_outer_residual", L0.A, ns, zero.p, B, (const double *)nullptr,
                                              R.p, (double *)nullptr, part.p, grid);
        RN_LAUNCH("multi_col_norms", 8.0 * grid * ns, s, col_norms_kernel, (ns + 31) / 32, 32 * kColWarps, 0, grid, ns,
                  part.p, nb2.p);
        RN_CUDA_CHECK(cudaMemcpyAsync(hb.data(), nb2.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    }
    auto worst = [&]() {  // largest relative residual over the columns (zero columns count as converged)
        RN_CUDA_CHECK(cudaMemcpyAsync(hr.data(), nr2.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        RN_CUDA_CHECK(cudaStreamSynchronize(s));
        double w = 0.0;
        for (int c = 0; c < ns; c++) {
            const double bn = std::sqrt(hb[c]);
            const double rel = bn > 0.0 ? std::sqrt(hr[c]) / bn : std::sqrt(hr[c]);
            w = std::max(w, rel);
        }
        return w;
    };
    residual(nr2.p);
    const double w0 = worst();
    double w = w0;
    int it = 0;
    // one iteration: Z = M R, X += Z, R = B - A X and the column norms; with
    // graphs it is captured once and replayed (one launch per iteration
    // instead of one per kernel: the small levels' launches cost more than
    // their work)
    auto iteration = [&]() {
        mcycle_top<T>(h, W, R.p, Z.p, ns);
        RN_LAUNCH("multi_outer_update", 24.0 * tot, s, add_multi_kernel, grid_for(tot, 1024), 256, 0, tot, X, Z.p);
        residual(nr2.p);
    };
    struct Graph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        int64_t kernels = 0;
        ~Graph() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
        }
    } graph;
    const bool use_graph = h.p.use_graphs && !profiling_enabled();
    while (w >= rtol && it < maxit) {
        if (use_graph) {
            if (!graph.e) {
                const int64_t before = launches_so_far();
                RN_CUDA_CHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                try {
                    iteration();
                } catch (...) {
                    cudaGraph_t g = nullptr;
                    cudaStreamEndCapture(s, &g);
                    if (g) cudaGraphDestroy(g);
                    throw;
                }
                RN_CUDA_CHECK(cudaStreamEndCapture(s, &graph.g));
                RN_CUDA_CHECK(cudaGraphInstantiate(&graph.e, graph.g, 0));
                graph.kernels = launches_so_far() - before;
                add_launches(-graph.kernels);  // captured, not launched
            }
            RN_CUDA_CHECK(cudaGraphLaunch(graph.e, s));
            add_launches(graph.kernels);
        } else {
            iteration();
        }
        w = worst();
        it++;
    }
    if (info) {
        info->iters = it;
        info->rel_res = w;
        info->rho = (it > 0 && w0 > 0.0) ? std::pow(w / w0, 1.0 / it) : 0.0;
        info->status = w < rtol ? RN_OK : RN_ENOTCONV;
    }
    return w < rtol ? RN_OK : RN_ENOTCONV;
}

rn_status solve_multi(rn_hierarchy &h, const double *B, double *X, int ns, double rtol, int maxit,
                      rn_solve_info *info) {
    if (h.p.precision == RN_MIXED) return solve_multi_t<float>(h, B, X, ns, rtol, maxit, info);
    return solve_multi_t<double>(h, B, X, ns, rtol, maxit, info);
}

}  // namespace rn
