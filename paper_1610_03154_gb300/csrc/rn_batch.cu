// rn_batch.cu - independent problems solved as one.  Their hierarchies are
// merged level by level into block-diagonal operators, so each step of the
// V(1,1) cycle (Sec. 2) and of the outer CG is one launch for all problems
// instead of one per problem: small problems are bound by launch latency,
// and the GPU front end, not HBM, limits many of them run side by side.
//
// Problem p keeps its own operators on levels it has (l < L_p - 1: A, P, R,
// omega / a_ii).  From its coarsest level L_p - 1 down to the merged
// hierarchy's last level it is passed through: relaxation weight 0 (diagonal
// +inf), identity P and R, no stored A rows below L_p - 1.  With a zero
// initial guess this is exact: x = 0 * b, r = b - A 0 = b, R r = r,
// x + 1 * x_c = x_c, and post-sweeps add 0 * (b - A x).  The last level
// solves every problem's coarsest block with its own dense inverse, so each
// problem's cycle is its own cycle.  The outer CG keeps per-problem scalars
// (alpha, beta, <r,z>, stopping) and reduces per problem over fixed row
// chunks in a fixed order.
#include <cmath>

#include "rn_hier.cuh"
#include "rn_spmv.cuh"

rn_batch::~rn_batch() {
    if (it_exec) cudaGraphExecDestroy(it_exec);
    if (it_graph) cudaGraphDestroy(it_graph);
}

namespace rn {

namespace {

constexpr int kBT = 256;          // threads per block of the batched kernels
constexpr int32_t kChunk = 4096;  // rows per reduction chunk (chunks never straddle problems)
constexpr int kItersPerPoll = 8;  // iteration graphs launched between reads of the active count

// per-problem doubles d[slot * np + p] and ints iv[slot * np + p]
enum { D_NB, D_RZ, D_RZP, D_ZRO, D_PQ, D_ALPHA, D_BETA, D_RR, D_R0, D_RRF, kD };
enum { I_IT, I_ACT, I_CONV, kI };  // iv[kI * np]: problems still iterating
enum BMode { BM_NB, BM_R0, BM_RZ_FIRST, BM_RZ, BM_PQ, BM_XR, BM_FINAL };

struct BCg {
    int np, nch;
    const int32_t *lo, *hi, *pid, *pc;  // chunk rows [lo, hi) of problem pid; problem p owns chunks [pc[p], pc[p+1])
    double *part;                       // 2 * nch chunk sums
    unsigned *counter;                  // arrivals (the last block resets it)
    double *d;
    int32_t *iv;
    double rtol;
    int maxit;
};

// Per-problem scalars from the chunk sums, in chunk order (the last block).
template <int NV>
__device__ void bcg_finish(const BCg &g, int mode, int flex) {
    for (int p = threadIdx.x; p < g.np; p += blockDim.x) {
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double a = 0.0;
            for (int c = g.pc[p]; c < g.pc[p + 1]; c++) a += __ldcg(&g.part[k * g.nch + c]);
            s[k] = a;
        }
        double *d = g.d;
        int32_t *iv = g.iv;
        const int np = g.np;
        const bool act = iv[I_ACT * np + p] != 0;
        switch (mode) {
            case BM_NB: {
                const double nb = sqrt(s[0]);
                d[D_NB * np + p] = nb == 0.0 ? 1.0 : nb;
                break;
            }
            case BM_R0: {
                d[D_RR * np + p] = s[0];
                d[D_R0 * np + p] = sqrt(s[0]);
                const bool conv = sqrt(s[0]) / d[D_NB * np + p] < g.rtol;
                iv[I_IT * np + p] = 0;
                iv[I_CONV * np + p] = conv ? 1 : 0;
                iv[I_ACT * np + p] = (!conv && g.maxit > 0) ? 1 : 0;
                break;
            }
            case BM_RZ_FIRST:
            case BM_RZ: {
                if (!act) break;
                const double zro = NV > 1 ? s[NV - 1] : 0.0;
                d[D_RZP * np + p] = d[D_RZ * np + p];
                d[D_RZ * np + p] = s[0];
                d[D_ZRO * np + p] = zro;
                d[D_BETA * np + p] = mode == BM_RZ_FIRST ? 0.0 : (flex ? s[0] - zro : s[0]) / d[D_RZP * np + p];
                break;
            }
            case BM_PQ:
                if (!act) break;
                d[D_PQ * np + p] = s[0];
                d[D_ALPHA * np + p] = d[D_RZ * np + p] / s[0];
                break;
            case BM_XR: {
                if (!act) break;
                d[D_RR * np + p] = s[0];
                const int it = ++iv[I_IT * np + p];
                const bool conv = sqrt(s[0]) / d[D_NB * np + p] < g.rtol;
                iv[I_CONV * np + p] = conv ? 1 : 0;
                if (conv || it >= g.maxit) iv[I_ACT * np + p] = 0;
                break;
            }
            case BM_FINAL: d[D_RRF * np + p] = s[0]; break;
            default: break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int p = 0; p < g.np; p++) a += g.iv[I_ACT * g.np + p];
        g.iv[kI * g.np] = a;
    }
}

// Chunk sums to part, then the last block to arrive finishes.
template <int NV>
__device__ void bcg_arrive(const BCg &g, int mode, int flex) {
    __shared__ int am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = atomicAdd(g.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    bcg_finish<NV>(g, mode, flex);
    if (threadIdx.x == 0) {
        *g.counter = 0u;
        __threadfence();
    }
}

// s0 = <a0, b0> (and s1 = <a1, b1>) per problem.  Rows of problems that
// stopped iterating are skipped in the CG modes.
template <int NV>
__global__ void __launch_bounds__(kBT)
bcg_dot_kernel(BCg g, int mode, int flex, const double *__restrict__ a0, const double *__restrict__ b0,
               const double *__restrict__ a1, const double *__restrict__ b1) {
    pdl_wait();
    __shared__ double sm[32];
    const bool cg_mode = mode == BM_RZ || mode == BM_RZ_FIRST || mode == BM_PQ;
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] = 0.0;
        if (!cg_mode || g.iv[I_ACT * g.np + g.pid[c]]) {
            for (int32_t i = g.lo[c] + threadIdx.x; i < g.hi[c]; i += kBT) {
                acc[0] = fma(a0[i], b0[i], acc[0]);
                if (NV > 1) acc[NV - 1] = fma(a1[i], b1[i], acc[NV - 1]);
            }
        }
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const double t = block_sum<kBT>(acc[k], sm);
            if (threadIdx.x == 0) g.part[k * g.nch + c] = t;
        }
    }
    bcg_arrive<NV>(g, mode, flex);
}

// p = z (first) or z + beta p, on problems still iterating
__global__ void __launch_bounds__(kBT)
bcg_p_kernel(BCg g, double *__restrict__ p, const double *__restrict__ z, int first) {
    pdl_wait();
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        const int q = g.pid[c];
        if (!g.iv[I_ACT * g.np + q]) continue;
        const double beta = g.d[D_BETA * g.np + q];
        for (int32_t i = g.lo[c] + threadIdx.x; i < g.hi[c]; i += kBT) p[i] = first ? z[i] : z[i] + beta * p[i];
    }
}

// x += alpha p, (r_old = r), r -= alpha q, ||r||^2 and the stopping test per problem
__global__ void __launch_bounds__(kBT)
bcg_xr_kernel(BCg g, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
              const double *__restrict__ q, double *__restrict__ rold) {
    pdl_wait();
    __shared__ double sm[32];
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        const int pp = g.pid[c];
        double acc = 0.0;
        if (g.iv[I_ACT * g.np + pp]) {
            const double a = g.d[D_ALPHA * g.np + pp];
            for (int32_t i = g.lo[c] + threadIdx.x; i < g.hi[c]; i += kBT) {
                x[i] = x[i] + a * p[i];
                const double rv = r[i];
                if (rold) rold[i] = rv;
                const double rn = rv - a * q[i];
                r[i] = rn;
                acc = fma(rn, rn, acc);
            }
        }
        const double t = block_sum<kBT>(acc, sm);
        if (threadIdx.x == 0) g.part[c] = t;
    }
    bcg_arrive<1>(g, BM_XR, 0);
}

// ---------------------------------------------------------------- tile lists
// A merged matrix's staged SpMV walks a list of tiles (kS / G rows each).
// While the CG runs, a tile stays listed only if one of its rows belongs to a
// problem still iterating: the others' rows keep their last values, which no
// later step of an active problem reads (the operators are block diagonal).
struct TileListDesc {
    int32_t n, rpt, ntiles;
    const int32_t *off;  // np + 1 row offsets of the problems in the matrix's rows
    int32_t *list, *count;
};

constexpr int kListThreads = 1024;

// One block per list; tiles in ascending order (an ordered block-wide scan).
__global__ void __launch_bounds__(kListThreads)
tile_list_kernel(const TileListDesc *__restrict__ D, int np, const int32_t *__restrict__ act, int all) {
    pdl_wait();
    __shared__ int32_t wsum[kListThreads / 32];
    __shared__ int32_t base;
    const TileListDesc d = D[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int32_t t0 = 0; t0 < d.ntiles; t0 += kListThreads) {
        const int32_t t = t0 + threadIdx.x;
        int keep = 0;
        if (t < d.ntiles) {
            keep = all;
            if (!keep) {
                const int32_t r0 = t * d.rpt, r1 = min(d.n, r0 + d.rpt) - 1;
                int lo = 0, hi = np - 1;  // the problem of row r0: the largest p with off[p] <= r0
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (d.off[mid] <= r0) lo = mid;
                    else hi = mid - 1;
                }
                for (int p = lo; p < np && d.off[p] <= r1 && !keep; p++) keep = act[p] != 0;
            }
        }
        int v = keep;  // inclusive scan within the warp, then over the warps
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        if (w == 0) {
            int x = lane < kListThreads / 32 ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            if (lane < kListThreads / 32) wsum[lane] = x;  // inclusive warp totals
        }
        __syncthreads();
        const int before = v - keep + (w > 0 ? wsum[w - 1] : 0);
        if (keep) d.list[base + before] = t;
        __syncthreads();
        if (threadIdx.x == 0) base += wsum[kListThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *d.count = base;
}

// ---------------------------------------------------------------- merging
struct MergeBlk {
    const int32_t *rp, *col;
    const double *val;
    int32_t row0, nrows, col0;
    int kind;  // 0: copy the source rows, 1: identity rows, 2: empty rows
    int64_t nz0, nnz;
};

__device__ __forceinline__ int find_row_block(int nb, const MergeBlk *B, int64_t i) {
    int lo = 0, hi = nb - 1;  // the largest b with row0 <= i (every block has rows)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B[mid].row0 <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void merge_rowptr_kernel(int nb, const MergeBlk *__restrict__ B, int32_t ntot, int64_t nztot,
                                    int32_t *__restrict__ rp) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ntot; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == ntot) {
            rp[i] = (int32_t)nztot;
            continue;
        }
        const MergeBlk &k = B[find_row_block(nb, B, i)];
        const int32_t li = (int32_t)(i - k.row0);
        rp[i] = (int32_t)(k.nz0 + (k.kind == 0 ? k.rp[li] : k.kind == 1 ? li : 0));
    }
}

__global__ void merge_entries_kernel(int nb, const MergeBlk *__restrict__ B, int64_t nztot, int32_t *__restrict__ col,
                                     double *__restrict__ val) {
    pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nztot; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nb - 1;  // the largest b with nz0 <= e: blocks without entries are passed over
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B[mid].nz0 <= e) lo = mid;
            else hi = mid - 1;
        }
        const MergeBlk &k = B[lo];
        const int64_t le = e - k.nz0;
        if (k.kind == 0) {
            col[e] = k.col[le] + k.col0;
            val[e] = k.val[le];
        } else {
            col[e] = k.col0 + (int32_t)le;
            val[e] = 1.0;
        }
    }
}

// One merged matrix from per-problem blocks (rows and columns offset).
void merge_matrix(const std::vector<MergeBlk> &blk, int32_t ncols, DCsr &out, cudaStream_t s) {
    const int nb = (int)blk.size();
    int32_t ntot = 0;
    int64_t nztot = 0;
    for (const MergeBlk &b : blk) {
        ntot += b.nrows;
        nztot += b.nnz;
    }
    if (nztot > INT32_MAX - 1) fail(RN_EINVAL, "merged batch: a level has more than 2^31 - 1 entries");
    out.n = ntot;
    out.m = ncols;
    out.nnz = nztot;
    DVec<unsigned char> bd(sizeof(MergeBlk) * nb, s);
    h2d(bd.p, reinterpret_cast<const unsigned char *>(blk.data()), sizeof(MergeBlk) * nb, s);
    const MergeBlk *B = reinterpret_cast<const MergeBlk *>(bd.p);
    out.rowptr.alloc(ntot + 1, s);
    out.col.alloc(nztot, s);
    out.val.alloc(nztot, s);
    RN_LAUNCH("batch_merge", 4.0 * ntot, s, merge_rowptr_kernel, grid_for(ntot + 1, 1024), 256, 0, nb, B, ntot, nztot,
              out.rowptr.p);
    if (nztot)
        RN_LAUNCH("batch_merge", 24.0 * nztot, s, merge_entries_kernel, grid_for(nztot, 1024), 256, 0, nb, B, nztot,
                  out.col.p, out.val.p);
    // bd is released stream-ordered after the kernels; blk was staged by the upload
}

BCg bcg_of(rn_batch &b) {
    BCg g{};
    g.np = b.np;
    g.nch = b.nch;
    g.lo = b.ch_lo.p;
    g.hi = b.ch_hi.p;
    g.pid = b.ch_pid.p;
    g.pc = b.pc.p;
    g.part = b.part.p;
    g.counter = b.counter.p;
    g.d = b.d.p;
    g.iv = b.iv.p;
    g.rtol = b.rtol;
    g.maxit = b.maxit;
    return g;
}

int bgrid(const rn_batch &b) { return std::max(1, std::min(b.nch, num_sms() * 8)); }

void launch_dot(rn_batch &b, int mode, const double *a0, const double *b0, const double *a1 = nullptr,
                const double *b1 = nullptr) {
    cudaStream_t s = b.M->s;
    const int64_t n = b.M->lev[0]->A.n;
    const BCg g = bcg_of(b);
    if (a1)
        RN_LAUNCH("batch_cg_dot", 32.0 * n, s, bcg_dot_kernel<2>, bgrid(b), kBT, 0, g, mode, b.flexible ? 1 : 0, a0,
                  b0, a1, b1);
    else
        RN_LAUNCH("batch_cg_dot", 16.0 * n, s, bcg_dot_kernel<1>, bgrid(b), kBT, 0, g, mode, b.flexible ? 1 : 0, a0,
                  b0, a0, b0);
}

// One CG iteration: q = A p, alpha, x and r with the stopping test, then
// z = M r, beta and p for the problems still iterating.
void batch_iteration(rn_batch &b) {
    rn_hierarchy &M = *b.M;
    cudaStream_t s = M.s;
    const int64_t n = M.lev[0]->A.n;
    const BCg g = bcg_of(b);
    outer_spmv(M, M.pv.p, M.q.p);
    launch_dot(b, BM_PQ, M.pv.p, M.q.p);
    RN_LAUNCH("batch_cg_vec", 48.0 * n, s, bcg_xr_kernel, bgrid(b), kBT, 0, g, b.xm.p, M.r.p, M.pv.p, M.q.p,
              b.flexible ? M.rold.p : nullptr);
    cycle_launches(M, M.r.p, M.z.p);
    if (b.flexible) launch_dot(b, BM_RZ, M.r.p, M.z.p, M.z.p, M.rold.p);
    else launch_dot(b, BM_RZ, M.r.p, M.z.p);
    RN_LAUNCH("batch_cg_vec", 24.0 * n, s, bcg_p_kernel, bgrid(b), kBT, 0, g, M.pv.p, M.z.p, 0);
}

void gather(rn_batch &b, const double *const *src, double *dst) {
    for (int p = 0; p < b.np; p++) d2d(dst + b.off0[p], src[p], (size_t)(b.off0[p + 1] - b.off0[p]), b.M->s);
}

void scatter(rn_batch &b, const double *src, double *const *dst) {
    for (int p = 0; p < b.np; p++) d2d(dst[p], src + b.off0[p], (size_t)(b.off0[p + 1] - b.off0[p]), b.M->s);
}

// Relist the tiles of every merged matrix (all: every tile).
void relist(rn_batch &b, bool all) {
    if (b.nlists == 0) return;
    RN_LAUNCH("batch_tile_list", 0, b.M->s, tile_list_kernel, b.nlists, kListThreads, 0,
              reinterpret_cast<const TileListDesc *>(b.lists.p), b.np, b.iv.p + I_ACT * b.np, all ? 1 : 0);
}

// Tile lists for one matrix whose rows are split among the problems by off.
void add_lists(rn_batch &b, DCsr &M, const int32_t *off, std::vector<TileListDesc> &out) {
    cudaStream_t s = b.M->s;
    if (M.n == 0) return;
    M.tcnt.alloc(2, s);
    const int groups[2] = {M.tile_group, M.tile_group64};
    for (int f = 0; f < 2; f++) {
        const int G = groups[f];
        if (G == 0) continue;  // rows too long for a stage: the unstaged kernel, every row
        const int32_t rpt = kS / G, nt = (M.n + rpt - 1) / rpt;
        DVec<int32_t> &L = f ? M.tl64 : M.tl32;
        L.alloc(nt, s);
        out.push_back(TileListDesc{M.n, rpt, nt, off, L.p, M.tcnt.p + f});
    }
}

}  // namespace

rn_batch *batch_merge(int count, rn_hierarchy *const *hs, cudaStream_t s) {
    const rn_hierarchy &h0 = *hs[0];
    int Lm = 0;
    for (int p = 0; p < count; p++) {
        const rn_hierarchy &h = *hs[p];
        if (h.p.precision != h0.p.precision || h.p.omega != h0.p.omega || h.p.nu_pre != h0.p.nu_pre ||
            h.p.nu_post != h0.p.nu_post)
            fail(RN_EINVAL, fmt("merged batch: problem %d's cycle settings differ from problem 0's "
                                "(precision, omega, nu_pre, nu_post)", p));
        if (h.p.gamma != 1) fail(RN_EINVAL, "merged batch: V-cycles only (gamma 1)");
        Lm = std::max(Lm, (int)h.lev.size());
    }
    std::unique_ptr<rn_batch> b(new rn_batch());
    b->np = count;
    b->M.reset(new rn_hierarchy());
    rn_hierarchy &M = *b->M;
    M.p = h0.p;
    M.p.coarse_cluster = 0;  // the merged coarse levels run level by level
    M.p.outer = RN_OUTER_CG;
    M.p.stream = s;
    M.s = s;
    M.pdl = h0.pdl;
    M.partial.alloc(2 * kReduceBlocks, s);
    M.counters.alloc(4, s);
    RN_CUDA_CHECK(cudaMemsetAsync(M.counters.p, 0, 4 * sizeof(unsigned), s));
    M.scal.alloc(64, s);
    M.iflags.alloc(16, s);
    fill_f64(M.scal.p, 0.0, 64, s);
    fill_i32(M.iflags.p, 0, 16, s);
    // rows of problem p on merged level l: its level min(l, L_p - 1)
    auto rows = [&](int p, int l) {
        const rn_hierarchy &h = *hs[p];
        return h.lev[std::min(l, (int)h.lev.size() - 1)]->A.n;
    };
    std::vector<std::vector<int32_t>> off(Lm, std::vector<int32_t>(count + 1, 0));
    for (int l = 0; l < Lm; l++)
        for (int p = 0; p < count; p++) off[l][p + 1] = off[l][p] + rows(p, l);
    for (int l = 0; l < Lm; l++) {
        auto L = std::make_unique<rn_level>();
        const int32_t nl = off[l][count];
        // A: the problem's own rows on its levels, none below
        std::vector<MergeBlk> blk(count);
        int64_t nz = 0;
        for (int p = 0; p < count; p++) {
            const rn_hierarchy &h = *hs[p];
            const int Lp = (int)h.lev.size();
            MergeBlk &k = blk[p];
            k = MergeBlk{};
            k.row0 = off[l][p];
            k.nrows = rows(p, l);
            k.col0 = off[l][p];
            k.nz0 = nz;
            if (l < Lp) {
                const DCsr &A = h.lev[l]->A;
                k.kind = 0;
                k.rp = A.rowptr.p;
                k.col = A.col.p;
                k.val = A.val.p;
                k.nnz = A.nnz;
            } else {
                k.kind = 2;
                k.nnz = 0;
            }
            nz += k.nnz;
        }
        merge_matrix(blk, nl, L->A, s);
        // diagonal: the problem's own where it relaxes; +inf (weight 0) where it passes through
        L->diag.alloc(nl, s);
        for (int p = 0; p < count; p++) {
            const rn_hierarchy &h = *hs[p];
            const int Lp = (int)h.lev.size();
            if (l < Lp - 1) d2d(L->diag.p + off[l][p], h.lev[l]->diag.p, (size_t)rows(p, l), s);
            else fill_f64(L->diag.p + off[l][p], INFINITY, rows(p, l), s);
        }
        if (l < Lm - 1) {
            // P (rows of level l, columns of level l + 1) and R (the reverse); identity where passed through
            std::vector<MergeBlk> bp(count), br(count);
            int64_t nzp = 0, nzr = 0;
            for (int p = 0; p < count; p++) {
                const rn_hierarchy &h = *hs[p];
                const int Lp = (int)h.lev.size();
                MergeBlk &kp = bp[p], &kr = br[p];
                kp = MergeBlk{};
                kr = MergeBlk{};
                kp.row0 = off[l][p];
                kp.nrows = rows(p, l);
                kp.col0 = off[l + 1][p];
                kp.nz0 = nzp;
                kr.row0 = off[l + 1][p];
                kr.nrows = rows(p, l + 1);
                kr.col0 = off[l][p];
                kr.nz0 = nzr;
                if (l < Lp - 1) {
                    const DCsr &P = h.lev[l]->P, &R = h.lev[l]->R;
                    kp.kind = kr.kind = 0;
                    kp.rp = P.rowptr.p;
                    kp.col = P.col.p;
                    kp.val = P.val.p;
                    kp.nnz = P.nnz;
                    kr.rp = R.rowptr.p;
                    kr.col = R.col.p;
                    kr.val = R.val.p;
                    kr.nnz = R.nnz;
                } else {
                    kp.kind = kr.kind = 1;
                    kp.nnz = kp.nrows;
                    kr.nnz = kr.nrows;
                }
                nzp += kp.nnz;
                nzr += kr.nnz;
            }
            merge_matrix(bp, off[l + 1][count], L->P, s);
            merge_matrix(br, nl, L->R, s);
            L->nc = off[l + 1][count];
        }
        M.lev.push_back(std::move(L));
    }
    // the last level: every problem's coarsest inverse, block diagonal
    {
        std::vector<int32_t> ro(count + 1);
        std::vector<int64_t> ao(count + 1, 0);
        for (int p = 0; p <= count; p++) ro[p] = off[Lm - 1][p];
        for (int p = 0; p < count; p++) {
            const int64_t nL = hs[p]->nL;
            if ((int64_t)hs[p]->Ainv.n != nL * nL || nL != rows(p, Lm - 1))
                fail(RN_EINTERNAL, "merged batch: a hierarchy's coarsest inverse does not match its coarsest level");
            ao[p + 1] = ao[p] + nL * nL;
        }
        M.Ainv.alloc((size_t)ao[count], s);
        for (int p = 0; p < count; p++) d2d(M.Ainv.p + ao[p], hs[p]->Ainv.p, (size_t)(ao[p + 1] - ao[p]), s);
        M.cblk_row.alloc(count + 1, s);
        M.cblk_inv.alloc(count + 1, s);
        h2d(M.cblk_row.p, ro.data(), count + 1, s);
        h2d(M.cblk_inv.p, ao.data(), count + 1, s);
        M.ncblk = count;
        M.nL = ro[count];
    }
    prepare_solve(M);
    // level-0 layout and the reduction chunks
    b->off0 = off[0];
    std::vector<int32_t> lo, hi, pid, pc(count + 1, 0);
    for (int p = 0; p < count; p++) {
        pc[p] = (int32_t)lo.size();
        for (int32_t r = off[0][p]; r < off[0][p + 1]; r += kChunk) {
            lo.push_back(r);
            hi.push_back(std::min(r + kChunk, off[0][p + 1]));
            pid.push_back(p);
        }
    }
    pc[count] = (int32_t)lo.size();
    b->nch = (int)lo.size();
    b->ch_lo.alloc(b->nch, s);
    b->ch_hi.alloc(b->nch, s);
    b->ch_pid.alloc(b->nch, s);
    b->pc.alloc(count + 1, s);
    h2d(b->ch_lo.p, lo.data(), b->nch, s);
    h2d(b->ch_hi.p, hi.data(), b->nch, s);
    h2d(b->ch_pid.p, pid.data(), b->nch, s);
    h2d(b->pc.p, pc.data(), count + 1, s);
    b->part.alloc(2 * (size_t)b->nch, s);
    b->counter.alloc(1, s);
    RN_CUDA_CHECK(cudaMemsetAsync(b->counter.p, 0, sizeof(unsigned), s));
    b->d.alloc((size_t)kD * count, s);
    b->iv.alloc((size_t)kI * count + 1, s);
    fill_f64(b->d.p, 0.0, (int64_t)kD * count, s);
    fill_i32(b->iv.p, 0, (int64_t)kI * count + 1, s);
    b->bm.alloc(off[0][count], s);
    b->xm.alloc(off[0][count], s);
    b->flexible = M.p.precision == RN_MIXED;
    // tile lists of every merged matrix, all tiles to begin with
    {
        std::vector<int32_t> oh((size_t)Lm * (count + 1));
        for (int l = 0; l < Lm; l++) std::copy(off[l].begin(), off[l].end(), oh.begin() + (size_t)l * (count + 1));
        b->offs.alloc(oh.size(), s);
        h2d(b->offs.p, oh.data(), oh.size(), s);
        std::vector<TileListDesc> D;
        for (int l = 0; l < Lm; l++) {
            rn_level &L = *M.lev[l];
            const int32_t *ol = b->offs.p + (size_t)l * (count + 1);
            add_lists(*b, L.A, ol, D);
            if (l < Lm - 1) {
                add_lists(*b, L.P, ol, D);
                add_lists(*b, L.R, ol + (count + 1), D);
            }
        }
        b->nlists = (int)D.size();
        b->lists.alloc(sizeof(TileListDesc) * D.size(), s);
        h2d(b->lists.p, reinterpret_cast<const unsigned char *>(D.data()), sizeof(TileListDesc) * D.size(), s);
        relist(*b, true);
    }
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    return b.release();
}

void batch_cycle(rn_batch &b, const double *const *rhs, double *const *out) {
    relist(b, true);  // every tile (a failed call may have left lists short)
    gather(b, rhs, b.bm.p);
    apply_cycle(*b.M, b.bm.p, b.xm.p);
    scatter(b, b.xm.p, out);
    RN_CUDA_CHECK(cudaStreamSynchronize(b.M->s));
    if (read_scalar(b.M->iflags.p + 8, b.M->s))
        fail(RN_ETIMEOUT, "a shared-memory staging wait gave up (bulk copy did not complete)");
}

rn_status batch_solve(rn_batch &b, const double *const *rhs, double *const *x, double rtol, int maxit,
                      rn_solve_info *info) {
    rn_hierarchy &M = *b.M;
    cudaStream_t s = M.s;
    const double t0 = now_ms();
    b.rtol = rtol;
    b.maxit = maxit;
    relist(b, true);  // every tile (a failed call may have left lists short)
    gather(b, rhs, b.bm.p);
    gather(b, x, b.xm.p);
    launch_dot(b, BM_NB, b.bm.p, b.bm.p);
    outer_residual(M, b.xm.p, b.bm.p, M.r.p);
    launch_dot(b, BM_R0, M.r.p, M.r.p);
    // the first preconditioned direction
    apply_cycle(M, M.r.p, M.z.p);
    launch_dot(b, BM_RZ_FIRST, M.r.p, M.z.p);
    RN_LAUNCH("batch_cg_vec", 16.0 * M.lev[0]->A.n, s, bcg_p_kernel, bgrid(b), kBT, 0, bcg_of(b), M.pv.p, M.z.p, 1);
    // iterations: one graph per iteration (its scalars live on the device, so
    // the graph is rebuilt only when the tolerance or limit changes)
    if (!b.it_exec || b.graph_rtol != rtol || b.graph_maxit != maxit) {
        if (b.it_exec) cudaGraphExecDestroy(b.it_exec);
        if (b.it_graph) cudaGraphDestroy(b.it_graph);
        b.it_exec = nullptr;
        b.it_graph = nullptr;
        const int64_t before = launches_so_far();
        RN_CUDA_CHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            batch_iteration(b);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        RN_CUDA_CHECK(cudaStreamEndCapture(s, &b.it_graph));
        RN_CUDA_CHECK(cudaGraphInstantiate(&b.it_exec, b.it_graph, 0));
        b.it_kernels = launches_so_far() - before;
        add_launches(-b.it_kernels);
        b.graph_rtol = rtol;
        b.graph_maxit = maxit;
    }
    int launched = 0, listed = b.np;
    for (;;) {
        const int active = read_scalar(b.iv.p + (size_t)kI * b.np, s);
        if (active == 0 || launched >= maxit) break;
        if (active < listed) {  // problems stopped: drop their tiles
            relist(b, false);
            listed = active;
        }
        const int k = std::min(kItersPerPoll, maxit - launched);
        for (int j = 0; j < k; j++) RN_CUDA_CHECK(cudaGraphLaunch(b.it_exec, s));
        add_launches((int64_t)k * b.it_kernels);
        launched += k;
    }
    relist(b, true);
    // true residuals, then every problem's record
    outer_residual(M, b.xm.p, b.bm.p, M.r.p);
    launch_dot(b, BM_FINAL, M.r.p, M.r.p);
    scatter(b, b.xm.p, x);
    std::vector<double> d((size_t)kD * b.np);
    std::vector<int32_t> iv((size_t)kI * b.np + 1);
    d2h(d.data(), b.d.p, d.size(), s);
    d2h(iv.data(), b.iv.p, iv.size(), s);
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    if (read_scalar(M.iflags.p + 8, s)) {
        RN_CUDA_CHECK(cudaMemsetAsync(M.iflags.p + 8, 0, sizeof(int32_t), s));
        fail(RN_ETIMEOUT, "a shared-memory staging wait gave up (bulk copy did not complete)");
    }
    const double ms = now_ms() - t0;
    rn_status st = RN_OK;
    const int np = b.np;
    for (int p = 0; p < np; p++) {
        const double nb = d[D_NB * np + p], rn = std::sqrt(d[D_RRF * np + p]), r0 = d[D_R0 * np + p];
        const int it = iv[I_IT * np + p];
        const rn_status sp = rn / nb < rtol ? RN_OK : RN_ENOTCONV;
        if (sp != RN_OK) st = sp;
        if (info) {
            info[p].iters = it;
            info[p].rel_res = rn / nb;
            info[p].rho = (it > 0 && r0 > 0.0) ? std::pow(rn / r0, 1.0 / it) : 0.0;
            info[p].solve_ms = ms;
            info[p].status = sp;
        }
    }
    return st;
}

}  // namespace rn
