// rn_spgemm.cu - sparse-sparse products on the GPU.
//
// * spgemm_symbolic: the pattern of C = A B (the symbolic product; explicit
//   zeros kept).  One warp per row inserts the columns of the rows B_k,
//   k in A_i, into a 1024-slot shared-memory hash table; rows with more than
//   512 distinct columns move to a block-per-row tier with a 32768-slot
//   table in dynamic shared memory.  Two passes: count, then fill with a rank
//   sort of the row's keys, so every row comes out sorted.
// * masked product (one kernel, three uses): for each output row i, G lanes
//   walk the entries a_ik of A_i in ascending k and, for each k, the entries
//   of X_k; a product lands in the output only when its column is in row i's
//   pattern (binary search in a shared-memory copy of the row's columns).
//   Every output entry therefore accumulates its terms in ascending k.
//     - numeric SpGEMM (output pattern = symbolic product);
//     - exact mode: rounded multiply then rounded add (no FMA), which gives
//       bit-identical values to a sequential CPU evaluation in the same
//       order - used for N = S^d C, whose values drive the pre-filter;
//     - energy minimisation: W = scale * Proj(Mask_N(A X)) with the row-wise
//       constraint projection (eq. Tproj with zero right-hand side) fused in
//       the epilogue, plus the Frobenius product <Y, W>.
#include "rn_internal.cuh"

namespace rn {

// ------------------------------------------------------------------ symbolic
constexpr int kHashSlots = 1024;        // per warp (fast tier)
constexpr int kHashMaxUnique = kHashSlots / 2;
constexpr int kSymWarps = 4;            // warps per block (fast tier)
constexpr int kBigSlots = 32768;        // block tier
constexpr int kBigMaxUnique = kBigSlots / 2;
constexpr int kBigThreads = 512;

__device__ __forceinline__ uint32_t hash_slot(int32_t key, uint32_t bits) {
    return ((uint32_t)key * 2654435761u) >> (32 - bits);
}

// 1 = inserted, 0 = present, -1 = table full
__device__ __forceinline__ int hash_insert(int32_t *tab, uint32_t bits, int32_t key) {
    const uint32_t cap = 1u << bits;
    uint32_t h = hash_slot(key, bits);
    for (uint32_t p = 0; p < cap; p++) {
        int32_t old = atomicCAS(&tab[h], -1, key);
        if (old == -1) return 1;
        if (old == key) return 0;
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

template <bool FILL>
__global__ void __launch_bounds__(kSymWarps * 32)
sym_warp_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol, int32_t *__restrict__ count,
                int32_t *__restrict__ ovf_list, int32_t *__restrict__ ovf_n, const int32_t *__restrict__ crp,
                int32_t *__restrict__ ccol) {
    __shared__ int32_t tab[kSymWarps][kHashSlots];
    __shared__ int32_t list[kSymWarps][kHashMaxUnique];
    __shared__ int32_t cnt[kSymWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int32_t i = blockIdx.x * kSymWarps + w; i < n; i += gridDim.x * kSymWarps) {
        if (FILL && crp[i + 1] - crp[i] > kHashMaxUnique) continue;  // long row: block tier
        // table size: the smallest power of two >= 2 x (products in the row), 32..1024
        int32_t ub = 0;
        for (int32_t e = arp[i] + lane; e < arp[i + 1]; e += 32) ub += brp[acol[e] + 1] - brp[acol[e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ub += __shfl_xor_sync(0xffffffffu, ub, o);
        uint32_t bits = 5;
        while (bits < 10 && (1 << bits) < 2 * ub) bits++;
        const int slots = 1 << bits;
        for (int s = lane; s < slots; s += 32) tab[w][s] = -1;
        if (lane == 0) cnt[w] = 0;
        __syncwarp();
        bool ovf = false;
        for (int32_t e = arp[i]; e < arp[i + 1] && !ovf; e++) {
            const int32_t k = acol[e];
            bool full = false;
            for (int32_t f = brp[k] + lane; f < brp[k + 1]; f += 32) {
                int r = hash_insert(tab[w], bits, bcol[f]);
                if (r == 1) atomicAdd(&cnt[w], 1);
                if (r < 0) full = true;
            }
            __syncwarp();
            ovf = __any_sync(0xffffffffu, full) || cnt[w] > kHashMaxUnique;
        }
        if (!FILL) {
            if (lane == 0) {
                if (ovf) {
                    count[i] = -1;
                    ovf_list[atomicAdd(ovf_n, 1)] = i;
                } else {
                    count[i] = cnt[w];
                }
            }
        } else {
            // compact the keys, then rank-sort them into the row
            int base = 0;
            for (int s0 = 0; s0 < slots; s0 += 32) {
                int32_t key = tab[w][s0 + lane];
                unsigned b = __ballot_sync(0xffffffffu, key >= 0);
                if (key >= 0) list[w][base + __popc(b & ((1u << lane) - 1u))] = key;
                base += __popc(b);
            }
            __syncwarp();
            const int32_t dst = crp[i];
            for (int e = lane; e < base; e += 32) {
                int32_t key = list[w][e];
                int rank = 0;
                for (int f = 0; f < base; f++) rank += (list[w][f] < key);
                ccol[dst + rank] = key;
            }
        }
        __syncwarp();
    }
}

template <bool FILL>
__global__ void __launch_bounds__(kBigThreads)
sym_block_kernel(const int32_t *__restrict__ rows, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                 const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol, int32_t *__restrict__ count,
                 const int32_t *__restrict__ crp, int32_t *__restrict__ ccol, int32_t *__restrict__ err) {
    extern __shared__ int32_t big[];
    int32_t *tab = big;                 // kBigSlots
    int32_t *list = big + kBigSlots;    // kBigMaxUnique
    __shared__ int32_t cnt, bad;
    const int32_t i = rows[blockIdx.x];
    for (int s = threadIdx.x; s < kBigSlots; s += blockDim.x) tab[s] = -1;
    if (threadIdx.x == 0) { cnt = 0; bad = 0; }
    __syncthreads();
    constexpr uint32_t bits = 15;
    for (int32_t e = arp[i]; e < arp[i + 1]; e++) {
        const int32_t k = acol[e];
        for (int32_t f = brp[k] + threadIdx.x; f < brp[k + 1]; f += blockDim.x) {
            int r = hash_insert(tab, bits, bcol[f]);
            if (r == 1) atomicAdd(&cnt, 1);
            if (r < 0) bad = 1;
        }
        __syncthreads();
        if (bad || cnt > kBigMaxUnique) break;
    }
    __syncthreads();
    if (bad || cnt > kBigMaxUnique) {
        if (threadIdx.x == 0) atomicMax(err, i + 1);
        return;
    }
    if (!FILL) {
        if (threadIdx.x == 0) count[i] = cnt;
        return;
    }
    __shared__ int32_t u;
    if (threadIdx.x == 0) u = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < kBigSlots; s += blockDim.x) {
        int32_t key = tab[s];
        if (key >= 0) list[atomicAdd(&u, 1)] = key;
    }
    __syncthreads();
    const int32_t dst = crp[i];
    for (int e = threadIdx.x; e < u; e += blockDim.x) {
        int32_t key = list[e];
        int rank = 0;
        for (int f = 0; f < u; f++) rank += (list[f] < key);
        ccol[dst + rank] = key;
    }
}

void spgemm_symbolic(const CsrView &A, const CsrView &B, DCsr &C, cudaStream_t s) {
    if (A.m != B.n) fail(RN_EINTERNAL, "spgemm_symbolic: inner dimensions differ");
    C.n = A.n;
    C.m = B.m;
    DVec<int32_t> count(A.n + 1, s), ovf_list(A.n > 0 ? A.n : 1, s), flags(2, s);
    fill_i32(flags.p, 0, 2, s);
    const int grid = grid_for(A.n, kSymWarps, 16);
    const double bytes_sym = 12.0 * A.nnz + 8.0 * A.n;  // the product's inputs are read through L2
    if (A.n)
        RN_LAUNCH("spgemm_symbolic", bytes_sym, s, sym_warp_kernel<false>, grid, kSymWarps * 32, 0, A.n, A.rowptr,
                  A.col, B.rowptr, B.col, count.p, ovf_list.p, flags.p, nullptr, nullptr);
    const int32_t novf = read_scalar(flags.p, s);
    const size_t big_smem = (size_t)(kBigSlots + kBigMaxUnique) * sizeof(int32_t);
    if (novf > 0) {
        RN_CUDA_CHECK(cudaFuncSetAttribute(sym_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)big_smem));
        RN_CUDA_CHECK(cudaFuncSetAttribute(sym_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)big_smem));
        RN_LAUNCH("spgemm_symbolic_long", 0, s, sym_block_kernel<false>, novf, kBigThreads, big_smem, ovf_list.p,
                  A.rowptr, A.col, B.rowptr, B.col, count.p, nullptr, nullptr, flags.p + 1);
        int32_t err = read_scalar(flags.p + 1, s);
        if (err) fail(RN_EINTERNAL, fmt("product row %d has more than %d distinct columns", err - 1, kBigMaxUnique));
    }
    C.rowptr.alloc(A.n + 1, s);
    C.nnz = scan_counts(count.p, C.rowptr.p, A.n, s);
    C.col.alloc(C.nnz, s);
    if (A.n)
        RN_LAUNCH("spgemm_symbolic", bytes_sym + 4.0 * C.nnz, s, sym_warp_kernel<true>, grid, kSymWarps * 32, 0, A.n,
                  A.rowptr, A.col, B.rowptr, B.col, nullptr, nullptr, nullptr, C.rowptr.p, C.col.p);
    if (novf > 0)
        RN_LAUNCH("spgemm_symbolic_long", 0, s, sym_block_kernel<true>, novf, kBigThreads, big_smem, ovf_list.p,
                  A.rowptr, A.col, B.rowptr, B.col, nullptr, C.rowptr.p, C.col.p, flags.p + 1);
}

// ------------------------------------------------------------------ masked numeric product
constexpr int kMpThreads = 256;

template <int G, bool EXACT, bool PROJ>
__global__ void __launch_bounds__(kMpThreads, 4)
masked_product_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                      const double *__restrict__ aval, const int32_t *__restrict__ xrp,
                      const int32_t *__restrict__ xcol, const double *__restrict__ xval,
                      const int32_t *__restrict__ crp, const int32_t *__restrict__ ccol, double *__restrict__ cval,
                      const int32_t *__restrict__ rowtype, const double *__restrict__ Bc, double scale,
                      const double *__restrict__ Y, Fin fin) {
    constexpr int GPB = kMpThreads / G;  // groups per block
    constexpr int CAP = 8 * G;           // pattern columns per chunk
    __shared__ int32_t s_col[GPB][CAP];
    __shared__ double s_acc[GPB][CAP];
    __shared__ double s_red[32];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    double dot_acc = 0.0;
    for (int32_t i = blockIdx.x * GPB + g; i < n; i += gridDim.x * GPB) {
        const int32_t cs = crp[i], ce = crp[i + 1];
        // fixed rows, and one-entry rows whose constraint space is exactly {0}
        if (PROJ && (rowtype[i] != 0 || ce - cs == 1)) {
            for (int32_t q = cs + lane; q < ce; q += G) cval[q] = 0.0;
            continue;
        }
        const int32_t as = arp[i], ae = arp[i + 1];
        double s1 = 0.0, s2 = 0.0;
        for (int32_t c0 = cs; c0 < ce; c0 += CAP) {
            const int len = (ce - c0) < CAP ? (ce - c0) : CAP;
            for (int q = lane; q < len; q += G) {
                s_col[g][q] = ccol[c0 + q];
                s_acc[g][q] = 0.0;
            }
            __syncwarp(mask);
            const int32_t lo = s_col[g][0], hi = s_col[g][len - 1];
            for (int32_t e = as; e < ae; e++) {
                const int32_t k = acol[e];
                const double a = aval[e];
                const int32_t xe = xrp[k + 1];
                for (int32_t f = xrp[k] + lane; f < xe; f += G) {
                    const int32_t j = xcol[f];
                    if (j < lo || j > hi) continue;
                    int l = 0, h = len - 1;
                    while (l < h) {
                        const int mid = (l + h) >> 1;
                        if (s_col[g][mid] < j) l = mid + 1; else h = mid;
                    }
                    if (s_col[g][l] == j) {
                        const double x = xval[f];
                        if (EXACT) s_acc[g][l] = __dadd_rn(s_acc[g][l], __dmul_rn(a, x));
                        else s_acc[g][l] = fma(a, x, s_acc[g][l]);
                    }
                }
                __syncwarp(mask);
            }
            for (int q = lane; q < len; q += G) {
                const double v = s_acc[g][q];
                if (PROJ) {
                    const double b = Bc[s_col[g][q]];
                    s1 = fma(v, b, s1);
                    s2 = fma(b, b, s2);
                }
                cval[c0 + q] = v;
            }
            __syncwarp(mask);
        }
        if (PROJ) {
            // chunks are multiples of G, so each lane re-reads the entries it wrote
            s1 = group_sum<G>(s1, mask);
            s2 = group_sum<G>(s2, mask);
            const double c = s1 / s2;
            for (int32_t q = cs + lane; q < ce; q += G) {
                const double w = scale * (cval[q] - c * Bc[ccol[q]]);
                cval[q] = w;
                if (Y) dot_acc = fma(Y[q], w, dot_acc);
            }
        }
    }
    if (PROJ) {
        const double v[1] = {dot_acc};
        grid_finish<kMpThreads, 1>(v, fin, s_red);
    }
}

template <bool EXACT, bool PROJ>
static void launch_mp(int G, int grid, cudaStream_t s, const char *name, double bytes, int32_t n, const int32_t *arp,
                      const int32_t *acol, const double *aval, const int32_t *xrp, const int32_t *xcol,
                      const double *xval, const int32_t *crp, const int32_t *ccol, double *cval,
                      const int32_t *rowtype, const double *Bc, double scale, const double *Y, const Fin &fin) {
#define RN_MP_CASE(GG)                                                                                         \
    case GG:                                                                                                   \
        RN_LAUNCH(name, bytes, s, (masked_product_kernel<GG, EXACT, PROJ>), grid, kMpThreads, 0, n, arp, acol, \
                  aval, xrp, xcol, xval, crp, ccol, cval, rowtype, Bc, scale, Y, fin);                         \
        break;
    switch (G) {
        RN_MP_CASE(4)
        RN_MP_CASE(8)
        RN_MP_CASE(16)
        RN_MP_CASE(32)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_MP_CASE
}

static int pick_group(double avg_len) {
    if (avg_len <= 4.5) return 4;
    if (avg_len <= 10.0) return 8;
    if (avg_len <= 20.0) return 16;
    return 32;
}

void spgemm_numeric(const CsrView &A, const CsrView &B, DCsr &C, bool exact, cudaStream_t s) {
    C.val.alloc(C.nnz, s);
    if (A.n == 0) return;
    const int G = pick_group(B.n ? (double)B.nnz / B.n : 1.0);
    const int grid = grid_for(A.n, kMpThreads / G, 8);
    // algorithmic bytes: A and the pattern of C once, B gathered once, C written once
    const double bytes = 12.0 * A.nnz + 4.0 * A.n + 12.0 * B.nnz + 12.0 * C.nnz;
    const Fin none;
    if (exact)
        launch_mp<true, false>(G, grid, s, "spgemm_numeric_exact", bytes, A.n, A.rowptr, A.col, A.val, B.rowptr,
                               B.col, B.val, C.rowptr.p, C.col.p, C.val.p, nullptr, nullptr, 1.0, nullptr, none);
    else
        launch_mp<false, false>(G, grid, s, "spgemm_numeric", bytes, A.n, A.rowptr, A.col, A.val, B.rowptr, B.col,
                                B.val, C.rowptr.p, C.col.p, C.val.p, nullptr, nullptr, 1.0, nullptr, none);
}

void masked_product_proj(const CsrView &A, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN, int32_t nc,
                         const double *X, double *W, const ProjArgs &pa, double scale, const double *Y,
                         const Fin &fin, cudaStream_t s) {
    if (A.n == 0) return;
    const int G = pick_group((double)nnzN / A.n);
    int grid = grid_for(A.n, kMpThreads / G, 8);
    if (grid > kReduceBlocks) grid = kReduceBlocks;
    // algorithmic bytes of one energy-minimisation product: A once, the
    // pattern (row pointers + columns) once, X once, W written once, Y once
    // when the Frobenius product is taken, row types and Bc once.
    const double bytes = 12.0 * A.nnz + 4.0 * (A.n + 1) + 4.0 * A.n + 4.0 * nnzN + 8.0 * nnzN + 8.0 * nnzN +
                         (Y ? 8.0 * nnzN : 0.0) + 8.0 * nc;
    launch_mp<false, true>(G, grid, s, "energy_masked_product", bytes, A.n, A.rowptr, A.col, A.val, nrowptr, ncol, X,
                           nrowptr, ncol, W, pa.rowtype, pa.Bc, scale, Y, fin);
}

}  // namespace rn
