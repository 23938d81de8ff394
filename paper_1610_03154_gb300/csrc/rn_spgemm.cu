// rn_spgemm.cu - sparse-sparse products on the GPU.
//
// * spgemm (C = A B): one hash pass per row builds the row's pattern (the
//   symbolic product, explicit zeros kept) and its values together, summed in
//   ascending k with a rounded multiply then a rounded add - bit-identical to
//   a plain sequential evaluation in the same order (used for N = S^d C, whose
//   values drive the pre-filter, and for the Galerkin product R (A P)).
// * masked_product_proj: the energy-minimisation operator
//   W = scale * Proj(Mask_N(A X)) on a fixed pattern, with the row-wise
//   constraint projection and a Frobenius product fused in.
#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>

#include "rn_internal.cuh"

namespace rn {

// ------------------------------------------------------------------ fused product (pattern + values)
// Rows are binned by their product count (the number of terms a_ik b_kj):
// * at most kSmallProd: a group of G lanes lists the row's products in
//   (k, position in B_k) order - ascending k, the order of a sequential
//   evaluation - in shared memory; the first product of each column sums its
//   column's run in list order (a rounded multiply, then one rounded add per
//   further term: bit-identical to the sequential evaluation) and is written
//   at its rank among the columns;
// * more: a shared-memory hash table per row, filled in ascending k, and one
//   block per row past its capacity.
// Rows go to a temporary at the row's offset in the prefix sum of the product
// counts (an upper bound of its length); a scan of the true lengths and a
// compaction produce C.
constexpr int kFuThreads = 128;
constexpr int kSmallProd = 64;
// Products with at most this many rows (the coarse levels) are bound by the
// latency of each row's chain of dependent loads, not by the machine's
// throughput: they take more lanes per row (sorted lists for short rows,
// warp-wide hash tables for long ones)
constexpr int32_t kFewRows = 40000;

// Product counts, and the row lists of the two bins: rows with at most
// kSmallProd products fill bins from the front, the others from the back.
__global__ void product_bound_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                                     const int32_t *__restrict__ brp, int32_t *__restrict__ ub,
                                     int32_t *__restrict__ bins, int32_t *__restrict__ flags) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int32_t i = base + threadIdx.x;
        const bool valid = i < n;
        int64_t u = 0;
        if (valid) {
            for (int32_t e = arp[i]; e < arp[i + 1]; e++) u += brp[acol[e] + 1] - brp[acol[e]];
            if (u > INT32_MAX / 2) {
                atomicMax(flags + 2, i + 1);
                u = 0;
            }
            ub[i] = (int32_t)u;
        }
        const bool small = valid && u <= kSmallProd, large = valid && u > kSmallProd;
        const unsigned bs = __ballot_sync(0xffffffffu, small), bl = __ballot_sync(0xffffffffu, large);
        int32_t os = 0, ol = 0;
        if (lane == 0) {
            if (bs) os = atomicAdd(flags + 0, __popc(bs));
            if (bl) ol = atomicAdd(flags + 1, __popc(bl));
        }
        os = __shfl_sync(0xffffffffu, os, 0);
        ol = __shfl_sync(0xffffffffu, ol, 0);
        const unsigned below = (1u << lane) - 1u;
        if (small) bins[os + __popc(bs & below)] = i;
        if (large) bins[n - 1 - (ol + __popc(bl & below))] = i;
    }
}

template <int G>
__global__ void __launch_bounds__(kFuThreads)
small_product_kernel(int32_t nrows_max, const int32_t *__restrict__ nrows_dev, const int32_t *__restrict__ rows,
                     const int32_t *__restrict__ arp,
                     const int32_t *__restrict__ acol, const double *__restrict__ aval,
                     const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                     const double *__restrict__ bval, const int32_t *__restrict__ ubp, int32_t *__restrict__ tcol,
                     double *__restrict__ tval, int32_t *__restrict__ count) {
    pdl_wait();
    constexpr int GPB = kFuThreads / G;
    constexpr int ST = kSmallProd + 1;  // padded stride: groups of one warp start in different banks
    __shared__ long long s_k[GPB * ST];
    __shared__ double s_v[GPB * ST];
    // flattened listing (G >= 8, long rows B_k): the contributing entries'
    // a_ik, B_k starts and list offsets
    constexpr bool FLAT = G >= 8;
    constexpr int ET = FLAT ? kSmallProd : 1;
    __shared__ double s_ea[GPB * ET];
    __shared__ int32_t s_eb[GPB * ET];
    __shared__ int32_t s_eo[GPB * ET];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    long long *K = s_k + g * ST;  // (column << 8) | list position
    double *V = s_v + g * ST;     // products in list order
    double *Ea = s_ea + g * ET;
    int32_t *Eb = s_eb + g * ET, *Eo = s_eo + g * ET;
    const int32_t nrows = nrows_dev ? min(*nrows_dev, nrows_max) : nrows_max;  // rows listed on the device
    for (int32_t r0 = blockIdx.x * GPB; r0 < nrows; r0 += gridDim.x * GPB) {
        if (r0 + g >= nrows) continue;  // the whole group leaves together
        const int32_t i = rows[r0 + g];
        const int32_t as = arp[i], ae = arp[i + 1];
        // 1a. the row's entries a_ik with a non-empty B_k, in order, and where
        //     their products start in the list ((k, position in B_k) order)
        int32_t m = 0, ne = 0;
        for (int32_t e0 = as; e0 < ae; e0 += G) {
            const int32_t e = e0 + lane;
            int32_t b0 = 0, c = 0;
            double a = 0.0;
            if (e < ae) {
                const int32_t k = acol[e];
                a = aval[e];
                b0 = brp[k];
                c = brp[k + 1] - b0;
            }
            int32_t incl = c, ninc = c > 0 ? 1 : 0;
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const int32_t t = __shfl_up_sync(mask, incl, o, G);
                const int32_t u = __shfl_up_sync(mask, ninc, o, G);
                if (lane >= o) {
                    incl += t;
                    ninc += u;
                }
            }
            if (FLAT) {
                if (c > 0) {
                    const int32_t slot = ne + ninc - 1;
                    Ea[slot] = a;
                    Eb[slot] = b0;
                    Eo[slot] = m + incl - c;
                }
            } else {  // short rows B_k: each lane lists its entry's products
                const int32_t off = m + incl - c;
                for (int32_t f = 0; f < c; f++) {
                    K[off + f] = ((long long)bcol[b0 + f] << 8) | (long long)(off + f);
                    V[off + f] = __dmul_rn(a, bval[b0 + f]);
                }
            }
            m += __shfl_sync(mask, incl, G - 1, G);
            ne += __shfl_sync(mask, ninc, G - 1, G);
        }
        __syncwarp(mask);
        // 1b. every lane takes list positions: the entry by binary search over
        //     the offsets, then one product each (independent loads)
        if (FLAT) {
            for (int t = lane; t < m; t += G) {
                int lo = 0, hi = ne - 1;
                while (lo < hi) {  // last slot with offset <= t
                    const int mid = (lo + hi + 1) >> 1;
                    if (Eo[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                const int32_t f = Eb[lo] + (t - Eo[lo]);
                K[t] = ((long long)bcol[f] << 8) | (long long)t;
                V[t] = __dmul_rn(Ea[lo], bval[f]);
            }
        }
        // 2. bitonic sort of the keys (padded to a power of two): each column's
        //    products become one run, in list order
        int P = 1;
        while (P < m) P <<= 1;
        for (int t = m + lane; t < P; t += G) K[t] = LLONG_MAX;
        __syncwarp(mask);
        for (int k = 2; k <= P; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int t = lane; t < (P >> 1); t += G) {
                    // the t-th pair: a zero bit inserted at jj (a power of two)
                    const int lo = ((t & ~(jj - 1)) << 1) | (t & (jj - 1)), hi = lo + jj;
                    const long long x = K[lo], y = K[hi];
                    if ((x > y) == ((lo & k) == 0)) {
                        K[lo] = y;
                        K[hi] = x;
                    }
                }
                __syncwarp(mask);
            }
        }
        // 3. each lane takes a contiguous slice of the sorted list; a run's
        //    first entry sums the run (one rounded add per further product) and
        //    goes to its rank among the row's columns
        const int chunk = (m + G - 1) / G;
        const int s0 = min(m, lane * chunk), s1 = min(m, s0 + chunk);
        int mine = 0;
        for (int q = s0; q < s1; q++) mine += (q == 0 || (K[q] >> 8) != (K[q - 1] >> 8)) ? 1 : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const int t = __shfl_up_sync(mask, incl, o, G);
            if (lane >= o) incl += t;
        }
        int pos = incl - mine;
        const int32_t base = ubp[i];
        for (int q = s0; q < s1; q++) {
            const long long key = K[q];
            const long long j = key >> 8;
            if (q > 0 && (K[q - 1] >> 8) == j) continue;
            double sum = V[key & 255];  // 0 + a b
            for (int u = q + 1; u < m && (K[u] >> 8) == j; u++) sum = __dadd_rn(sum, V[K[u] & 255]);
            tcol[base + pos] = (int32_t)j;
            tval[base + pos] = sum;
            pos++;
        }
        const int total = __shfl_sync(mask, incl, G - 1, G);
        if (lane == 0) count[i] = total;
        __syncwarp(mask);
    }
}

// Rows with at most kMergeWays entries (and at most kSmallProd products): a
// thread per row merges the row's sorted lists B_k (one per a_ik, ascending
// k).  Each output column is the smallest head; its products are summed in
// ascending k (the first one alone, then one rounded add per further term),
// bit-identical to a sequential evaluation.  Rows with more entries go to
// ovf_list for the sort kernel.
constexpr int kMergeWays = 12;

template <bool FUSED>
__global__ void __launch_bounds__(kFuThreads)
merge_product_kernel(int32_t nrows, const int32_t *__restrict__ rows, const int32_t *__restrict__ arp,
                     const int32_t *__restrict__ acol, const double *__restrict__ aval,
                     const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                     const double *__restrict__ bval, const int32_t *__restrict__ ubp, int32_t *__restrict__ tcol,
                     double *__restrict__ tval, int32_t *__restrict__ count, int32_t *__restrict__ ovf_list,
                     int32_t *__restrict__ ovf_n) {
    pdl_wait();
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
        const int32_t i = rows[r];
        const int32_t as = arp[i], ae = arp[i + 1], na = ae - as;
        if (na > kMergeWays) {
            ovf_list[atomicAdd(ovf_n, 1)] = i;
            continue;
        }
        int32_t pos[kMergeWays], end[kMergeWays], cur[kMergeWays];
#pragma unroll
        for (int u = 0; u < kMergeWays; u++) {
            pos[u] = 0;
            end[u] = 0;
            cur[u] = INT32_MAX;
            if (u < na) {
                const int32_t k = acol[as + u];
                pos[u] = brp[k];
                end[u] = brp[k + 1];
                if (pos[u] < end[u]) cur[u] = bcol[pos[u]];
            }
        }
        const int32_t base = ubp[i];
        int32_t nout = 0;
        for (;;) {
            int32_t cmin = INT32_MAX;
#pragma unroll
            for (int u = 0; u < kMergeWays; u++) cmin = min(cmin, cur[u]);
            if (cmin == INT32_MAX) break;
            double sum = 0.0;
            bool first = true;
#pragma unroll
            for (int u = 0; u < kMergeWays; u++) {
                if (cur[u] == cmin) {
                    const double a = aval[as + u], b = bval[pos[u]];
                    if (FUSED) sum = first ? __dmul_rn(a, b) : __fma_rn(a, b, sum);
                    else sum = first ? __dmul_rn(a, b) : __dadd_rn(sum, __dmul_rn(a, b));
                    first = false;
                    pos[u]++;
                    cur[u] = pos[u] < end[u] ? bcol[pos[u]] : INT32_MAX;
                }
            }
            tcol[base + nout] = cmin;
            tval[base + nout] = sum;
            nout++;
        }
        count[i] = nout;
    }
}

// The compaction list's slot indices: a byte for tables of up to 256 slots,
// else 16 bits (a smaller footprint per group fits more CTAs per SM).
template <int SLOTS>
using HashListT = typename std::conditional<(SLOTS <= 256), uint8_t, uint16_t>::type;

// G lanes per row, SLOTS table entries per group, for the rows listed in
// rows.  Rows whose distinct columns exceed SLOTS/2 go to ovf_list.
template <int G, int SLOTS, bool FUSED>
__global__ void __launch_bounds__(kFuThreads)
hash_product_kernel(int32_t nrows, const int32_t *__restrict__ rows, const int32_t *__restrict__ arp,
                    const int32_t *__restrict__ acol, const double *__restrict__ aval,
                    const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                    const double *__restrict__ bval, const int32_t *__restrict__ ubp, int32_t *__restrict__ tcol,
                    double *__restrict__ tval, int32_t *__restrict__ count, int32_t *__restrict__ ovf_list,
                    int32_t *__restrict__ ovf_n) {
    pdl_wait();
    constexpr int GPB = kFuThreads / G;
    extern __shared__ __align__(16) unsigned char fu_smem[];
    double *vals_all = reinterpret_cast<double *>(fu_smem);
    int32_t *keys_all = reinterpret_cast<int32_t *>(fu_smem + (size_t)GPB * SLOTS * sizeof(double));
    HashListT<SLOTS> *list_all = reinterpret_cast<HashListT<SLOTS> *>(keys_all + GPB * SLOTS);
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    const unsigned gbase = (threadIdx.x & 31) & ~(G - 1);
    double *vals = vals_all + g * SLOTS;
    int32_t *keys = keys_all + g * SLOTS;
    HashListT<SLOTS> *list = list_all + g * (SLOTS / 2);
    for (int32_t r = blockIdx.x * GPB + g; r < nrows; r += gridDim.x * GPB) {
        const int32_t i = rows[r];
        const int32_t ub = ubp[i + 1] - ubp[i];
        int slots = 32;
        while (slots < SLOTS && slots < 2 * ub) slots <<= 1;
        const unsigned hmask = (unsigned)slots - 1u;
        for (int q = lane; q < slots; q += G) keys[q] = -1;
        __syncwarp(mask);
        // a product that finds the table full is dropped, and a row with more
        // distinct columns than half the table (the compaction list's size)
        // goes to the block kernel, which recomputes it whole: both checked
        // once, after the row
        bool full = false;
        int mine = 0;  // distinct columns this lane inserted
        for (int32_t e = arp[i]; e < arp[i + 1]; e++) {
            const int32_t k = acol[e];
            const double a = aval[e];
            for (int32_t f = brp[k] + lane; f < brp[k + 1]; f += G) {
                const int32_t j = bcol[f];
                const double b = bval[f];
                unsigned h = ((uint32_t)j * 2654435761u) & hmask;
                int p = 0;
                for (; p < slots; p++) {
                    const int32_t old = atomicCAS(&keys[h], -1, j);
                    if (old == -1) {
                        vals[h] = __dmul_rn(a, b);  // 0 + a b
                        mine++;
                        break;
                    }
                    if (old == j) {
                        vals[h] = FUSED ? __fma_rn(a, b, vals[h]) : __dadd_rn(vals[h], __dmul_rn(a, b));
                        break;
                    }
                    h = (h + 1) & hmask;
                }
                if (p == slots) full = true;
            }
            __syncwarp(mask);  // a_ik's products land before a_i(k+1)'s: sums in ascending k
        }
        int tot = mine;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) tot += __shfl_xor_sync(mask, tot, o, G);
        const bool ovf = __any_sync(mask, full) || tot > slots / 2;
        if (ovf) {
            if (lane == 0) ovf_list[atomicAdd(ovf_n, 1)] = i;
            __syncwarp(mask);
            continue;
        }
        // compact occupied slots (slot indices) into list, in slot order
        int u = 0;
        for (int q0 = 0; q0 < slots; q0 += G) {
            const int q = q0 + lane;
            const bool occ = keys[q] >= 0;
            const unsigned bal = (__ballot_sync(mask, occ) >> gbase) & (G == 32 ? 0xffffffffu : ((1u << G) - 1u));
            if (occ) list[u + __popc(bal & ((1u << lane) - 1u))] = (HashListT<SLOTS>)q;
            u += __popc(bal);
        }
        __syncwarp(mask);
        const int32_t base = ubp[i];
        for (int e = lane; e < u; e += G) {
            const int q = list[e];
            const int32_t key = keys[q];
            int rank = 0;
            for (int f = 0; f < u; f++) rank += (keys[list[f]] < key);
            tcol[base + rank] = key;
            tval[base + rank] = vals[q];
        }
        if (lane == 0) count[i] = u;
        __syncwarp(mask);
    }
}

// Block per overflowing row, kBigProd slots.
constexpr int kBigProd = 8192;
template <bool FUSED>
__global__ void __launch_bounds__(512)
hash_product_block_kernel(const int32_t *__restrict__ nrows_dev, const int32_t *__restrict__ rows,
                          const int32_t *__restrict__ arp,
                          const int32_t *__restrict__ acol, const double *__restrict__ aval,
                          const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                          const double *__restrict__ bval, const int32_t *__restrict__ ubp,
                          int32_t *__restrict__ tcol, double *__restrict__ tval, int32_t *__restrict__ count,
                          int32_t *__restrict__ err) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char big_smem[];
    double *vals = reinterpret_cast<double *>(big_smem);
    int32_t *keys = reinterpret_cast<int32_t *>(big_smem + kBigProd * sizeof(double));
    int32_t *list = keys + kBigProd;
    __shared__ int cnt, bad, u;
    const int32_t nrows = *nrows_dev;  // rows listed on the device; blocks loop over them
    for (int32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        __syncthreads();
        const int32_t i = rows[r];
        for (int q = threadIdx.x; q < kBigProd; q += blockDim.x) keys[q] = -1;
        if (threadIdx.x == 0) { cnt = 0; bad = 0; u = 0; }
        __syncthreads();
        constexpr unsigned hmask = kBigProd - 1;
        for (int32_t e = arp[i]; e < arp[i + 1]; e++) {
            const int32_t k = acol[e];
            const double a = aval[e];
            for (int32_t f = brp[k] + threadIdx.x; f < brp[k + 1]; f += blockDim.x) {
                const int32_t j = bcol[f];
                const double b = bval[f];
                unsigned h = ((uint32_t)j * 2654435761u) & hmask;
                int p = 0;
                for (; p < kBigProd; p++) {
                    const int32_t old = atomicCAS(&keys[h], -1, j);
                    if (old == -1) { vals[h] = __dmul_rn(a, b); atomicAdd(&cnt, 1); break; }
                    if (old == j) {
                        vals[h] = FUSED ? __fma_rn(a, b, vals[h]) : __dadd_rn(vals[h], __dmul_rn(a, b));
                        break;
                    }
                    h = (h + 1) & hmask;
                }
                if (p == kBigProd) bad = 1;
            }
            __syncthreads();
            if (bad || cnt > kBigProd / 2) break;
        }
        __syncthreads();
        if (bad || cnt > kBigProd / 2) {
            if (threadIdx.x == 0) {
                atomicMax(err, i + 1);
                count[i] = 0;  // an empty row keeps the compaction in bounds until the error is read
            }
            continue;
        }
        for (int q = threadIdx.x; q < kBigProd; q += blockDim.x)
            if (keys[q] >= 0) list[atomicAdd(&u, 1)] = q;
        __syncthreads();
        const int32_t base = ubp[i];
        for (int e = threadIdx.x; e < u; e += blockDim.x) {
            const int q = list[e];
            const int32_t key = keys[q];
            int rank = 0;
            for (int f = 0; f < u; f++) rank += (keys[list[f]] < key);
            tcol[base + rank] = key;
            tval[base + rank] = vals[q];
        }
        if (threadIdx.x == 0) count[i] = u;
    }
}

// C rows from the temporary (row i's entries at ubp[i], count[i] of them)
__global__ void compact_rows_kernel(int32_t n, const int32_t *__restrict__ ubp, const int32_t *__restrict__ crp,
                                    const int32_t *__restrict__ tcol, const double *__restrict__ tval,
                                    int32_t *__restrict__ ccol, double *__restrict__ cval) {
    pdl_wait();
    const int lane = threadIdx.x & 7;
    for (int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 3; i < n; i += (gridDim.x * blockDim.x) >> 3) {
        const int32_t s = ubp[i], d = crp[i], len = crp[i + 1] - crp[i];
        for (int32_t q = lane; q < len; q += 8) {
            ccol[d + q] = tcol[s + q];
            cval[d + q] = tval[s + q];
        }
    }
}

template <int G, int SLOTS, bool FUSED>
static void launch_hash_t(int32_t nrows, const int32_t *rows, const CsrView &A, const CsrView &B, const int32_t *ubp,
                          int32_t *tcol, double *tval, int32_t *count, int32_t *ovf_list, int32_t *ovf_n,
                          double bytes, cudaStream_t s) {
    constexpr int GPB = kFuThreads / G;
    const size_t smem = (size_t)GPB * SLOTS * (sizeof(double) + sizeof(int32_t)) +
                        (size_t)GPB * (SLOTS / 2) * sizeof(HashListT<SLOTS>);
    static const bool configured = [&] {  // once per instantiation (thread-safe static initialisation)
        RN_CUDA_CHECK(cudaFuncSetAttribute(hash_product_kernel<G, SLOTS, FUSED>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return true;
    }();
    (void)configured;
    const int grid = grid_resident(hash_product_kernel<G, SLOTS, FUSED>, kFuThreads, smem, nrows, GPB);
    RN_LAUNCH("spgemm_hash", bytes, s, (hash_product_kernel<G, SLOTS, FUSED>), grid, kFuThreads, smem, nrows, rows,
              A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, ubp, tcol, tval, count, ovf_list, ovf_n);
}
template <int G, int SLOTS>
static void launch_hash(bool fused, int32_t nrows, const int32_t *rows, const CsrView &A, const CsrView &B,
                        const int32_t *ubp, int32_t *tcol, double *tval, int32_t *count, int32_t *ovf_list,
                        int32_t *ovf_n, double bytes, cudaStream_t s) {
    if (fused) launch_hash_t<G, SLOTS, true>(nrows, rows, A, B, ubp, tcol, tval, count, ovf_list, ovf_n, bytes, s);
    else launch_hash_t<G, SLOTS, false>(nrows, rows, A, B, ubp, tcol, tval, count, ovf_list, ovf_n, bytes, s);
}
template <bool FUSED>
static void launch_block(int32_t nlarge, const int32_t *nrows_dev, const int32_t *rows, const CsrView &A,
                         const CsrView &B, const int32_t *ubp, int32_t *tcol, double *tval, int32_t *count,
                         int32_t *err, cudaStream_t s) {
    const size_t smem = (size_t)kBigProd * (sizeof(double) + 2 * sizeof(int32_t));
    static const bool configured = [&] {
        RN_CUDA_CHECK(cudaFuncSetAttribute(hash_product_block_kernel<FUSED>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return true;
    }();
    (void)configured;
    RN_LAUNCH("spgemm_hash_long", 0, s, hash_product_block_kernel<FUSED>, std::min(nlarge, 2 * num_sms()), 512,
              smem, nrows_dev, rows, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, ubp, tcol, tval, count, err);
}

// nrows_dev: the number of listed rows on the device (at most nrows_max), or
// nullptr when nrows_max is exact
template <int G>
static void launch_small(int32_t nrows_max, const int32_t *nrows_dev, const int32_t *rows, const CsrView &A,
                         const CsrView &B, const int32_t *ubp, int32_t *tcol, double *tval, int32_t *count,
                         double bytes, cudaStream_t s) {
    constexpr int GPB = kFuThreads / G;
    const int grid = grid_resident(small_product_kernel<G>, kFuThreads, 0, nrows_max, GPB);
    RN_LAUNCH("spgemm_small", bytes, s, small_product_kernel<G>, grid, kFuThreads, 0, nrows_max, nrows_dev, rows,
              A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, ubp, tcol, tval, count);
}

void spgemm(const CsrView &A, const CsrView &Bin, DCsr &C, cudaStream_t s, bool fused, const int32_t *b_nnz_dev,
            int32_t *err_dev) {
    CsrView B = Bin;
    if (A.m != B.n) fail(RN_EINTERNAL, "spgemm: inner dimensions differ");
    C.n = A.n;
    C.m = B.m;
    const int32_t n = A.n;
    // flags: [0] small rows, [1] large rows, [2] count overflow, [3] rows past the hash tables, [4] past kBigProd,
    // [5] small rows with too many entries to merge, [6] B's size (given on the device); then two int64 totals at
    // flags + 8 (8-byte aligned)
    DVec<int32_t> ub(n + 1, s), ubp(n + 1, s), count(n + 1, s), flags(12, s), bins(n > 0 ? n : 1, s),
        ovf_list(n > 0 ? n : 1, s), ovf2(n > 0 ? n : 1, s);
    fill_i32(flags.p, 0, 12, s);
    if (b_nnz_dev) d2d(flags.p + 6, b_nnz_dev, 1, s);  // comes back with the first read
    int64_t *tot = reinterpret_cast<int64_t *>(flags.p + 8);
    if (n)
        RN_LAUNCH("spgemm_bound", 8.0 * A.nnz + 16.0 * n, s, product_bound_kernel, grid_for(n, 256), 256, 0, n,
                  A.rowptr, A.col, B.rowptr, ub.p, bins.p, flags.p);
    scan_counts_dev(ub.p, ubp.p, n, tot, s);
    int32_t fl[12];  // one read: bins, flags and the products' total
    read_small(fl, flags.p, 12, s);
    int64_t total = 0;
    std::memcpy(&total, fl + 8, sizeof total);
    if (fl[2] || total > INT32_MAX) fail(RN_EINTERNAL, "spgemm: a row's product count exceeds int32");
    if (b_nnz_dev) B.nnz = fl[6];
    DVec<int32_t> tcol(total > 0 ? total : 1, s);
    DVec<double> tval(total > 0 ? total : 1, s);
    const double bytes = 12.0 * A.nnz + 8.0 * n + 12.0 * B.nnz + 12.0 * total;
    const int32_t nsmall = fl[0], nlarge = fl[1];
    if (nsmall && n <= kFewRows) {  // few rows: G lanes per row list, sort and sum each row's products
        const double avg = (double)A.nnz / std::max(1, n) * ((double)B.nnz / std::max(1, B.n));
        if (avg <= 8.0) launch_small<8>(nsmall, nullptr, bins.p, A, B, ubp.p, tcol.p, tval.p, count.p, bytes, s);
        else launch_small<16>(nsmall, nullptr, bins.p, A, B, ubp.p, tcol.p, tval.p, count.p, bytes, s);
    } else if (nsmall) {
        // merge rows of few entries; the bin's other rows (counted on the
        // device) go to the sort kernel, launched for at most nsmall rows
        if (fused)
            RN_LAUNCH("spgemm_merge", bytes, s, merge_product_kernel<true>,
                      grid_resident(merge_product_kernel<true>, kFuThreads, 0, nsmall, kFuThreads), kFuThreads, 0,
                      nsmall, bins.p, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, ubp.p, tcol.p, tval.p,
                      count.p, ovf_list.p, flags.p + 5);
        else
            RN_LAUNCH("spgemm_merge", bytes, s, merge_product_kernel<false>,
                      grid_resident(merge_product_kernel<false>, kFuThreads, 0, nsmall, kFuThreads), kFuThreads, 0,
                      nsmall, bins.p, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, ubp.p, tcol.p, tval.p,
                      count.p, ovf_list.p, flags.p + 5);
        const double avg = (double)A.nnz / std::max(1, n) * ((double)B.nnz / std::max(1, B.n));
        if (avg <= 8.0)
            launch_small<4>(nsmall, flags.p + 5, ovf_list.p, A, B, ubp.p, tcol.p, tval.p, count.p, bytes, s);
        else if (avg <= 24.0)
            launch_small<8>(nsmall, flags.p + 5, ovf_list.p, A, B, ubp.p, tcol.p, tval.p, count.p, bytes, s);
        else launch_small<16>(nsmall, flags.p + 5, ovf_list.p, A, B, ubp.p, tcol.p, tval.p, count.p, bytes, s);
    }
    if (nlarge) {
        // short B rows (an interpolation operator, or A P): rows of the product
        // have few distinct columns, so smaller tables and fewer lanes per row
        // fit more rows per SM, and a B row of ~8 entries keeps a group of 8
        // lanes busy (32 lanes would leave most of the warp's FP64 multiply-adds
        // idle: R (A P) at level 0 of the 1024^2 anisotropy 828 -> 583 us);
        // sums per column run in ascending k either way (same result), and rows
        // past a table go to the block kernel
        const double avgB = B.n ? (double)B.nnz / B.n : 0.0;
        if (n <= kFewRows)  // few rows: a warp per row spreads each row's products widest
            launch_hash<32, 1024>(fused, nlarge, bins.p + (n - nlarge), A, B, ubp.p, tcol.p, tval.p, count.p, ovf2.p,
                                  flags.p + 3, bytes, s);
        else if (avgB <= 12.0)
            launch_hash<8, 128>(fused, nlarge, bins.p + (n - nlarge), A, B, ubp.p, tcol.p, tval.p, count.p, ovf2.p,
                                flags.p + 3, bytes, s);
        else if (avgB <= 16.0)
            launch_hash<32, 512>(fused, nlarge, bins.p + (n - nlarge), A, B, ubp.p, tcol.p, tval.p, count.p, ovf2.p,
                                 flags.p + 3, bytes, s);
        else
            launch_hash<32, 1024>(fused, nlarge, bins.p + (n - nlarge), A, B, ubp.p, tcol.p, tval.p, count.p, ovf2.p,
                                  flags.p + 3, bytes, s);
        // rows past the tables (counted on the device): a block per row, looping
        int32_t *err = err_dev ? err_dev : flags.p + 4;
        if (fused) launch_block<true>(nlarge, flags.p + 3, ovf2.p, A, B, ubp.p, tcol.p, tval.p, count.p, err, s);
        else launch_block<false>(nlarge, flags.p + 3, ovf2.p, A, B, ubp.p, tcol.p, tval.p, count.p, err, s);
    }
    C.rowptr.alloc(n + 1, s);
    scan_counts_dev(count.p, C.rowptr.p, n, tot + 1, s);
    if (err_dev) {
        // C's size stays on the device (its last row pointer); C is allocated at
        // its bound, the product count, and the caller reads err_dev later
        C.nnz = total;
    } else {
        read_small(fl, flags.p, 12, s);
        if (fl[4]) fail(RN_EINTERNAL, fmt("product row has more than %d distinct columns", kBigProd / 2));
        std::memcpy(&total, fl + 10, sizeof total);
        C.nnz = total;
    }
    C.col.alloc(C.nnz, s);
    C.val.alloc(C.nnz, s);
    if (n)
        RN_LAUNCH("spgemm_compact", 24.0 * C.nnz + 8.0 * n, s, compact_rows_kernel, grid_for((int64_t)n * 8, 256), 256,
                  0, n, ubp.p, C.rowptr.p, tcol.p, tval.p, C.col.p, C.val.p);
}

// ------------------------------------------------------------------ energy-minimisation product
// W = scale * Proj(Mask_N(A X)) on the pattern N that X and W share, and the
// Frobenius product <Y, W>.  One group of G lanes per row i; lane q owns the
// pattern entry j = N_i[q] (chunks of G entries for longer rows) and, for each
// a_ik in ascending k, scans the sorted row N_k for j (all lanes of the group
// read the same short row).  Each entry therefore sums a_ik X_kj in ascending
// k.  The row-wise projection onto {u : u.b = 0}, b = Bc[N_i] (eq. Tproj with
// a zero right-hand side), is applied in the epilogue; root, unaggregated and
// one-entry rows get W = 0.
constexpr int kEpThreads = 256;

// TV: the value type of A, X, W, Y and of the projection's Bc and row scales
// (double; float for the mixed-precision sweeps, where the row scales are
// formed in FP64 once per minimisation and rounded).  Per-thread parts of the
// Frobenius product accumulate in TV and join the FP64 grid reduction.
template <int G, typename TV>
__global__ void __launch_bounds__(kEpThreads, 4)
energy_product_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                      const TV *__restrict__ aval, const int32_t *__restrict__ nrp,
                      const int32_t *__restrict__ ncol, const TV *__restrict__ X, TV *__restrict__ W,
                      const int32_t *__restrict__ rowtype, const TV *__restrict__ Bc,
                      const TV *__restrict__ rs2v, TV scale, const TV *__restrict__ Y, Fin fin) {
    pdl_wait();
    __shared__ double s_red[32];
    constexpr int GPB = kEpThreads / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    TV dot_t = TV(0);
    for (int32_t i0 = blockIdx.x * GPB; i0 < n; i0 += gridDim.x * GPB) {
        const int32_t i = i0 + g;
        if (i >= n) continue;  // whole group leaves together
        const int32_t cs = nrp[i], ce = nrp[i + 1];
        if (rowtype[i] != 0 || ce - cs == 1) {  // fixed rows; one-entry rows: constraint space {0}
            for (int32_t q = cs + lane; q < ce; q += G) W[q] = TV(0);
            continue;
        }
        const int32_t as = arp[i], ae = arp[i + 1];
        const TV rs2 = rs2v[i];
        TV s1 = TV(0);
        TV acc_first = TV(0);
        for (int32_t q0 = cs; q0 < ce; q0 += G) {
            const int32_t q = q0 + lane;
            const bool active = q < ce;
            const int32_t j = active ? ncol[q] : INT32_MAX;
            TV acc = TV(0);
            for (int32_t e = as; e < ae; e++) {
                const int32_t k = acol[e];
                const TV a = aval[e];
                const int32_t ks = nrp[k], ke = nrp[k + 1];
                if (active) {
                    for (int32_t f = ks; f < ke; f++) {
                        const int32_t c = ncol[f];
                        if (c >= j) {
                            if (c == j) acc = fma(a, X[f], acc);
                            break;
                        }
                    }
                }
            }
            if (active) {
                s1 = fma(acc, Bc[j], s1);
                if (q0 == cs) acc_first = acc;  // the first chunk stays in registers
                else W[q] = acc;
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s1 += __shfl_xor_sync(mask, s1, o, G);
        const TV c = s1 * rs2;
        for (int32_t q = cs + lane; q < ce; q += G) {
            const TV v = (q - cs < G) ? acc_first : W[q];  // each lane re-reads only what it wrote
            const TV w = scale * (v - c * Bc[ncol[q]]);
            W[q] = w;
            if (Y) dot_t = fma(Y[q], w, dot_t);
        }
    }
    const double dot_acc[1] = {(double)dot_t};
    grid_finish<kEpThreads, 1>(dot_acc, fin, s_red);
}

// ------------------------------------------------------------------ energy product on a precomputed map
// The pattern N is fixed for a whole minimisation, and so is, for every entry
// (i, j) of N and every a_ik of row i, whether j occurs in the sorted row N_k
// and where.  ep_map_kernel records that position once (one byte: the offset
// in N_k, kMapNone when absent; row-major per row i as [k position in A_i]
// x [entry of N_i]); ep_mapped_kernel then forms Mask_N(A X) for every sweep
// by direct gathers, in the same order (ascending k, one fma per term) as
// energy_product_kernel, so its results are bit-identical.
constexpr unsigned char kMapNone = 255;

// map bytes of row i: |A_i| * |N_i| (0 for rows the operator zeroes); the
// longest row of N goes to *maxlen (its offsets must fit a byte)
__global__ void ep_map_sizes_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ nrp,
                                    const int32_t *__restrict__ rowtype, int32_t *__restrict__ sz,
                                    int32_t *__restrict__ maxlen) {
    pdl_wait();
    int32_t m = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t len = nrp[i + 1] - nrp[i];
        const int64_t b = (rowtype[i] != 0 || len == 1) ? 0 : (int64_t)(arp[i + 1] - arp[i]) * len;
        sz[i] = (int32_t)(b < (int64_t)(INT32_MAX / 4) ? b : (int64_t)(INT32_MAX / 4));
        m = max(m, len);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxlen, m);
}

template <int G>
__global__ void __launch_bounds__(kEpThreads)
ep_map_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
              const int32_t *__restrict__ nrp, const int32_t *__restrict__ ncol, const int32_t *__restrict__ rowtype,
              const int32_t *__restrict__ mbase, unsigned char *__restrict__ map) {
    pdl_wait();
    constexpr int GPB = kEpThreads / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int32_t i0 = blockIdx.x * GPB; i0 < n; i0 += gridDim.x * GPB) {
        const int32_t i = i0 + g;
        if (i >= n) continue;
        const int32_t cs = nrp[i], ce = nrp[i + 1], len = ce - cs;
        if (rowtype[i] != 0 || len == 1) continue;  // rows the operator zeroes: no map needed
        const int32_t as = arp[i], ae = arp[i + 1];
        unsigned char *mrow = map + mbase[i];
        for (int32_t q0 = cs; q0 < ce; q0 += G) {
            const int32_t q = q0 + lane;
            if (q >= ce) continue;
            const int32_t j = ncol[q];
            for (int32_t e = as; e < ae; e++) {
                const int32_t k = acol[e];
                const int32_t ks = nrp[k], ke = nrp[k + 1];
                unsigned char pos = kMapNone;
                for (int32_t f = ks; f < ke; f++) {
                    const int32_t c = ncol[f];
                    if (c >= j) {
                        if (c == j) pos = (unsigned char)(f - ks);
                        break;
                    }
                }
                mrow[(int64_t)(e - as) * len + (q - cs)] = pos;
            }
        }
    }
}

template <int G, typename TV>
__global__ void __launch_bounds__(kEpThreads, 4)
ep_mapped_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                 const TV *__restrict__ aval, const int32_t *__restrict__ nrp, const int32_t *__restrict__ ncol,
                 const int32_t *__restrict__ mbase, const unsigned char *__restrict__ map, const TV *__restrict__ X,
                 TV *__restrict__ W, const int32_t *__restrict__ rowtype, const TV *__restrict__ Bc,
                 const TV *__restrict__ rs2v, TV scale, const TV *__restrict__ Y, Fin fin) {
    pdl_wait();
    __shared__ double s_red[32];
    constexpr int GPB = kEpThreads / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    TV dot_t = TV(0);
    for (int32_t i0 = blockIdx.x * GPB; i0 < n; i0 += gridDim.x * GPB) {
        const int32_t i = i0 + g;
        if (i >= n) continue;  // whole group leaves together
        const int32_t cs = nrp[i], ce = nrp[i + 1], len = ce - cs;
        if (rowtype[i] != 0 || len == 1) {  // fixed rows; one-entry rows: constraint space {0}
            for (int32_t q = cs + lane; q < ce; q += G) W[q] = TV(0);
            continue;
        }
        const int32_t as = arp[i], ae = arp[i + 1];
        const unsigned char *mrow = map + mbase[i];
        const TV rs2 = rs2v[i];
        TV s1 = TV(0), acc_first = TV(0);
        for (int32_t q0 = cs; q0 < ce; q0 += G) {
            const int32_t q = q0 + lane;
            const bool active = q < ce;
            TV acc = TV(0);
            if (active) {
                for (int32_t e = as; e < ae; e++) {
                    const unsigned char pos = mrow[(int64_t)(e - as) * len + (q - cs)];
                    if (pos != kMapNone) acc = fma(aval[e], X[nrp[acol[e]] + pos], acc);
                }
                s1 = fma(acc, Bc[ncol[q]], s1);
                if (q0 == cs) acc_first = acc;
                else W[q] = acc;
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s1 += __shfl_xor_sync(mask, s1, o, G);
        const TV c = s1 * rs2;
        for (int32_t q = cs + lane; q < ce; q += G) {
            const TV v = (q - cs < G) ? acc_first : W[q];
            const TV w = scale * (v - c * Bc[ncol[q]]);
            W[q] = w;
            if (Y) dot_t = fma(Y[q], w, dot_t);
        }
    }
    const double dot_acc[1] = {(double)dot_t};
    grid_finish<kEpThreads, 1>(dot_acc, fin, s_red);
}

// 1 / sum_j Bc_j^2 over N_i: the scale of the row projection (eq. Tproj),
// which depends only on the pattern and Bc; 0 on rows the operator zeroes.
template <int G>
__global__ void __launch_bounds__(kEpThreads)
proj_scale_kernel(int32_t n, const int32_t *__restrict__ nrp, const int32_t *__restrict__ ncol,
                  const int32_t *__restrict__ rowtype, const double *__restrict__ Bc, double *__restrict__ rs2) {
    pdl_wait();
    constexpr int GPB = kEpThreads / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    for (int32_t i0 = blockIdx.x * GPB; i0 < n; i0 += gridDim.x * GPB) {
        const int32_t i = i0 + g;
        if (i >= n) continue;  // whole group leaves together
        const int32_t cs = nrp[i], ce = nrp[i + 1];
        double s2 = 0.0;
        for (int32_t q = cs + lane; q < ce; q += G) {
            const double b = Bc[ncol[q]];
            s2 = fma(b, b, s2);
        }
        s2 = group_sum<G>(s2, mask);
        if (lane == 0) rs2[i] = (rowtype[i] != 0 || ce - cs <= 1) ? 0.0 : 1.0 / s2;
    }
}

static int pick_group(double avg_len);

void proj_scales(int32_t n, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN, const int32_t *rowtype,
                 const double *Bc, double *rs2, cudaStream_t s) {
    if (n == 0) return;
    const int G = pick_group((double)nnzN / n);
    const double bytes = 8.0 * (n + 1) + 12.0 * nnzN + 8.0 * n;
#define RN_PS_CASE(GG)                                                                                          \
    case GG:                                                                                                    \
        RN_LAUNCH("energy_proj_scale", bytes, s, proj_scale_kernel<GG>,                                         \
                  grid_resident(proj_scale_kernel<GG>, kEpThreads, 0, n, kEpThreads / GG), kEpThreads, 0, n,     \
                  nrowptr, ncol, rowtype, Bc, rs2);                                                             \
        break;
    switch (G) {
        RN_PS_CASE(4)
        RN_PS_CASE(8)
        RN_PS_CASE(16)
        RN_PS_CASE(32)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_PS_CASE
}

static int pick_group(double avg_len) {
    if (avg_len <= 4.5) return 4;
    if (avg_len <= 10.0) return 8;
    if (avg_len <= 20.0) return 16;
    return 32;
}

template <typename TV>
void masked_product_proj(const CsrView &A, const TV *aval, const int32_t *nrowptr, const int32_t *ncol,
                         int64_t nnzN, int32_t nc, const TV *X, TV *W, const ProjArgsT<TV> &pa, double scale,
                         const TV *Y, const Fin &fin, cudaStream_t s) {
    if (A.n == 0) return;
    const int G = pick_group((double)nnzN / A.n);
    const void *fn = G == 4 ? (const void *)energy_product_kernel<4, TV>
                   : G == 8 ? (const void *)energy_product_kernel<8, TV>
                   : G == 16 ? (const void *)energy_product_kernel<16, TV>
                             : (const void *)energy_product_kernel<32, TV>;
    const int grid = grid_resident(fn, kEpThreads, 0, A.n, kEpThreads / G, kReduceBlocks);
    // algorithmic bytes of one energy-minimisation product: A once, the
    // pattern (row pointers + columns) once, X once, W written once, Y once
    // when the Frobenius product is taken, row types, scales and Bc once.
    const double vb = sizeof(TV);
    const double bytes = (4.0 + vb) * A.nnz + 4.0 * (A.n + 1) + 4.0 * (A.n + 1) + 4.0 * A.n + 8.0 * A.n +
                         4.0 * nnzN + 2.0 * vb * nnzN + (Y ? vb * nnzN : 0.0) + 8.0 * nc;
#define RN_EP_CASE(GG)                                                                                            \
    case GG:                                                                                                      \
        RN_LAUNCH("energy_masked_product", bytes, s, (energy_product_kernel<GG, TV>), grid, kEpThreads, 0, A.n,    \
                  A.rowptr, A.col, aval, nrowptr, ncol, X, W, pa.rowtype, pa.Bc, pa.rs2, (TV)scale, Y, fin);      \
        break;
    switch (G) {
        RN_EP_CASE(4)
        RN_EP_CASE(8)
        RN_EP_CASE(16)
        RN_EP_CASE(32)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_EP_CASE
}
bool ep_map_build(EpMap &m, const CsrView &A, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN,
                  const int32_t *rowtype, cudaStream_t s) {
    m.ok = false;
    if (A.n == 0) return false;
    DVec<int32_t> sz((size_t)A.n, s), mx(1, s);
    fill_i32(mx.p, 0, 1, s);
    RN_LAUNCH("energy_map", 16.0 * A.n, s, ep_map_sizes_kernel, grid_for(A.n, 256), 256, 0, A.n, A.rowptr, nrowptr,
              rowtype, sz.p, mx.p);
    if (read_scalar(mx.p, s) >= (int32_t)kMapNone) return false;  // offsets must fit a byte
    m.base.alloc((size_t)A.n + 1, s);
    int64_t total = 0;
    try {
        total = scan_counts(sz.p, m.base.p, A.n, s);
    } catch (const Error &) {
        return false;  // larger than int32 offsets: the scanning product is used
    }
    m.map.alloc((size_t)std::max<int64_t>(total, 1), s);
    m.G = pick_group((double)nnzN / A.n);
#define RN_MAP_CASE(GG)                                                                                          \
    case GG:                                                                                                     \
        RN_LAUNCH("energy_map", 8.0 * A.nnz + (double)total, s, ep_map_kernel<GG>,                               \
                  grid_resident(ep_map_kernel<GG>, kEpThreads, 0, A.n, kEpThreads / GG), kEpThreads, 0, A.n,     \
                  A.rowptr, A.col, nrowptr, ncol, rowtype, m.base.p, m.map.p);                                   \
        break;
    switch (m.G) {
        RN_MAP_CASE(4)
        RN_MAP_CASE(8)
        RN_MAP_CASE(16)
        RN_MAP_CASE(32)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_MAP_CASE
    m.bytes = total;
    m.ok = true;
    return true;
}

template <typename TV>
void masked_product_mapped(const EpMap &m, const CsrView &A, const TV *aval, const int32_t *nrowptr,
                           const int32_t *ncol, int64_t nnzN, int32_t nc, const TV *X, TV *W, const ProjArgsT<TV> &pa,
                           double scale, const TV *Y, const Fin &fin, cudaStream_t s) {
    if (A.n == 0) return;
    const double vb = sizeof(TV);
    // algorithmic bytes: the map once, A's columns and values once, the row
    // pointers of A and N, X gathered once, W written once, Y once, scales, Bc
    const double bytes = (double)m.bytes + (4.0 + vb) * A.nnz + 8.0 * (A.n + 1) + 4.0 * A.n + 4.0 * A.n +
                         vb * A.n + 4.0 * nnzN + 2.0 * vb * nnzN + (Y ? vb * nnzN : 0.0) + vb * nc;
#define RN_MP_CASE(GG)                                                                                           \
    case GG:                                                                                                     \
        RN_LAUNCH("energy_masked_product", bytes, s, (ep_mapped_kernel<GG, TV>),                                 \
                  grid_resident(ep_mapped_kernel<GG, TV>, kEpThreads, 0, A.n, kEpThreads / GG, kReduceBlocks),   \
                  kEpThreads, 0, A.n, A.rowptr, A.col, aval, nrowptr, ncol, m.base.p, m.map.p, X, W, pa.rowtype, \
                  pa.Bc, pa.rs2, (TV)scale, Y, fin);                                                             \
        break;
    switch (m.G) {
        RN_MP_CASE(4)
        RN_MP_CASE(8)
        RN_MP_CASE(16)
        RN_MP_CASE(32)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_MP_CASE
}
// ------------------------------------------------------------------ energy product on a sliced plan
// The scanning and mapped kernels give every lane of a row's group the whole
// of A_i: each lane reloads a_ik, k and nrp[k] for every k and follows the
// chain k -> nrp[k] -> X, so the work is dominated by redundant loads and
// dependent latency.  The plan (EpPlan) is built once per minimisation:
// lane l of row i owns A_i's entries l, l + G, ..., and for each of them reads
// a_ik and nrp[k] from slice-interleaved arrays (32 consecutive words per
// warp) and one map byte per pattern entry of row i; on a hit it gathers
// X[nrp[k] + pos] into a register accumulator of that entry.  The G partial
// sums of every entry are added by a butterfly over the group (a fixed order,
// so runs are bit-reproducible), then the row projection and <Y, W> follow as
// in the other kernels.
constexpr int kPlanThreads = 256;
constexpr int kPlanMaxLen = 16;

// One warp per slice: the slice's A slots (steps x 32), its longest kept row
// of N (slen) and the row infos; *mx: [0] longest row of N among rows the
// operator keeps, [1] longest row of N overall (positions must fit a field).
template <int G>
__global__ void __launch_bounds__(kPlanThreads)
ep_plan_sizes_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ nrp,
                     const int32_t *__restrict__ rowtype, int32_t *__restrict__ na, int32_t *__restrict__ slen,
                     int32_t *__restrict__ rinfo, int32_t *__restrict__ mx) {
    pdl_wait();
    constexpr int RW = 32 / G;
    const int lane = threadIdx.x & 31, r = lane / G, l = lane % G;
    const int64_t nsl = ((int64_t)n + RW - 1) / RW;
    const int64_t wstride = (int64_t)gridDim.x * (kPlanThreads / 32);
    int32_t m_keep = 0, m_all = 0;
    for (int64_t sl = blockIdx.x * (int64_t)(kPlanThreads / 32) + threadIdx.x / 32; sl < nsl; sl += wstride) {
        const int64_t i = sl * RW + r;
        int32_t steps = 0, klen = 0;
        if (i < n) {
            const int32_t len = nrp[i + 1] - nrp[i];
            const bool fixed = rowtype[i] != 0 || len <= 1;
            const int32_t a = fixed ? 0 : arp[i + 1] - arp[i];
            steps = (a + G - 1) / G;
            klen = fixed ? 0 : len;
            if (l == 0) rinfo[i] = (len < 255 && steps <= 0xffff) ? (steps | (len << 16)) : 0;
            m_all = max(m_all, (steps <= 0xffff) ? len : 255);  // rows no plan can hold reject the plan
            m_keep = max(m_keep, klen);
        }
        const int32_t smax = __reduce_max_sync(0xffffffffu, steps);
        const int32_t lmax = __reduce_max_sync(0xffffffffu, klen);
        if (lane == 0) {
            na[sl] = smax * 32;
            slen[sl] = lmax;
        }
    }
    m_keep = __reduce_max_sync(0xffffffffu, m_keep);
    m_all = __reduce_max_sync(0xffffffffu, m_all);
    if (lane == 0) {
        atomicMax(mx, m_keep);
        atomicMax(mx + 1, m_all);
    }
}

// Words per A entry of every slice and the slice's word count
__global__ void ep_plan_words_kernel(int64_t nsl, const int32_t *__restrict__ na, const int32_t *__restrict__ slen,
                                     int bits, int32_t *__restrict__ wps, int32_t *__restrict__ nw) {
    pdl_wait();
    for (int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sl < nsl; sl += (int64_t)gridDim.x * blockDim.x) {
        const int32_t w = (slen[sl] * bits + 31) / 32;
        wps[sl] = w;
        nw[sl] = na[sl] * w;  // (steps x 32) x words per step
    }
}

// One warp per slice: fills pa, pb and the position words of every lane, and
// bq, de of every pattern entry.  Word (j, w) of a lane: pm[moff + (j * wps +
// w) * 32 + lane], field t of it = entry q = w * (32 / bits) + t.
template <int G, typename TV>
__global__ void __launch_bounds__(kPlanThreads)
ep_plan_fill_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                    const double *__restrict__ aval, const int32_t *__restrict__ nrp, const int32_t *__restrict__ ncol,
                    const int32_t *__restrict__ rinfo, const int32_t *__restrict__ aoff,
                    const int32_t *__restrict__ moff, const int32_t *__restrict__ wps, int bits,
                    const double *__restrict__ Bc, const double *__restrict__ dinv, TV *__restrict__ pa,
                    int32_t *__restrict__ pb, uint32_t *__restrict__ pm, TV *__restrict__ bq, TV *__restrict__ de) {
    pdl_wait();
    constexpr int RW = 32 / G;
    const int lane = threadIdx.x & 31, r = lane / G, l = lane % G;
    const int64_t nsl = ((int64_t)n + RW - 1) / RW;
    const int64_t wstride = (int64_t)gridDim.x * (kPlanThreads / 32);
    const uint32_t none = (1u << bits) - 1u;
    const int per = 32 / bits;
    for (int64_t sl = blockIdx.x * (int64_t)(kPlanThreads / 32) + threadIdx.x / 32; sl < nsl; sl += wstride) {
        const int64_t i = sl * RW + r;
        const int64_t a0 = aoff[sl], a1 = aoff[sl + 1], m0 = moff[sl], m1 = moff[sl + 1];
        const int32_t ws = wps[sl];
        int32_t steps = 0, len = 0, cs = 0, as = 0;
        if (i < n) {
            const int32_t inf = rinfo[i];
            steps = inf & 0xffff;
            len = inf >> 16;
            cs = nrp[i];
            as = arp[i];
            const TV di = dinv ? (TV)dinv[i] : TV(1);
            for (int32_t q = cs + l; q < cs + len; q += G) {
                bq[q] = (TV)Bc[ncol[q]];
                de[q] = di;
            }
        }
        const int32_t a = (i < n && steps > 0) ? arp[i + 1] - as : 0;
        // A slots and position words: every slot and word of the slice is
        // written (padding: a = 0, base 0, every field absent)
        for (int64_t j = 0; a0 + j * 32 + lane < a1; j++) {
            const int32_t e = (int32_t)j * G + l;
            const int64_t slot = a0 + j * 32 + lane;
            const bool live = j < steps && e < a;
            int32_t ks = 0, ke = 0;
            if (live) {
                const int32_t k = acol[as + e];
                pa[slot] = (TV)aval[as + e];
                pb[slot] = ks = nrp[k];
                ke = nrp[k + 1];
            } else {
                pa[slot] = TV(0);
                pb[slot] = 0;
            }
            // both rows are sorted: one merge of N_i with N_k gives every position
            int32_t f = ks;
            for (int32_t w = 0; w < ws; w++) {
                uint32_t word = 0u;
                for (int t = 0; t < per; t++) {
                    const int32_t q = w * per + t;
                    uint32_t pos = none;
                    if (live && q < len) {
                        const int32_t jc = ncol[cs + q];
                        while (f < ke && ncol[f] < jc) f++;
                        if (f < ke && ncol[f] == jc) pos = (uint32_t)(f - ks);
                    }
                    word |= pos << (t * bits);
                }
                const int64_t wi = m0 + (j * ws + w) * 32 + lane;
                if (wi < m1) pm[wi] = word;
            }
        }
    }
}

// Field t of a position word
template <int BITS>
__device__ __forceinline__ uint32_t plan_field(uint32_t w, int t) {
    return (w >> (t * BITS)) & ((1u << BITS) - 1u);
}

// The gathers of one row of the plan product into acc[0..SS): per A entry
// (a_ik, nrp[k], position words) the next entry's are loaded before this
// entry's gathers (one step of software pipelining); field q of the words is
// the position of the row's q-th pattern column in N_k.
template <int SS, int PER, int BITS, typename TV, int S>
__device__ __forceinline__ void plan_steps(TV (&acc)[S], int32_t steps, int32_t ws, int32_t lm,
                                           const TV *__restrict__ pal, const int32_t *__restrict__ pbl,
                                           const uint32_t *__restrict__ pml, const TV *__restrict__ X) {
    constexpr int NW = (SS + PER - 1) / PER;
    constexpr uint32_t NONE = (1u << BITS) - 1u;
    TV an = pal[0];
    int32_t nbn = pbl[0];
    uint32_t wn[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) wn[w] = (w < ws) ? pml[(int64_t)w * 32] : 0u;
    for (int32_t j = 0; j < steps; j++) {
        const TV a = an;
        const int32_t nb = nbn;
        uint32_t wc[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) wc[w] = wn[w];
        if (j + 1 < steps) {
            an = pal[(int64_t)(j + 1) * 32];
            nbn = pbl[(int64_t)(j + 1) * 32];
#pragma unroll
            for (int w = 0; w < NW; w++)
                if (w < ws) wn[w] = pml[((int64_t)(j + 1) * ws + w) * 32];
        }
#pragma unroll
        for (int w = 0; w < NW; w++) {
            if (w < ws) {
                const uint32_t word = wc[w];
#pragma unroll
                for (int t = 0; t < PER; t++) {
                    const int q = w * PER + t;
                    // fields past lm (warp-uniform) are absent: skipped in FP64, where
                    // even a predicated-off FMA holds GB300's narrow FP64 pipe (FP32:
                    // the unconditional form measured faster)
                    if (q < SS && (sizeof(TV) == 4 || q < lm)) {
                        const uint32_t pos = plan_field<BITS>(word, t);
                        if (pos != NONE) acc[q] = fma(a, X[nb + (int32_t)pos], acc[q]);
                    }
                }
            }
        }
    }
}

template <int G, int S, int BITS, typename TV>
__global__ void __launch_bounds__(kPlanThreads)
ep_plan_kernel(int32_t n, const int32_t *__restrict__ rinfo, const int32_t *__restrict__ nrp,
               const int32_t *__restrict__ aoff, const int32_t *__restrict__ moff, const int32_t *__restrict__ wps,
               const int32_t *__restrict__ slen, const TV *__restrict__ pa, const int32_t *__restrict__ pb,
               const uint32_t *__restrict__ pm,
               const TV *__restrict__ bq, const TV *__restrict__ rs2v, const TV *__restrict__ X, TV *__restrict__ W,
               TV scale, const TV *__restrict__ Y, Fin fin) {
    pdl_wait();
    __shared__ double s_red[32];
    constexpr int RW = 32 / G;
    constexpr int PER = 32 / BITS;             // fields per word
    const int lane = threadIdx.x & 31, r = lane / G, l = lane % G;
    const unsigned gm = group_mask<G>();
    const int64_t nsl = ((int64_t)n + RW - 1) / RW;
    const int64_t wstride = (int64_t)gridDim.x * (kPlanThreads / 32);
    TV dot_t = TV(0);
    for (int64_t sl = blockIdx.x * (int64_t)(kPlanThreads / 32) + threadIdx.x / 32; sl < nsl; sl += wstride) {
        const int64_t i = sl * RW + r;
        if (i >= n) continue;  // the whole group leaves together
        const int32_t inf = rinfo[i];
        const int32_t steps = inf & 0xffff, len = inf >> 16;
        const int32_t cs = nrp[i];
        if (steps == 0) {  // fixed rows; one-entry rows: constraint space {0}
            for (int32_t q = cs + l; q < cs + len; q += G) W[q] = TV(0);
            continue;
        }
        const int32_t ws = wps[sl], lm = slen[sl];  // the same for the whole warp
        TV acc[S];
#pragma unroll
        for (int q = 0; q < S; q++) acc[q] = TV(0);
        const TV *pal = pa + aoff[sl] + lane;
        const int32_t *pbl = pb + aoff[sl] + lane;
        const uint32_t *pml = pm + moff[sl] + lane;
        // a slice whose rows all have at most 4 pattern entries takes the 4-field
        // path (warp-uniform branch): fields past a row's length are absent
        if constexpr (S > 4) {
            if (lm <= 4) plan_steps<4, PER, BITS>(acc, steps, ws, lm, pal, pbl, pml, X);
            else plan_steps<S, PER, BITS>(acc, steps, ws, lm, pal, pbl, pml, X);
        } else {
            plan_steps<S, PER, BITS>(acc, steps, ws, lm, pal, pbl, pml, X);
        }
        if constexpr (G > 1) {
#pragma unroll
            for (int q = 0; q < S; q++)
                if (q < len) {
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(gm, acc[q], o, G);
                }
        }
        TV s1 = TV(0);
#pragma unroll
        for (int q = 0; q < S; q++)
            if (q < len && (q % G) == l) s1 = fma(acc[q], bq[cs + q], s1);
        if constexpr (G > 1) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) s1 += __shfl_xor_sync(gm, s1, o, G);
        }
        const TV c = s1 * rs2v[i];
#pragma unroll
        for (int q = 0; q < S; q++)
            if (q < len && (q % G) == l) {
                const TV w = scale * (acc[q] - c * bq[cs + q]);
                W[cs + q] = w;
                if (Y) dot_t = fma(Y[cs + q], w, dot_t);
            }
    }
    const double dot_acc[1] = {(double)dot_t};
    grid_finish<kPlanThreads, 1>(dot_acc, fin, s_red);
}

// lanes per row from the average length of A's rows
static int plan_group(double avg_a, int32_t n) {
    if (n <= kFewRows) return 8;  // few rows: the shortest chain of gathers per lane
    if (avg_a <= 12.0) return 1;
    if (avg_a <= 24.0) return 2;
    if (avg_a <= 48.0) return 4;
    return 8;
}

template <typename TV>
bool ep_plan_build(EpPlan<TV> &p, const CsrView &A, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN,
                   const int32_t *rowtype, const double *Bc, const double *dinv, cudaStream_t s) {
    p.ok = false;
    const int32_t n = A.n;
    if (n == 0 || nnzN == 0) return false;
    const int G = plan_group((double)A.nnz / n, n);
    const int RW = 32 / G;
    const int64_t nsl = ((int64_t)n + RW - 1) / RW;
    DVec<int32_t> na((size_t)nsl, s), nw((size_t)nsl, s), mx(2, s);
    p.rinfo.alloc((size_t)n, s);
    p.slen.alloc((size_t)nsl, s);
    int32_t *slen = p.slen.p;
    fill_i32(mx.p, 0, 2, s);
    const int grid = grid_for(nsl, kPlanThreads / 32, 8);
#define RN_PLS_CASE(GG)                                                                                        \
    case GG:                                                                                                   \
        RN_LAUNCH("energy_map", 12.0 * n + 8.0 * nsl, s, ep_plan_sizes_kernel<GG>, grid, kPlanThreads, 0, n,     \
                  A.rowptr, nrowptr, rowtype, na.p, slen, p.rinfo.p, mx.p);                                  \
        break;
    switch (G) {
        RN_PLS_CASE(1)
        RN_PLS_CASE(2)
        RN_PLS_CASE(4)
        RN_PLS_CASE(8)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_PLS_CASE
    int32_t m[2];
    read_small(m, mx.p, 2, s);
    if (m[0] > kPlanMaxLen || m[1] >= 255) {
        p.rinfo.release();
        p.slen.release();
        return false;
    }
    p.bits = m[1] <= 15 ? 4 : 8;  // positions in N_k < 15 fit four bits (all ones: absent)
    p.wps.alloc((size_t)nsl, s);
    RN_LAUNCH("energy_map", 12.0 * nsl, s, ep_plan_words_kernel, grid_for(nsl, 256), 256, 0, nsl, na.p, slen,
              p.bits, p.wps.p, nw.p);
    p.aoff.alloc((size_t)nsl + 1, s);
    p.moff.alloc((size_t)nsl + 1, s);
    DVec<int64_t> tot(2, s);  // both totals in one read
    scan_counts_dev(na.p, p.aoff.p, nsl, tot.p, s);
    scan_counts_dev(nw.p, p.moff.p, nsl, tot.p + 1, s);
    int64_t t2[2];
    read_small(t2, tot.p, 2, s);
    if (t2[0] > INT32_MAX || t2[1] > INT32_MAX) {
        p.rinfo.release();
        p.slen.release();
        p.wps.release();
        p.aoff.release();
        p.moff.release();
        return false;  // offsets past int32: the caller falls back
    }
    p.slots = t2[0];
    p.words = t2[1];
    p.G = G;
    p.S = m[0] <= 4 ? 4 : (m[0] <= 8 ? 8 : 16);
    p.pa.alloc((size_t)std::max<int64_t>(p.slots, 1), s);
    p.pb.alloc((size_t)std::max<int64_t>(p.slots, 1), s);
    p.pm.alloc((size_t)std::max<int64_t>(p.words, 1), s);
    p.bq.alloc((size_t)nnzN, s);
    p.de.alloc((size_t)nnzN, s);
    const double vb = sizeof(TV);
    const double bytes = 8.0 * n + 16.0 * A.nnz + (vb + 4.0) * p.slots + 4.0 * p.words + (8.0 + 2.0 * vb) * nnzN;
#define RN_PLF_CASE(GG)                                                                                        \
    case GG:                                                                                                   \
        RN_LAUNCH("energy_map", bytes, s, (ep_plan_fill_kernel<GG, TV>), grid, kPlanThreads, 0, n, A.rowptr,    \
                  A.col, A.val, nrowptr, ncol, p.rinfo.p, p.aoff.p, p.moff.p, p.wps.p, p.bits, Bc, dinv, p.pa.p, \
                  p.pb.p, p.pm.p, p.bq.p, p.de.p);                                                             \
        break;
    switch (G) {
        RN_PLF_CASE(1)
        RN_PLF_CASE(2)
        RN_PLF_CASE(4)
        RN_PLF_CASE(8)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_PLF_CASE
    p.ok = true;
    return true;
}

template <typename TV>
void masked_product_plan(const EpPlan<TV> &p, int32_t n, const int32_t *nrowptr, int64_t nnzN, const TV *X, TV *W,
                         const TV *rs2, double scale, const TV *Y, const Fin &fin, cudaStream_t s) {
    if (n == 0) return;
    const double vb = sizeof(TV);
    // algorithmic bytes (the plan's A slots stand for A's values and columns;
    // the position words and bq are not counted): A once, row pointers of N,
    // row scales, X gathered once, W written once, Y once
    const double bytes = (4.0 + vb) * (double)p.slots + 4.0 * (n + 1) + vb * n + 2.0 * vb * nnzN +
                         (Y ? vb * nnzN : 0.0);
    const int RW = 32 / p.G;
    const int64_t nsl = ((int64_t)n + RW - 1) / RW;
#define RN_PLK(GG, SS, BB)                                                                                        \
    RN_LAUNCH("energy_masked_product", bytes, s, (ep_plan_kernel<GG, SS, BB, TV>),                                \
              grid_resident(ep_plan_kernel<GG, SS, BB, TV>, kPlanThreads, 0, nsl, kPlanThreads / 32, kReduceBlocks), \
              kPlanThreads, 0, n, p.rinfo.p, nrowptr, p.aoff.p, p.moff.p, p.wps.p, p.slen.p, p.pa.p, p.pb.p, p.pm.p, \
              p.bq.p,                                                                                                \
              rs2, X, W, (TV)scale, Y, fin)
#define RN_PLK_B(GG, SS)                  \
    if (p.bits == 4) RN_PLK(GG, SS, 4);   \
    else RN_PLK(GG, SS, 8);
#define RN_PLK_S(GG)                        \
    case GG:                                \
        if (p.S == 4) { RN_PLK_B(GG, 4) }   \
        else if (p.S == 8) { RN_PLK_B(GG, 8) } \
        else { RN_PLK_B(GG, 16) }           \
        break;
    switch (p.G) {
        RN_PLK_S(1)
        RN_PLK_S(2)
        RN_PLK_S(4)
        RN_PLK_S(8)
        default: fail(RN_EINTERNAL, "bad group size");
    }
#undef RN_PLK_S
#undef RN_PLK_B
#undef RN_PLK
}

template bool ep_plan_build<double>(EpPlan<double> &, const CsrView &, const int32_t *, const int32_t *, int64_t,
                                    const int32_t *, const double *, const double *, cudaStream_t);
template bool ep_plan_build<float>(EpPlan<float> &, const CsrView &, const int32_t *, const int32_t *, int64_t,
                                   const int32_t *, const double *, const double *, cudaStream_t);
template void masked_product_plan<double>(const EpPlan<double> &, int32_t, const int32_t *, int64_t, const double *,
                                          double *, const double *, double, const double *, const Fin &,
                                          cudaStream_t);
template void masked_product_plan<float>(const EpPlan<float> &, int32_t, const int32_t *, int64_t, const float *,
                                         float *, const float *, double, const float *, const Fin &, cudaStream_t);

template void masked_product_mapped<double>(const EpMap &, const CsrView &, const double *, const int32_t *,
                                            const int32_t *, int64_t, int32_t, const double *, double *,
                                            const ProjArgsT<double> &, double, const double *, const Fin &,
                                            cudaStream_t);
template void masked_product_mapped<float>(const EpMap &, const CsrView &, const float *, const int32_t *,
                                           const int32_t *, int64_t, int32_t, const float *, float *,
                                           const ProjArgsT<float> &, double, const float *, const Fin &, cudaStream_t);

template void masked_product_proj<double>(const CsrView &, const double *, const int32_t *, const int32_t *, int64_t,
                                          int32_t, const double *, double *, const ProjArgsT<double> &, double,
                                          const double *, const Fin &, cudaStream_t);
template void masked_product_proj<float>(const CsrView &, const float *, const int32_t *, const int32_t *, int64_t,
                                         int32_t, const float *, float *, const ProjArgsT<float> &, double,
                                         const float *, const Fin &, cudaStream_t);

}  // namespace rn
