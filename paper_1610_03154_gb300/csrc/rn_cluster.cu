// rn_cluster.cu - the bottom of the V-cycle (Sec. 2: the two-grid correction
// applied recursively) on the smallest coarse levels, run by one thread-block
// cluster.
//
// On a level of a few thousand rows a smoothing sweep, a restriction or a
// prolongation moves a few hundred kilobytes: as separate launches each costs
// its launch, ramp and drain, several microseconds, for well under one of
// memory traffic.  Here every operation of the cycle from level k+1 down to
// the coarsest and back up is one phase of a single cluster launch, phases
// separated by the cluster barrier (hardware, release/acquire at cluster
// scope, split into arrive and wait).  The host writes the phase list once (the buffers each phase reads
// and writes are fixed by nu_pre / nu_post); the kernel stages it in shared
// memory and walks it.  Between arriving at a barrier and waiting on it every
// thread loads the row bounds and its first matrix entries of the next phase,
// which do not depend on the phase being finished, so after the barrier only
// the gathers of x remain.
//
// Rows are summed lane-strided in storage order, like the per-level launches;
// only the number of lanes per row may differ.  Vectors written inside the
// kernel are read with ld.global.cg (L2), never through L1, so no CTA reads a
// stale line of data another CTA wrote in an earlier phase; the matrices and
// relaxation weights are read-only for the kernel's life.
#include <cooperative_groups.h>

#include "rn_hier.cuh"

namespace cg = cooperative_groups;

namespace rn {

constexpr int kClusterThreads = 1024;
constexpr int kPrefetch = 4;  // matrix entries per lane loaded ahead of the barrier

template <typename T>
__device__ __forceinline__ T gather(int op, int32_t j, const T *x, const T *b, const T *d) {
    return op == SUB_JZ_RESID ? __ldg(d + j) * __ldcg(b + j) : __ldcg(x + j);
}

template <typename T>
__global__ void __launch_bounds__(kClusterThreads, 1)
subcycle_cluster_kernel(const SubPhase<T> *__restrict__ phases, int nph, const double *__restrict__ Ainv) {
    __shared__ SubPhase<T> ph[kSubMaxPhases];
    cg::cluster_group cl = cg::this_cluster();
    const int nthr = (int)cl.num_blocks() * blockDim.x;
    const int gt = (int)cl.block_rank() * blockDim.x + threadIdx.x;
    {
        const int words = nph * (int)(sizeof(SubPhase<T>) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(phases);
        int *dst = reinterpret_cast<int *>(ph);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    // prefetched first pass of the current phase: row bounds, first entries
    int32_t s = 0, e = 0, cj[kPrefetch];
    T av[kPrefetch];
    auto prefetch = [&](const SubPhase<T> &P) {
        s = e = 0;
        if (P.op > SUB_JZ_RESID) return;
        const int G = P.M.g;
        const int32_t i = gt / G;
        if (i < P.M.n) {
            s = __ldg(P.M.rp + i);
            e = __ldg(P.M.rp + i + 1);
        }
        const int lane = gt % G;
#pragma unroll
        for (int u = 0; u < kPrefetch; u++) {
            const int32_t q = s + lane + u * G;
            cj[u] = q < e ? __ldg(P.M.col + q) : 0;
            av[u] = q < e ? __ldg(P.M.val + q) : T(0);
        }
    };
    prefetch(ph[0]);  // matrix data only: may run while the predecessor finishes
    pdl_wait();
    pdl_trigger();
    for (int p = 0; p < nph; p++) {
        const SubPhase<T> &P = ph[p];
        const int op = P.op;
        if (op == SUB_COARSE) {  // x = A_L^{-1} b in FP64 arithmetic, warp per row
            const int32_t nc = P.M.n;
            const int lane = gt & 31;
            for (int32_t i = gt >> 5; i < nc; i += nthr >> 5) {
                double acc = 0.0;
                for (int32_t j = lane; j < nc; j += 32)
                    acc = fma(__ldg(Ainv + (int64_t)i * nc + j), (double)__ldcg(P.b + j), acc);
                acc = warp_sum(acc);
                if (lane == 0) P.y[i] = (T)acc;
            }
        } else if (op == SUB_SCALE) {  // y = d b (or 0 without d): first sweep from a zero guess
            for (int32_t i = gt; i < P.M.n; i += nthr) P.y[i] = P.d ? __ldg(P.d + i) * __ldcg(P.b + i) : T(0);
        } else {
            const int G = P.M.g;
            const int grp = gt / G, lane = gt % G;
            const int rpp = nthr / G;
            for (int32_t base = 0; base < P.M.n; base += rpp) {
                const int32_t i = base + grp;
                T acc = T(0);
                if (base == 0) {  // bounds and the first entries were prefetched
#pragma unroll
                    for (int u = 0; u < kPrefetch; u++)
                        if (s + lane + u * G < e) acc = fma(av[u], gather<T>(op, cj[u], P.x, P.b, P.d), acc);
                    for (int32_t q = s + lane + kPrefetch * G; q < e; q += G)
                        acc = fma(__ldg(P.M.val + q), gather<T>(op, __ldg(P.M.col + q), P.x, P.b, P.d), acc);
                } else if (i < P.M.n) {
                    const int32_t s2 = __ldg(P.M.rp + i), e2 = __ldg(P.M.rp + i + 1);
                    for (int32_t q = s2 + lane; q < e2; q += G)
                        acc = fma(__ldg(P.M.val + q), gather<T>(op, __ldg(P.M.col + q), P.x, P.b, P.d), acc);
                }
                for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
                if (lane == 0 && i < P.M.n) {
                    if (op == SUB_SPMV) {
                        P.y[i] = acc;
                    } else if (op == SUB_SPMV_ADD) {
                        P.y[i] = __ldcg(P.y + i) + acc;
                    } else if (op == SUB_RESID) {
                        P.y[i] = __ldcg(P.b + i) - acc;
                    } else if (op == SUB_JACOBI) {
                        P.y[i] = __ldcg(P.x + i) + __ldg(P.d + i) * (__ldcg(P.b + i) - acc);
                    } else {  // SUB_JZ_RESID: xz = (omega / a_ii) b, y = b - A xz
                        const T bi = __ldcg(P.b + i);
                        P.xz[i] = __ldg(P.d + i) * bi;
                        P.y[i] = bi - acc;
                    }
                }
            }
        }
        if (p + 1 < nph) {
            // split barrier: this phase's stores are released on arrival; the next
            // phase's matrix loads then fly while the other CTAs arrive
            asm volatile("barrier.cluster.arrive.release;" ::: "memory");
            prefetch(ph[p + 1]);
            asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
        }
    }
}

// ------------------------------------------------------------------ host side
static int lanes_for(const DCsr &M) {
    const double avg = M.n ? (double)M.nnz / M.n : 1.0;
    int G = 1;
    while (G < 32 && avg > 2.0 * G) G *= 2;
    return G;
}

template <typename T>
static SubMat<T> sub_mat(const DCsr &M) {
    SubMat<T> s{};
    s.n = M.n;
    s.g = lanes_for(M);
    s.rp = M.rowptr.p;
    s.col = M.col.p;
    if constexpr (sizeof(T) == 4) s.val = M.val32.p;
    else s.val = M.val.p;
    return s;
}

template <typename T>
struct SubVecs {
    const T *d;
    T *b, *x, *t, *r;
};
template <typename T>
static SubVecs<T> sub_vecs(rn_level &L) {
    if constexpr (sizeof(T) == 4) return {L.wd32.p, L.b32.p, L.x32.p, L.t32.p, L.r32.p};
    else return {L.wd.p, L.b.p, L.x.p, L.t.p, L.r.p};
}

template <typename T>
static int cluster_size_for() {
    static int cached = -1;
    if (cached >= 0) return cached;
    RN_CUDA_CHECK(cudaFuncSetAttribute(subcycle_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClusterThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int cs = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&cs, subcycle_cluster_kernel<T>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        cs = 0;
    }
    cs = std::min(cs, 16);
    while (cs > 1) {  // largest power of two that can be resident
        int p = 1;
        while (2 * p <= cs) p *= 2;
        cs = p;
        cfg.gridDim = dim3(cs);
        attr[0].val.clusterDim.x = cs;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, subcycle_cluster_kernel<T>, &cfg) == cudaSuccess &&
            nclusters > 0)
            break;
        cudaGetLastError();
        cs /= 2;
    }
    cached = cs >= 2 ? cs : 0;
    return cached;
}

// passes of the cluster's threads over the rows of M
static int64_t passes(const DCsr &M, int nthr) {
    const int64_t rpp = nthr / lanes_for(M);
    return (M.n + rpp - 1) / rpp;
}

// The buffer that holds level l's iterate after its pre-smoothing: x, or t
// after an odd number of swapping sweeps (sweeps after the first swap).
template <typename T>
T *pre_smoothed(rn_level &L, int nu_pre) {
    const SubVecs<T> v = sub_vecs<T>(L);
    return (nu_pre >= 2 && ((nu_pre - 1) & 1)) ? v.t : v.x;
}
template float *pre_smoothed<float>(rn_level &, int);
template double *pre_smoothed<double>(rn_level &, int);

// Choose the cluster's levels and write its phase list.  Level l joins when
// every phase on it (and the restriction into it, the prolongation out of
// it) takes at most max_passes passes of the cluster's threads.
template <typename T>
static void prepare_sub_t(rn_hierarchy &h) {
    const int L = (int)h.lev.size();
    const int maxp = h.p.coarse_cluster;
    h.sub_k = -1;
    if (maxp <= 0 || L < 3 || h.lev[L - 1]->A.n > kSubMaxCoarse || h.p.gamma != 1) return;  // V-cycles only
    const int cs = cluster_size_for<T>();
    if (cs == 0) return;
    const int nthr = cs * kClusterThreads;
    auto level_ok = [&](int l) {  // A_l, and R_l / P_l unless coarsest
        rn_level &V = *h.lev[l];
        if (passes(V.A, nthr) > maxp) return false;
        if (l < L - 1 && (passes(V.P, nthr) > maxp || passes(V.R, nthr) > maxp)) return false;
        return true;
    };
    int first = L;
    for (int l = L - 1; l >= 1; l--) {
        if (!level_ok(l)) break;
        rn_level &U = *h.lev[l - 1];  // transfers between l-1 and l run in the cluster too
        if (passes(U.P, nthr) > maxp || passes(U.R, nthr) > maxp) break;
        first = l;
    }
    if (first > L - 2) return;  // nothing but the coarsest solve
    const int k = first - 1;
    std::vector<SubPhase<T>> ph;
    auto add = [&](int op, const SubMat<T> &M, const T *x, const T *b, const T *d, T *y, T *xz) {
        SubPhase<T> q{};
        q.op = op;
        q.M = M;
        q.x = x;
        q.b = b;
        q.d = d;
        q.y = y;
        q.xz = xz;
        ph.push_back(q);
    };
    std::vector<T *> cur(L), oth(L);
    {
        const SubVecs<T> vk = sub_vecs<T>(*h.lev[k]), v1 = sub_vecs<T>(*h.lev[k + 1]);
        add(SUB_SPMV, sub_mat<T>(h.lev[k]->R), vk.r, nullptr, nullptr, v1.b, nullptr);
    }
    for (int m = k + 1; m < L - 1; m++) {
        rn_level &V = *h.lev[m];
        const SubVecs<T> v = sub_vecs<T>(V), vc = sub_vecs<T>(*h.lev[m + 1]);
        const SubMat<T> A = sub_mat<T>(V.A);
        T *c = v.x, *o = v.t;
        if (h.p.nu_pre == 1) {
            add(SUB_JZ_RESID, A, nullptr, v.b, v.d, v.r, v.x);
        } else {
            SubMat<T> rows{};
            rows.n = V.A.n;
            add(SUB_SCALE, rows, nullptr, v.b, h.p.nu_pre == 0 ? nullptr : v.d, v.x, nullptr);
            for (int sw = 1; sw < h.p.nu_pre; sw++) {
                add(SUB_JACOBI, A, c, v.b, v.d, o, nullptr);
                std::swap(c, o);
            }
            add(SUB_RESID, A, c, v.b, nullptr, v.r, nullptr);
        }
        cur[m] = c;
        oth[m] = o;
        add(SUB_SPMV, sub_mat<T>(V.R), v.r, nullptr, nullptr, vc.b, nullptr);
    }
    const SubVecs<T> vl = sub_vecs<T>(*h.lev[L - 1]);
    SubMat<T> cm{};
    cm.n = h.lev[L - 1]->A.n;
    add(SUB_COARSE, cm, nullptr, vl.b, nullptr, vl.x, nullptr);
    T *xc = vl.x;
    for (int m = L - 2; m > k; m--) {
        rn_level &V = *h.lev[m];
        const SubVecs<T> v = sub_vecs<T>(V);
        add(SUB_SPMV_ADD, sub_mat<T>(V.P), xc, nullptr, nullptr, cur[m], nullptr);
        for (int sw = 0; sw < h.p.nu_post; sw++) {
            add(SUB_JACOBI, sub_mat<T>(V.A), cur[m], v.b, v.d, oth[m], nullptr);
            std::swap(cur[m], oth[m]);
        }
        xc = cur[m];
    }
    add(SUB_SPMV_ADD, sub_mat<T>(h.lev[k]->P), xc, nullptr, nullptr, pre_smoothed<T>(*h.lev[k], h.p.nu_pre),
        nullptr);
    if ((int)ph.size() > kSubMaxPhases) return;
    h.sub_k = k;
    h.sub_cs = cs;
    h.sub_nph = (int)ph.size();
    h.sub_desc.alloc(sizeof(SubPhase<T>) * ph.size(), h.s);
    h2d(h.sub_desc.p, reinterpret_cast<const unsigned char *>(ph.data()), sizeof(SubPhase<T>) * ph.size(), h.s);
    RN_CUDA_CHECK(cudaStreamSynchronize(h.s));  // ph is a host temporary
}

void prepare_subcycle(rn_hierarchy &h) {
    if (h.p.precision == RN_MIXED) prepare_sub_t<float>(h);
    else prepare_sub_t<double>(h);
}

template <typename T>
void launch_subcycle(rn_hierarchy &h, T *cur_k, const char *name) {
    if (cur_k != pre_smoothed<T>(*h.lev[h.sub_k], h.p.nu_pre))
        fail(RN_EINTERNAL, "cluster cycle: unexpected level iterate buffer");
    double bytes = 0.0;  // the matrices of every phase, once each
    const int L = (int)h.lev.size();
    for (int l = h.sub_k + 1; l < L; l++) {
        const rn_level &V = *h.lev[l];
        bytes += ((4.0 + sizeof(T)) * V.A.nnz + 4.0 * V.A.n) * (h.p.nu_pre + h.p.nu_post);
    }
    for (int l = h.sub_k; l < L - 1; l++) bytes += (4.0 + sizeof(T)) * (h.lev[l]->P.nnz + h.lev[l]->R.nnz);
    ProfScope ps(name, bytes, h.s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h.sub_cs);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.stream = h.s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = h.sub_cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = h.pdl ? 2 : 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, subcycle_cluster_kernel<T>,
                                             reinterpret_cast<const SubPhase<T> *>(h.sub_desc.p), h.sub_nph,
                                             (const double *)h.Ainv.p);
    if (e != cudaSuccess) fail(RN_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
}

template void launch_subcycle<float>(rn_hierarchy &, float *, const char *);
template void launch_subcycle<double>(rn_hierarchy &, double *, const char *);

}  // namespace rn
