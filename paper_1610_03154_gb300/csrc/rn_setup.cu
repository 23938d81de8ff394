// rn_setup.cu - root-node AMG setup (Alg. 3) on the GPU.
//
// Every step of the level loop runs in the kernels below; the host only
// sizes allocations (one device->host read per prefix sum) and steps the
// aggregation rounds.  Pattern decisions (strength, aggregation, S^d C and
// its pre-filter) use the same FP64 operation sequence as a plain sequential
// evaluation - rounded divide, square root, multiply and add with no fused
// multiply-add - so the integer outcomes (patterns, roots, aggregates) are
// reproducible bit for bit.
#include <algorithm>
#include <cmath>

#include "rn_hier.cuh"

namespace rn {

constexpr double kGuard = 1e-10;     // keep <=> v >= theta * ref * (1 - kGuard)
constexpr double kCgStop = 1e-22;    // CG energy minimisation stops at <R,Z> <= kCgStop <R0,Z0>
constexpr double kGmresBreak = 1e-14; // GMRES energy minimisation: h_{j+1,j} <= kGmresBreak * beta ends it
constexpr int kMaxAggRounds = 4096;  // bound on distance-2 MIS rounds
constexpr int kMaxDense = 4096;      // largest coarsest level for the dense LU
constexpr int kT = 256;              // threads per block of the row kernels

enum { FREE_ROW = 0, ROOT_ROW = 1, UNAGG_ROW = 2 };
enum { UNDECIDED = 0, TAKEN = 1, REMOVED = 2, ISOLATED = 3 };

// ------------------------------------------------------------------ input validation
__global__ void validate_kernel(int32_t n, int64_t nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const double *__restrict__ val, int32_t *__restrict__ bad) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t s = rp[i], e = rp[i + 1];
        bool ok = (s >= 0 && e >= s && e <= nnz) && (i != 0 || s == 0) && (i != n - 1 || e == nnz);
        bool diag = false;
        for (int32_t q = s; ok && q < e; q++) {
            int32_t j = col[q];
            if (j < 0 || j >= n || (q > s && j <= col[q - 1]) || !isfinite(val[q])) ok = false;
            if (j == i) diag = true;
        }
        if (!ok || !diag) atomicMax(bad, i + 1);
    }
}

// ------------------------------------------------------------------ strength (Sec. 3.2, eq. soc)
__device__ __forceinline__ double soc_value(double aij, double di, double dj) {
    return __ddiv_rn(fabs(aij), __dsqrt_rn(__dmul_rn(fabs(di), fabs(dj))));
}

// soc_value(aij, di, dj) >= thr, decided exactly as the FP64 expression
// decides it.  The test is |a|^2 >= thr^2 |di dj|; evaluated in FP32 its
// relative error is below 1e-6 when every operand lies in [2^-40, 2^40] (no
// FP32 underflow or overflow on the way), so a margin of 1e-5 either side
// settles it; only entries within that band of the threshold (or with
// operands out of range) take the FP64 square root and division.
__device__ __forceinline__ bool soc_strong(double aij, double di, double dj, double thr, float thr2f, bool fast) {
    const double aa = fabs(aij), ai = fabs(di), aj = fabs(dj);
    constexpr double lo = 0x1p-40, hi = 0x1p40;
    if (fast && aa >= lo && aa <= hi && ai >= lo && ai <= hi && aj >= lo && aj <= hi) {
        const float af = (float)aa;
        const float lhs = af * af;
        const float rhs = thr2f * ((float)ai * (float)aj);
        if (lhs > rhs * 1.00001f) return true;
        if (lhs < rhs * 0.99999f) return false;
    }
    return soc_value(aij, di, dj) >= thr;
}

// Pass 1 (FILL false): per row the count of S's entries (strong entries plus
// the diagonal), each strong entry's value v in vtmp (-1 for the others) and
// the row's largest strong value.  Pass 2: S's columns, and values v / vmax
// (1 on the diagonal).
// With classical (pass 1 only): v = -a_ij is strong when the row's largest
// such value m_i is positive and v >= thr m_i; vmaxv[i] = m_i, so pass 2
// writes -a_ij / m_i.
template <bool FILL>
__global__ void strength_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                                const double *__restrict__ aval, const double *__restrict__ diag, double thr,
                                int32_t *__restrict__ count, double *__restrict__ vtmp, double *__restrict__ vmaxv,
                                const int32_t *__restrict__ srp, int32_t *__restrict__ scol,
                                double *__restrict__ sval, int classical) {
    pdl_wait();
    const bool fast = thr >= 0x1p-10 && thr <= 0x1p10;  // thr^2 stays a normal FP32 number
    const float thr2f = (float)(thr * thr);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t e0 = arp[i], e1 = arp[i + 1];
        if (!FILL && classical) {
            double m = 0.0;
            for (int32_t e = e0; e < e1; e++)
                if (acol[e] != i && -aval[e] > m) m = -aval[e];
            const double cut = __dmul_rn(thr, m);
            int32_t c = 1;
            for (int32_t e = e0; e < e1; e++) {
                double v = -1.0;
                if (acol[e] != i && m > 0.0 && -aval[e] >= cut) {
                    v = -aval[e];
                    c++;
                }
                vtmp[e] = v;
            }
            count[i] = c;
            vmaxv[i] = m;
        } else if (!FILL) {
            const double di = diag[i];
            int32_t c = 1;
            double vmax = 0.0;
            for (int32_t e = e0; e < e1; e++) {
                const int32_t j = acol[e];
                double v = -1.0;
                if (j != i && soc_strong(aval[e], di, diag[j], thr, thr2f, fast)) {
                    v = soc_value(aval[e], di, diag[j]);
                    if (v > vmax) vmax = v;
                    c++;
                }
                vtmp[e] = v;
            }
            count[i] = c;
            vmaxv[i] = vmax;
        } else {
            const double vmax = vmaxv[i];
            int32_t dst = srp[i];
            for (int32_t e = e0; e < e1; e++) {
                const int32_t j = acol[e];
                if (j == i) {
                    scol[dst] = i;
                    sval[dst++] = 1.0;
                } else {
                    const double v = vtmp[e];
                    if (v >= 0.0) {
                        scol[dst] = j;
                        sval[dst++] = __ddiv_rn(v, vmax);
                    }
                }
            }
        }
    }
}

// aggregation graph: pattern(S) united with pattern(S)^T, diagonal removed
template <bool FILL>
__global__ void union_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                             const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                             int32_t *__restrict__ count, const int32_t *__restrict__ grp, int32_t *__restrict__ gcol) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t a = arp[i], ae = arp[i + 1], b = brp[i], be = brp[i + 1];
        int32_t c = 0, dst = FILL ? grp[i] : 0;
        while (a < ae || b < be) {
            int32_t ja = a < ae ? acol[a] : INT32_MAX;
            int32_t jb = b < be ? bcol[b] : INT32_MAX;
            int32_t j = ja < jb ? ja : jb;
            if (ja == j) a++;
            if (jb == j) b++;
            if (j != i) {
                if (FILL) gcol[dst++] = j;
                c++;
            }
        }
        if (!FILL) count[i] = c;
    }
}

// ------------------------------------------------------------------ seeded MIS-2 aggregation (Sec. 3.3)
// priority pi(i) = (splitmix64(seed ^ i), i), compared lexicographically; i
// is the node's index within its own problem: off is the first row of the
// problem both nodes belong to (0 for a single problem; independent problems
// set up together pass each row's problem offset, so every problem gets the
// aggregates it gets alone)
__device__ __forceinline__ bool prio_gt(int32_t a, int32_t b, uint64_t seed, int32_t off = 0) {
    a -= off;
    b -= off;
    uint64_t ha = splitmix64(seed ^ (uint64_t)(uint32_t)a), hb = splitmix64(seed ^ (uint64_t)(uint32_t)b);
    return ha > hb || (ha == hb && a > b);
}

__global__ void mis_init_kernel(int32_t n, const int32_t *__restrict__ grp, int32_t *__restrict__ state) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        state[i] = (grp[i + 1] > grp[i]) ? UNDECIDED : ISOLATED;
}

// m1[i] = best undecided node in the closed neighbourhood of i (or -1)
__global__ void mis_m1_kernel(int32_t n, const int32_t *__restrict__ grp, const int32_t *__restrict__ gcol,
                              const int32_t *__restrict__ state, uint64_t seed, const int32_t *__restrict__ roff,
                              int32_t *__restrict__ m1) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t off = roff ? roff[i] : 0;
        int32_t best = (state[i] == UNDECIDED) ? i : -1;
        for (int32_t e = grp[i]; e < grp[i + 1]; e++) {
            int32_t j = gcol[e];
            if (state[j] == UNDECIDED && (best < 0 || prio_gt(j, best, seed, off))) best = j;
        }
        m1[i] = best;
    }
}

// an undecided node is taken when it is the best undecided node within distance 2
__global__ void mis_take_kernel(int32_t n, const int32_t *__restrict__ grp, const int32_t *__restrict__ gcol,
                                const int32_t *__restrict__ m1, uint64_t seed, const int32_t *__restrict__ roff,
                                int32_t *__restrict__ state) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != UNDECIDED) continue;
        const int32_t off = roff ? roff[i] : 0;
        int32_t best = m1[i];
        for (int32_t e = grp[i]; e < grp[i + 1]; e++) {
            int32_t c = m1[gcol[e]];
            if (c >= 0 && (best < 0 || prio_gt(c, best, seed, off))) best = c;
        }
        if (best == i) state[i] = TAKEN;
    }
}

// r1[i] = 1 when i is taken or adjacent to a taken node
__global__ void mis_r1_kernel(int32_t n, const int32_t *__restrict__ grp, const int32_t *__restrict__ gcol,
                              const int32_t *__restrict__ state, int32_t *__restrict__ r1) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t f = (state[i] == TAKEN);
        for (int32_t e = grp[i]; e < grp[i + 1] && !f; e++) f = (state[gcol[e]] == TAKEN);
        r1[i] = f;
    }
}

// undecided nodes within distance 2 of a taken node are removed
__global__ void mis_remove_kernel(int32_t n, const int32_t *__restrict__ grp, const int32_t *__restrict__ gcol,
                                  const int32_t *__restrict__ r1, int32_t *__restrict__ state,
                                  int32_t *__restrict__ undecided) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != UNDECIDED) continue;
        int32_t f = r1[i];
        for (int32_t e = grp[i]; e < grp[i + 1] && !f; e++) f = r1[gcol[e]];
        if (f) state[i] = REMOVED;
        else atomicAdd(undecided, 1);
    }
}

__global__ void flag_taken_kernel(int32_t n, const int32_t *__restrict__ state, int32_t *__restrict__ flag) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = (state[i] == TAKEN);
}

__global__ void roots_kernel(int32_t n, const int32_t *__restrict__ state, const int32_t *__restrict__ cidx,
                             int32_t *__restrict__ roots) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (state[i] == TAKEN) roots[cidx[i]] = i;
}

// pass 1: join the neighbouring root of largest priority
__global__ void agg_pass1_kernel(int32_t n, const int32_t *__restrict__ grp, const int32_t *__restrict__ gcol,
                                 const int32_t *__restrict__ state, const int32_t *__restrict__ cidx, uint64_t seed,
                                 const int32_t *__restrict__ roff, int32_t *__restrict__ pass1) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t a = -1;
        if (state[i] == TAKEN) {
            a = cidx[i];
        } else if (state[i] == REMOVED) {
            const int32_t off = roff ? roff[i] : 0;
            int32_t best = -1;
            for (int32_t e = grp[i]; e < grp[i + 1]; e++) {
                int32_t j = gcol[e];
                if (state[j] == TAKEN && (best < 0 || prio_gt(j, best, seed, off))) best = j;
            }
            if (best >= 0) a = cidx[best];
        }
        pass1[i] = a;
    }
}

// pass 2: join the aggregate of the pass-1 neighbour whose root has the largest priority
__global__ void agg_pass2_kernel(int32_t n, const int32_t *__restrict__ grp, const int32_t *__restrict__ gcol,
                                 const int32_t *__restrict__ state, const int32_t *__restrict__ pass1,
                                 const int32_t *__restrict__ roots, uint64_t seed, const int32_t *__restrict__ roff,
                                 int32_t *__restrict__ agg, int32_t *__restrict__ bad) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t a = pass1[i];
        if (a < 0 && state[i] == REMOVED) {
            const int32_t off = roff ? roff[i] : 0;
            for (int32_t e = grp[i]; e < grp[i + 1]; e++) {
                int32_t c = pass1[gcol[e]];
                if (c < 0 || state[gcol[e]] == TAKEN) continue;
                if (a < 0 || prio_gt(roots[c], roots[a], seed, off)) a = c;
            }
            if (a < 0) atomicMax(bad, i + 1);
        }
        agg[i] = a;
    }
}

__global__ void rowtype_kernel(int32_t n, const int32_t *__restrict__ state, const int32_t *__restrict__ agg,
                               int32_t *__restrict__ rowtype) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        rowtype[i] = (state[i] == TAKEN) ? ROOT_ROW : (agg[i] < 0 ? UNAGG_ROW : FREE_ROW);
}

// ------------------------------------------------------------------ candidates (Sec. 3.1)
// one weighted-Jacobi sweep on A B = 0, summed in CSR order without FMA
__global__ void cand_jacobi_kernel(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                                   const double *__restrict__ aval, const double *__restrict__ B, double omega,
                                   double *__restrict__ Bn) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0, d = 0.0;
        for (int32_t e = arp[i]; e < arp[i + 1]; e++) {
            acc = __dadd_rn(acc, __dmul_rn(aval[e], B[acol[e]]));
            if (acol[e] == i) d = aval[e];
        }
        Bn[i] = __dsub_rn(B[i], __dmul_rn(omega, __ddiv_rn(acc, d)));
    }
}

__global__ void gather_kernel(int32_t nc, const int32_t *__restrict__ roots, const double *__restrict__ B,
                              double *__restrict__ Bc, int32_t *__restrict__ bad) {
    pdl_wait();
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        double v = B[roots[c]];
        Bc[c] = v;
        if (!(fabs(v) >= 1e-300)) atomicMax(bad, c + 1);
    }
}

// k > 1 candidates: the k columns of the row-major n x k B swept together,
// each column summed exactly as the single-candidate kernel sums it
__global__ void cand_jacobi_k_kernel(int32_t n, int k, const int32_t *__restrict__ arp,
                                     const int32_t *__restrict__ acol, const double *__restrict__ aval,
                                     const double *__restrict__ B, double omega, double *__restrict__ Bn) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc[RN_MAX_CANDIDATES] = {}, d = 0.0;
        for (int32_t e = arp[i]; e < arp[i + 1]; e++) {
            const int32_t j = acol[e];
            for (int c = 0; c < k; c++) acc[c] = __dadd_rn(acc[c], __dmul_rn(aval[e], B[(int64_t)j * k + c]));
            if (j == i) d = aval[e];
        }
        for (int c = 0; c < k; c++)
            Bn[(int64_t)i * k + c] = __dsub_rn(B[(int64_t)i * k + c], __dmul_rn(omega, __ddiv_rn(acc[c], d)));
    }
}

// Bc = B at the roots (nc x k); the first candidate must not vanish there
__global__ void gather_k_kernel(int32_t nc, int k, const int32_t *__restrict__ roots, const double *__restrict__ B,
                                double *__restrict__ Bc, int32_t *__restrict__ bad) {
    pdl_wait();
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        for (int a = 0; a < k; a++) Bc[(int64_t)c * k + a] = B[(int64_t)roots[c] * k + a];
        if (!(fabs(Bc[(int64_t)c * k]) >= 1e-300)) atomicMax(bad, c + 1);
    }
}

// k > 1 candidates (Sec. 3.6, eq. Tproj): every row fit works from the
// singular value decomposition Bc_J = U Sigma V^T of the row's |J| x k block
// of candidates, not from the Gram matrix Bc_J^T Bc_J, whose formation would
// square the condition number that multiplies rounding.  Singular values at
// most kSvCut of the largest are dropped (Gram eigenvalues at most 1e-12 of
// the largest): combinations the pattern carries only below that stay
// unfitted (minimal-norm least squares on the rest).
constexpr double kSvCut = 1e-6;

// One-sided Jacobi SVD (Hestenes) of every free row's Bc_J, thread per row:
// the columns of W = Bc_J V are rotated in U (the row's |J| x k slice,
// pattern-entry major) until every pair is orthogonal to 1e-15 of its norms
// (at most 30 sweeps).  On return U holds W_a / sigma_a for the kept
// directions (zero columns for dropped ones), VS (k x k per row) V_a /
// sigma_a, and zero_row marks rows whose constraints fix them (no more
// pattern entries than the rank kept; one-entry rows): those are projected to
// exactly 0, like a one-entry row for k = 1.
template <int K>
__global__ void row_svd_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ rowtype, const double *__restrict__ Bc,
                               double *__restrict__ U, double *__restrict__ VS, int32_t *__restrict__ zero_row) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t s0 = rp[i], len = rp[i + 1] - s0;
        double *W = U + (int64_t)s0 * K;
        double v[K * K];
#pragma unroll
        for (int a = 0; a < K; a++)
#pragma unroll
            for (int c = 0; c < K; c++) v[a * K + c] = (a == c) ? 1.0 : 0.0;
        const bool free_row = rowtype[i] == FREE_ROW && len >= 1;
        for (int32_t q = 0; q < len; q++)
#pragma unroll
            for (int a = 0; a < K; a++) W[(int64_t)q * K + a] = free_row ? Bc[(int64_t)col[s0 + q] * K + a] : 0.0;
        int rank = 0;
        if (free_row) {
            for (int sweep = 0; sweep < 30; sweep++) {
                bool rotated = false;
#pragma unroll
                for (int p = 0; p < K - 1; p++)
#pragma unroll
                    for (int r = p + 1; r < K; r++) {
                        double al = 0.0, be = 0.0, ga = 0.0;
                        for (int32_t q = 0; q < len; q++) {
                            const double wp = W[(int64_t)q * K + p], wr = W[(int64_t)q * K + r];
                            al += wp * wp;
                            be += wr * wr;
                            ga += wp * wr;
                        }
                        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                        rotated = true;
                        const double ze = (be - al) / (2.0 * ga);
                        const double t = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(ze * ze + 1.0));
                        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                        for (int32_t q = 0; q < len; q++) {
                            const double wp = W[(int64_t)q * K + p], wr = W[(int64_t)q * K + r];
                            W[(int64_t)q * K + p] = c * wp - sn * wr;
                            W[(int64_t)q * K + r] = sn * wp + c * wr;
                        }
#pragma unroll
                        for (int x = 0; x < K; x++) {
                            const double vp = v[x * K + p], vr = v[x * K + r];
                            v[x * K + p] = c * vp - sn * vr;
                            v[x * K + r] = sn * vp + c * vr;
                        }
                    }
                if (!rotated) break;
            }
            double sig[K], smax = 0.0;
#pragma unroll
            for (int a = 0; a < K; a++) {
                double ss = 0.0;
                for (int32_t q = 0; q < len; q++) ss += W[(int64_t)q * K + a] * W[(int64_t)q * K + a];
                sig[a] = sqrt(ss);
                smax = fmax(smax, sig[a]);
            }
#pragma unroll
            for (int a = 0; a < K; a++) {
                const bool keep = sig[a] > kSvCut * smax;
                rank += keep ? 1 : 0;
                const double is = keep ? 1.0 / sig[a] : 0.0;
                for (int32_t q = 0; q < len; q++) W[(int64_t)q * K + a] = keep ? W[(int64_t)q * K + a] * is : 0.0;
#pragma unroll
                for (int x = 0; x < K; x++) v[x * K + a] = keep ? v[x * K + a] * is : 0.0;
            }
        }
#pragma unroll
        for (int x = 0; x < K * K; x++) VS[(int64_t)i * K * K + x] = free_row ? v[x] : 0.0;
        zero_row[i] = free_row ? (len <= 1 || rank >= len) : 1;
    }
}

// Minimal-norm fit of every free row (eq. Tproj): (t + u) Bc_J = B_i with
// r = B_i - t Bc_J and u = (r V Sigma^+) U^T, from row_svd_kernel on the same
// pattern and Bc; T's construction and enforce for k > 1.
template <int K>
__global__ void row_fit_u_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 double *__restrict__ val, const int32_t *__restrict__ rowtype,
                                 const double *__restrict__ B, const double *__restrict__ Bc,
                                 const double *__restrict__ U, const double *__restrict__ VS) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (rowtype[i] != FREE_ROW) continue;
        double r[K], y[K];
#pragma unroll
        for (int a = 0; a < K; a++) r[a] = B[(int64_t)i * K + a];
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            const double *b = Bc + (int64_t)col[e] * K;
#pragma unroll
            for (int a = 0; a < K; a++) r[a] -= val[e] * b[a];
        }
        const double *vs = VS + (int64_t)i * K * K;
#pragma unroll
        for (int c = 0; c < K; c++) {
            y[c] = 0.0;
#pragma unroll
            for (int a = 0; a < K; a++) y[c] += r[a] * vs[a * K + c];
        }
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            const double *u = U + (int64_t)e * K;
            double d = 0.0;
#pragma unroll
            for (int c = 0; c < K; c++) d += y[c] * u[c];
            val[e] += d;
        }
    }
}

// launch of a K-templated row kernel for the runtime k (2..RN_MAX_CANDIDATES)
#define RN_K_SWITCH(k, CALL)          \
    switch (k) {                      \
        case 2: { constexpr int KK = 2; CALL; } break; \
        case 3: { constexpr int KK = 3; CALL; } break; \
        default: { constexpr int KK = 4; CALL; } break; \
    }

// ------------------------------------------------------------------ systems (Sec. 3.2-3.6, block size m > 1)
constexpr int kAmalMax = 256;  // entries of one node row of S gathered for amalgamation

// S_m(I, J) = the largest entry of S's m x m block (I, J) (entries S stores):
// thread per node, its m rows' entries merged by node column in a sorted
// list.  Pass 1 (FILL false) counts; pass 2 writes.
template <bool FILL>
__global__ void amalgamate_kernel(int32_t nn, int m, const int32_t *__restrict__ srp, const int32_t *__restrict__ scol,
                                  const double *__restrict__ sval, int32_t *__restrict__ count,
                                  const int32_t *__restrict__ orp, int32_t *__restrict__ ocol, double *__restrict__ oval,
                                  int32_t *__restrict__ bad) {
    pdl_wait();
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nn; I += gridDim.x * blockDim.x) {
        int32_t cols[kAmalMax];
        double vals[kAmalMax];
        int u = 0;
        bool over = false;
        for (int32_t i = I * m; i < I * m + m && !over; i++)
            for (int32_t e = srp[i]; e < srp[i + 1]; e++) {
                const int32_t J = scol[e] / m;
                const double v = sval[e];
                int q = u;
                while (q > 0 && cols[q - 1] > J) q--;
                if (q > 0 && cols[q - 1] == J) {
                    if (v > vals[q - 1]) vals[q - 1] = v;
                    continue;
                }
                if (u == kAmalMax) { over = true; break; }
                for (int t = u; t > q; t--) { cols[t] = cols[t - 1]; vals[t] = vals[t - 1]; }
                cols[q] = J;
                vals[q] = v;
                u++;
            }
        if (over) atomicMax(bad, I + 1);
        if (!FILL) {
            count[I] = u;
        } else {
            for (int q = 0; q < u; q++) {
                ocol[orp[I] + q] = cols[q];
                oval[orp[I] + q] = vals[q];
            }
        }
    }
}

// node aggregates and row types to unknowns; root nodes to their m root unknowns
__global__ void unamalgamate_nodes_kernel(int32_t n, int m, const int32_t *__restrict__ aggn,
                                          const int32_t *__restrict__ rtn, int32_t *__restrict__ agg,
                                          int32_t *__restrict__ rowtype) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        agg[i] = aggn[i / m];
        rowtype[i] = rtn[i / m];
    }
}
__global__ void unamalgamate_roots_kernel(int32_t ncn, int m, const int32_t *__restrict__ rootsn,
                                          int32_t *__restrict__ roots) {
    pdl_wait();
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < ncn; r += gridDim.x * blockDim.x)
        for (int c = 0; c < m; c++) roots[m * r + c] = m * rootsn[r] + c;
}

// N(i, m J + c) = N_m(floor(i/m), J), c < m; a root unknown i of aggregate a
// gets the identity row {m a + i mod m}
template <bool FILL>
__global__ void unamalgamate_pattern_kernel(int32_t n, int m, const int32_t *__restrict__ nrp,
                                            const int32_t *__restrict__ ncol, const double *__restrict__ nval,
                                            const int32_t *__restrict__ agg, const int32_t *__restrict__ rowtype,
                                            int32_t *__restrict__ count, const int32_t *__restrict__ orp,
                                            int32_t *__restrict__ ocol, double *__restrict__ oval) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t I = i / m;
        if (!FILL) {
            count[i] = rowtype[i] == ROOT_ROW ? 1 : m * (nrp[I + 1] - nrp[I]);
            continue;
        }
        int32_t dst = orp[i];
        if (rowtype[i] == ROOT_ROW) {
            ocol[dst] = m * agg[i] + i % m;
            oval[dst] = 1.0;
            continue;
        }
        for (int32_t e = nrp[I]; e < nrp[I + 1]; e++)
            for (int c = 0; c < m; c++) {
                ocol[dst] = m * ncol[e] + c;
                oval[dst++] = nval[e];
            }
    }
}

// The inverse of every aggregate's root block Broot_a (m x m: the first m
// candidates at its m root unknowns), Gauss-Jordan with partial pivoting;
// a pivot at most 1e-12 of the block's largest entry flags the aggregate.
__global__ void root_block_inverse_kernel(int32_t na, int m, int k, const int32_t *__restrict__ roots,
                                          const double *__restrict__ B, double *__restrict__ Binv,
                                          int32_t *__restrict__ bad) {
    pdl_wait();
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
        double M[RN_MAX_BLOCK * RN_MAX_BLOCK], X[RN_MAX_BLOCK * RN_MAX_BLOCK];
        double amax = 0.0;
        for (int r = 0; r < m; r++)
            for (int c = 0; c < m; c++) {
                M[r * m + c] = B[(int64_t)roots[m * a + r] * k + c];
                X[r * m + c] = (r == c) ? 1.0 : 0.0;
                amax = fmax(amax, fabs(M[r * m + c]));
            }
        bool ok = true;
        for (int col = 0; col < m && ok; col++) {
            int piv = col;
            for (int r = col + 1; r < m; r++)
                if (fabs(M[r * m + col]) > fabs(M[piv * m + col])) piv = r;
            if (!(fabs(M[piv * m + col]) > 1e-12 * amax)) { ok = false; break; }
            for (int c = 0; c < m; c++) {
                double t = M[col * m + c]; M[col * m + c] = M[piv * m + c]; M[piv * m + c] = t;
                t = X[col * m + c]; X[col * m + c] = X[piv * m + c]; X[piv * m + c] = t;
            }
            const double d = M[col * m + col];
            for (int c = 0; c < m; c++) { M[col * m + c] /= d; X[col * m + c] /= d; }
            for (int r = 0; r < m; r++) {
                if (r == col) continue;
                const double f = M[r * m + col];
                for (int c = 0; c < m; c++) {
                    M[r * m + c] -= f * M[col * m + c];
                    X[r * m + c] -= f * X[col * m + c];
                }
            }
        }
        if (!ok) atomicMax(bad, a + 1);
        for (int q = 0; q < m * m; q++) Binv[(int64_t)a * m * m + q] = ok ? X[q] : 0.0;
    }
}

// T for block size m (eq. root-nodeform): T_i,(m a + c) = (B_i,0:m Broot_a^{-1})_c
// on the own aggregate's block, 0 elsewhere; root unknowns exact identity rows
__global__ void tentative_block_kernel(int32_t n, int m, int k, const int32_t *__restrict__ rp,
                                       const int32_t *__restrict__ col, const int32_t *__restrict__ agg,
                                       const int32_t *__restrict__ rowtype, const double *__restrict__ B,
                                       const double *__restrict__ Binv, double *__restrict__ T) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t a = agg[i];
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            const int32_t j = col[e];
            double t = 0.0;
            if (a >= 0 && j / m == a) {
                if (rowtype[i] == ROOT_ROW) {
                    t = (j == m * a + i % m) ? 1.0 : 0.0;
                } else {
                    const double *X = Binv + (int64_t)a * m * m;
                    for (int r = 0; r < m; r++) t += B[(int64_t)i * k + r] * X[r * m + j % m];
                }
            }
            T[e] = t;
        }
    }
}

// ------------------------------------------------------------------ pattern (Sec. 3.4-3.5)
__global__ void aggflag_kernel(int32_t n, const int32_t *__restrict__ agg, int32_t *__restrict__ flag) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = agg[i] >= 0;
}

__global__ void c_matrix_kernel(int32_t n, const int32_t *__restrict__ agg, const int32_t *__restrict__ rp,
                                int32_t *__restrict__ col, double *__restrict__ val) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (agg[i] >= 0) {
            col[rp[i]] = agg[i];
            val[rp[i]] = 1.0;
        }
}

// pre-filter (Alg. 4, drop tolerance) on free rows, root rows -> identity row
template <bool FILL>
__global__ void prefilter_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const double *__restrict__ val, const int32_t *__restrict__ rowtype,
                                 const int32_t *__restrict__ agg, double theta, double omg, int32_t *__restrict__ count,
                                 const int32_t *__restrict__ frp, int32_t *__restrict__ fcol,
                                 double *__restrict__ fval) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = rowtype[i];
        const int32_t a = agg[i];
        double thr = 0.0;
        if (t == FREE_ROW && theta > 0.0) {
            double m = 0.0;
            for (int32_t e = rp[i]; e < rp[i + 1]; e++)
                if (fabs(val[e]) > m) m = fabs(val[e]);
            thr = __dmul_rn(__dmul_rn(theta, m), omg);
        }
        int32_t c = 0, dst = FILL ? frp[i] : 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            bool keep;
            if (t == ROOT_ROW) keep = (col[e] == a);
            else if (t == FREE_ROW) keep = (theta <= 0.0) || (fabs(val[e]) >= thr) || (col[e] == a);
            else keep = false;
            if (keep) {
                if (FILL) {
                    fcol[dst] = col[e];
                    fval[dst] = (t == ROOT_ROW) ? 1.0 : val[e];
                    dst++;
                }
                c++;
            }
        }
        if (!FILL) count[i] = c;
    }
}

// T on the pattern (eq. root-nodeform): T_{i,agg(i)} = B_i / Bc_{agg(i)}
// (first candidate; k the row stride of B and Bc)
__global__ void tentative_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const int32_t *__restrict__ agg, const double *__restrict__ B,
                                 const double *__restrict__ Bc, double *__restrict__ T, int k) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            int32_t j = col[e];
            T[e] = (j == agg[i]) ? __ddiv_rn(B[(int64_t)i * k], Bc[(int64_t)j * k]) : 0.0;
        }
}

// ------------------------------------------------------------------ k > 1: the row projection as a pass
// W <- scale (W - (W_i U) U^T) on every free row that the constraints do not
// fix (eq. Tproj with a zero right-hand side, through the orthonormal basis U
// of the range of Bc_J: no division by a singular value), rows they fix <- 0;
// the product kernels ran unprojected (their row scales are zero).  <Y, W>
// finishes in Fin.
template <typename TV, int K>
__global__ void __launch_bounds__(256)
proj_k_kernel(int32_t n, const int32_t *__restrict__ nrp, const int32_t *__restrict__ zero_row,
              const TV *__restrict__ U, TV *__restrict__ W, TV scale, const TV *__restrict__ Y, Fin fin) {
    pdl_wait();
    __shared__ double s_red[32];
    TV dot = TV(0);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t cs = nrp[i], ce = nrp[i + 1];
        if (zero_row[i]) {  // constraint space {0}
            for (int32_t q = cs; q < ce; q++) W[q] = TV(0);
            continue;
        }
        TV c[K] = {};
        for (int32_t q = cs; q < ce; q++) {
            const TV *u = U + (int64_t)q * K;
#pragma unroll
            for (int a = 0; a < K; a++) c[a] = fma(W[q], u[a], c[a]);
        }
        for (int32_t q = cs; q < ce; q++) {
            const TV *u = U + (int64_t)q * K;
            TV d = TV(0);
#pragma unroll
            for (int a = 0; a < K; a++) d = fma(c[a], u[a], d);
            const TV w = scale * (W[q] - d);
            W[q] = w;
            if (Y) dot = fma(Y[q], w, dot);
        }
    }
    const double d[1] = {(double)dot};
    grid_finish<256, 1>(d, fin, s_red);
}

// Per-minimisation data of the k > 1 projection: U on the pattern (FP64, or
// rounded for FP32 sweeps) and the rows the constraints fix.
template <typename TV>
struct KProj {
    int k = 1;
    DVec<double> u64, vs_own;
    DVec<int32_t> zero_row_own;
    DVec<TV> uv;
    const TV *u = nullptr;
    const int32_t *zero_row = nullptr;
    // pre_u / pre_zr: U and the fixed-row flags already formed on this
    // pattern and Bc (row_svd_kernel), or null to form them here
    void build(int k_, const Pattern &N, const int32_t *rowtype, const double *Bc, cudaStream_t s,
               const double *pre_u = nullptr, const int32_t *pre_zr = nullptr) {
        k = k_;
        if (k == 1) return;
        const double *U64 = pre_u;
        zero_row = pre_zr;
        if (!pre_u || !pre_zr) {
            u64.alloc((size_t)std::max<int64_t>(N.nnz, 1) * k, s);
            vs_own.alloc((size_t)N.n * k * k, s);
            zero_row_own.alloc(N.n, s);
            RN_K_SWITCH(k, RN_LAUNCH("energy_proj_scale", 4.0 * N.nnz + 16.0 * k * N.nnz + 8.0 * k * k * N.n, s,
                                     row_svd_kernel<KK>, grid_for(N.n, 256), 256, 0, N.n, N.rp, N.col, rowtype, Bc,
                                     u64.p, vs_own.p, zero_row_own.p));
            U64 = u64.p;
            zero_row = zero_row_own.p;
        }
        if constexpr (sizeof(TV) == 4) {
            uv.alloc((size_t)std::max<int64_t>(N.nnz, 1) * k, s);
            to_float(U64, uv.p, (int64_t)N.nnz * k, s);
            u = uv.p;
        } else {
            u = U64;
        }
    }
    void apply(const Pattern &N, const int32_t *rowtype, TV *W, double scale, const TV *Y, const Fin &f,
               cudaStream_t s) const {
        (void)rowtype;
        RN_K_SWITCH(k, {
            const int g = grid_resident(proj_k_kernel<TV, KK>, 256, 0, N.n, 256, kReduceBlocks);
            RN_LAUNCH("energy_masked_product", (2.0 * sizeof(TV) + sizeof(TV) * k) * N.nnz + 8.0 * N.n, s,
                      (proj_k_kernel<TV, KK>), g, 256, 0, N.n, N.rp, zero_row, u, W, (TV)scale, Y, f);
        });
    }
};

// ------------------------------------------------------------------ CG energy minimisation (Sec. 3.6)
// Device scalars: sc[0] rho, sc[1] rho0, sc[2] beta, sc[3] <Dd,W>, sc[4] alpha; fl[0] = done.
// The scalar recurrences run in the finishing block of each reduction (Fin).
// dinv: the preconditioner D^{-1} as the inverted diagonal (nullptr: none).
// TV: the value type of the sweeps (double; float in mixed precision, with
// per-thread sums in TV joining the FP64 grid reduction).
template <int G, typename TV>
__global__ void __launch_bounds__(kT)
cg_rho_kernel(int32_t n, const int32_t *__restrict__ rp, const TV *__restrict__ R, const TV *__restrict__ dinv,
              Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    TV acc = TV(0);
    for (int32_t i = blockIdx.x * (kT / G) + g; i < n; i += gridDim.x * (kT / G)) {
        const int32_t q0 = rp[i], q1 = rp[i + 1];
        const TV di = dinv ? dinv[i] : TV(1);
        for (int32_t q = q0 + lane; q < q1; q += G) acc = fma(R[q], R[q] * di, acc);
    }
    const double v[1] = {(double)acc};
    grid_finish<kT, 1>(v, fin, sm);
}

template <int G, typename TV>
__global__ void __launch_bounds__(kT)
cg_dd_kernel(int32_t n, const int32_t *__restrict__ rp, const TV *__restrict__ R, const TV *__restrict__ dinv,
             const double *__restrict__ sc, const int32_t *__restrict__ fl, int first, TV *__restrict__ Dd) {
    pdl_wait();
    if (fl[0]) return;
    const TV beta = (TV)sc[2];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    for (int32_t i = blockIdx.x * (kT / G) + g; i < n; i += gridDim.x * (kT / G)) {
        const int32_t q0 = rp[i], q1 = rp[i + 1];
        const TV di = dinv ? dinv[i] : TV(1);
        for (int32_t q = q0 + lane; q < q1; q += G) {
            const TV z = R[q] * di;
            Dd[q] = first ? z : z + beta * Dd[q];
        }
    }
}

template <int G, typename TV>
__global__ void __launch_bounds__(kT)
cg_update_kernel(int32_t n, const int32_t *__restrict__ rp, TV *__restrict__ P, TV *__restrict__ R,
                 const TV *__restrict__ Dd, const TV *__restrict__ W, const TV *__restrict__ dinv,
                 const double *__restrict__ sc, const int32_t *__restrict__ fl, Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    const bool done = fl[0] != 0;
    const TV alpha = (TV)sc[4];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    TV acc = TV(0);
    if (!done) {
        for (int32_t i = blockIdx.x * (kT / G) + g; i < n; i += gridDim.x * (kT / G)) {
            const int32_t q0 = rp[i], q1 = rp[i + 1];
            const TV di = dinv ? dinv[i] : TV(1);
            for (int32_t q = q0 + lane; q < q1; q += G) {
                P[q] = P[q] + alpha * Dd[q];
                const TV r = R[q] - alpha * W[q];
                R[q] = r;
                acc = fma(r, r * di, acc);
            }
        }
    }
    const double v[1] = {(double)acc};
    grid_finish<kT, 1>(v, fin, sm);  // the finisher ignores the sum once done is set
}

// Elementwise forms of the three kernels above for the plan's per-entry
// D^{-1} (de): no row structure, four consecutive entries per thread (vector
// loads when VEC: every array 16-byte aligned), the same expressions per
// entry.  The reductions add per-thread sums in a fixed order.
template <typename TV, bool VEC>
__device__ __forceinline__ void ld4(const TV *__restrict__ p, int64_t q, TV (&v)[4]) {
    if constexpr (VEC && sizeof(TV) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p + q);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (VEC) {
        const double2 a = *reinterpret_cast<const double2 *>(p + q);
        const double2 b = *reinterpret_cast<const double2 *>(p + q + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = p[q + k];
    }
}
template <typename TV, bool VEC>
__device__ __forceinline__ void st4(TV *__restrict__ p, int64_t q, const TV (&v)[4]) {
    if constexpr (VEC && sizeof(TV) == 4) {
        *reinterpret_cast<float4 *>(p + q) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (VEC) {
        *reinterpret_cast<double2 *>(p + q) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + q + 2) = make_double2(v[2], v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) p[q + k] = v[k];
    }
}

template <typename TV, bool VEC>
__global__ void __launch_bounds__(kT)
cg_rho_flat_kernel(int64_t nz, const TV *__restrict__ R, const TV *__restrict__ de, Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    TV acc = TV(0);
    const int64_t stride = (int64_t)gridDim.x * kT * 4;
    for (int64_t q = ((int64_t)blockIdx.x * kT + threadIdx.x) * 4; q < nz; q += stride) {
        if (q + 4 <= nz) {
            TV r[4], d[4];
            ld4<TV, VEC>(R, q, r);
            ld4<TV, VEC>(de, q, d);
#pragma unroll
            for (int k = 0; k < 4; k++) acc = fma(r[k], r[k] * d[k], acc);
        } else {
            for (int64_t t = q; t < nz; t++) acc = fma(R[t], R[t] * de[t], acc);
        }
    }
    const double v[1] = {(double)acc};
    grid_finish<kT, 1>(v, fin, sm);
}

template <typename TV, bool VEC>
__global__ void __launch_bounds__(kT)
cg_dd_flat_kernel(int64_t nz, const TV *__restrict__ R, const TV *__restrict__ de, const double *__restrict__ sc,
                  const int32_t *__restrict__ fl, int first, TV *__restrict__ Dd) {
    pdl_wait();
    if (fl[0]) return;
    const TV beta = (TV)sc[2];
    const int64_t stride = (int64_t)gridDim.x * kT * 4;
    for (int64_t q = ((int64_t)blockIdx.x * kT + threadIdx.x) * 4; q < nz; q += stride) {
        if (q + 4 <= nz) {
            TV r[4], d[4], o[4];
            ld4<TV, VEC>(R, q, r);
            ld4<TV, VEC>(de, q, d);
            if (!first) ld4<TV, VEC>(Dd, q, o);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const TV z = r[k] * d[k];
                o[k] = first ? z : z + beta * o[k];
            }
            st4<TV, VEC>(Dd, q, o);
        } else {
            for (int64_t t = q; t < nz; t++) {
                const TV z = R[t] * de[t];
                Dd[t] = first ? z : z + beta * Dd[t];
            }
        }
    }
}

template <typename TV, bool VEC>
__global__ void __launch_bounds__(kT)
cg_update_flat_kernel(int64_t nz, TV *__restrict__ P, TV *__restrict__ R, const TV *__restrict__ Dd,
                      const TV *__restrict__ W, const TV *__restrict__ de, const double *__restrict__ sc,
                      const int32_t *__restrict__ fl, Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    const bool done = fl[0] != 0;
    const TV alpha = (TV)sc[4];
    TV acc = TV(0);
    if (!done) {
        const int64_t stride = (int64_t)gridDim.x * kT * 4;
        for (int64_t q = ((int64_t)blockIdx.x * kT + threadIdx.x) * 4; q < nz; q += stride) {
            if (q + 4 <= nz) {
                TV p[4], r[4], d[4], w[4], di[4];
                ld4<TV, VEC>(P, q, p);
                ld4<TV, VEC>(R, q, r);
                ld4<TV, VEC>(Dd, q, d);
                ld4<TV, VEC>(W, q, w);
                ld4<TV, VEC>(de, q, di);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    p[k] = p[k] + alpha * d[k];
                    r[k] = r[k] - alpha * w[k];
                    acc = fma(r[k], r[k] * di[k], acc);
                }
                st4<TV, VEC>(P, q, p);
                st4<TV, VEC>(R, q, r);
            } else {
                for (int64_t t = q; t < nz; t++) {
                    P[t] = P[t] + alpha * Dd[t];
                    const TV rr = R[t] - alpha * W[t];
                    R[t] = rr;
                    acc = fma(rr, rr * de[t], acc);
                }
            }
        }
    }
    const double v[1] = {(double)acc};
    grid_finish<kT, 1>(v, fin, sm);  // the finisher ignores the sum once done is set
}

// ------------------------------------------------------------------ per-problem energy CG (merged setup)
// Independent problems set up together share the pattern's value arrays
// (problem p's entries are one contiguous range), but each keeps its own CG
// step lengths, as if set up alone.  Reductions go by chunks of at most
// kSegChunk entries of one problem: a block sums a chunk's entries into
// part[c]; the last block to arrive adds every problem's chunks in chunk
// order and runs that problem's recurrence (the single-problem finisher's,
// per problem).  sc: 8 doubles per problem ([0] rho, [1] rho0, [2] beta,
// [3] <D,W>, [4] alpha); fl: one "done" flag per problem.
constexpr int kSegChunk = 4096;

struct SegCg {
    const int32_t *lo = nullptr, *hi = nullptr, *pid = nullptr, *pc = nullptr;
    int nch = 0, np = 0;
    double *part = nullptr;
    unsigned *counter = nullptr;
    double *sc = nullptr;
    int32_t *fl = nullptr;
    double stop = 0.0;
};

__device__ void seg_finish(const SegCg &g, int mode, int it) {
    for (int p = threadIdx.x; p < g.np; p += blockDim.x) {
        double v = 0.0;
        for (int c = g.pc[p]; c < g.pc[p + 1]; c++) v += __ldcg(&g.part[c]);
        if (g.fl[p]) continue;
        double *sc = g.sc + 8 * p;
        if (mode == FIN_CG_RHO) {
            if (it == 0) sc[1] = v;
            if (v == 0.0 || v <= g.stop * sc[1]) {
                g.fl[p] = 1;
                continue;
            }
            sc[2] = (it == 0) ? 0.0 : v / sc[0];
            sc[0] = v;
        } else {  // FIN_CG_DW
            sc[3] = v;
            if (!(v > 0.0)) {
                g.fl[p] = 1;
                continue;
            }
            sc[4] = sc[0] / v;
        }
    }
}

// the block's chunk sum to part[c]
__device__ __forceinline__ void seg_chunk_store(const SegCg &g, int c, double v, double *sm) {
    const double t = block_sum<kT>(v, sm);
    if (threadIdx.x == 0) g.part[c] = t;
}

__device__ __forceinline__ void seg_arrive(const SegCg &g, int mode, int it) {
    __shared__ int am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(g.counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) {
        __threadfence();
        seg_finish(g, mode, it);
        __syncthreads();
        if (threadIdx.x == 0) {
            *g.counter = 0u;
            __threadfence();
        }
    }
}

// rho = <R, D^{-1} R> per problem
template <typename TV>
__global__ void __launch_bounds__(kT) seg_rho_kernel(SegCg g, const TV *__restrict__ R, const TV *__restrict__ de,
                                                     int it) {
    pdl_wait();
    __shared__ double sm[32];
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        TV acc = TV(0);
        if (!g.fl[g.pid[c]])
            for (int32_t q = g.lo[c] + threadIdx.x; q < g.hi[c]; q += kT) acc = fma(R[q], R[q] * de[q], acc);
        seg_chunk_store(g, c, (double)acc, sm);
    }
    seg_arrive(g, FIN_CG_RHO, it);
}

// Dd = D^{-1} R (+ beta_p Dd after the first sweep)
template <typename TV>
__global__ void __launch_bounds__(kT) seg_dd_kernel(SegCg g, const TV *__restrict__ R, const TV *__restrict__ de,
                                                    int first, TV *__restrict__ Dd) {
    pdl_wait();
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        const int p = g.pid[c];
        if (g.fl[p]) continue;
        const TV beta = (TV)g.sc[8 * p + 2];
        for (int32_t q = g.lo[c] + threadIdx.x; q < g.hi[c]; q += kT) {
            const TV z = R[q] * de[q];
            Dd[q] = first ? z : z + beta * Dd[q];
        }
    }
}

// <Dd, W> per problem and alpha
template <typename TV>
__global__ void __launch_bounds__(kT) seg_dw_kernel(SegCg g, const TV *__restrict__ Dd, const TV *__restrict__ W) {
    pdl_wait();
    __shared__ double sm[32];
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        TV acc = TV(0);
        if (!g.fl[g.pid[c]])
            for (int32_t q = g.lo[c] + threadIdx.x; q < g.hi[c]; q += kT) acc = fma(Dd[q], W[q], acc);
        seg_chunk_store(g, c, (double)acc, sm);
    }
    seg_arrive(g, FIN_CG_DW, 0);
}

// X += alpha_p Dd, R -= alpha_p W, rho and beta per problem
template <typename TV>
__global__ void __launch_bounds__(kT) seg_update_kernel(SegCg g, TV *__restrict__ P, TV *__restrict__ R,
                                                        const TV *__restrict__ Dd, const TV *__restrict__ W,
                                                        const TV *__restrict__ de, int it) {
    pdl_wait();
    __shared__ double sm[32];
    for (int c = blockIdx.x; c < g.nch; c += gridDim.x) {
        const int p = g.pid[c];
        TV acc = TV(0);
        if (!g.fl[p]) {
            const TV alpha = (TV)g.sc[8 * p + 4];
            for (int32_t q = g.lo[c] + threadIdx.x; q < g.hi[c]; q += kT) {
                P[q] = P[q] + alpha * Dd[q];
                const TV rr = R[q] - alpha * W[q];
                R[q] = rr;
                acc = fma(rr, rr * de[q], acc);
            }
        }
        seg_chunk_store(g, c, (double)acc, sm);
    }
    seg_arrive(g, FIN_CG_RHO, it);
}

// D^{-1} per pattern entry from the per-row diagonal inverse (1 without the preconditioner)
template <typename TV>
__global__ void entry_dinv_kernel(int32_t n, const int32_t *__restrict__ rp, const double *__restrict__ dinv,
                                  TV *__restrict__ de) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const TV d = dinv ? (TV)dinv[i] : TV(1);
        for (int32_t q = rp[i]; q < rp[i + 1]; q++) de[q] = d;
    }
}

// out[t] = src[idx[t]] (the values of a row-pointer array at given rows)
__global__ void gather_i32_kernel(int32_t m, const int32_t *__restrict__ src, const int32_t *__restrict__ idx,
                                  int32_t *__restrict__ out) {
    pdl_wait();
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) out[t] = src[idx[t]];
}

// ------------------------------------------------------------------ GMRES energy minimisation (Sec. 4.2)
// sc[0] beta, sc[1] ||w||^2 / scratch, fl[0] done, fl[1] k (number of finished steps)
__global__ void gm_start_kernel(double *sc, int32_t *fl, double *g) {
    pdl_wait();
    const double b2 = sc[1];
    fl[0] = 0;
    fl[1] = 0;
    if (!(b2 > 0.0)) {
        fl[0] = 1;
        return;
    }
    const double beta = sqrt(b2);
    sc[0] = beta;
    g[0] = beta;
}

// TV: the sweeps' value type (double; float in mixed precision, the Arnoldi
// scalars staying FP64)
template <typename TV>
__global__ void gm_scale_kernel(int64_t nz, TV *__restrict__ v, const double *__restrict__ den,
                                const int32_t *__restrict__ fl) {
    pdl_wait();
    if (fl[0]) return;
    const TV d = (TV)*den;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nz; q += (int64_t)gridDim.x * blockDim.x)
        v[q] = v[q] / d;
}

template <typename TV>
__global__ void gm_axpy_kernel(int64_t nz, TV *__restrict__ w, const TV *__restrict__ v,
                               const double *__restrict__ h, const int32_t *__restrict__ fl) {
    pdl_wait();
    if (fl[0]) return;
    const TV c = (TV)*h;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nz; q += (int64_t)gridDim.x * blockDim.x)
        w[q] = w[q] - c * v[q];
}

// <x, y> of two TV arrays: per-thread sums in TV, grid reduction in FP64
template <typename TV>
__global__ void __launch_bounds__(kT) gm_dot_kernel(int64_t nz, const TV *__restrict__ x, const TV *__restrict__ y,
                                                    Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    TV acc = TV(0);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nz; q += (int64_t)gridDim.x * blockDim.x)
        acc = fma(x[q], y[q], acc);
    const double v[1] = {(double)acc};
    grid_finish<kT, 1>(v, fin, sm);
}

// Givens update of Hessenberg column j; H row-major (m+1) x m
__global__ void gm_givens_kernel(int m, int j, double *H, double *cs, double *sn, double *g, double *sc, int32_t *fl,
                                 double brk) {
    pdl_wait();
    if (fl[0]) return;
    const double hn = sqrt(sc[1]);
    H[(j + 1) * m + j] = hn;
    for (int i = 0; i < j; i++) {
        double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
    }
    const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
    if (den == 0.0) {
        fl[0] = 1;
        return;
    }
    cs[j] = H[j * m + j] / den;
    sn[j] = H[(j + 1) * m + j] / den;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    fl[1] = j + 1;
    sc[2] = hn;  // next basis vector = w / hn
    if (hn <= brk * sc[0]) fl[0] = 1;
}

__global__ void gm_backsolve_kernel(int m, const double *H, const double *g, double *y, const int32_t *fl) {
    pdl_wait();
    const int k = fl[1];
    for (int i = k - 1; i >= 0; i--) {
        double s = g[i];
        for (int j = i + 1; j < k; j++) s -= H[i * m + j] * y[j];
        y[i] = s / H[i * m + i];
    }
    for (int i = k; i < m; i++) y[i] = 0.0;
}

template <typename TV>
__global__ void gm_combine_kernel(int64_t nz, int m, TV *__restrict__ P, const TV *__restrict__ V,
                                  const double *__restrict__ y, const int32_t *__restrict__ fl) {
    pdl_wait();
    const int k = fl[1];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nz; q += (int64_t)gridDim.x * blockDim.x) {
        TV p = P[q];
        for (int j = 0; j < k; j++) p = p + (TV)y[j] * V[(int64_t)j * nz + q];
        P[q] = p;
    }
}

// ------------------------------------------------------------------ post-filter + enforce (Sec. 3.7)
template <bool FILL>
__global__ void postfilter_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                  const double *__restrict__ val, const int32_t *__restrict__ rowtype,
                                  const int32_t *__restrict__ agg, double theta, double omg,
                                  int32_t *__restrict__ count, const int32_t *__restrict__ frp,
                                  int32_t *__restrict__ fcol, double *__restrict__ fval, int mb) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool fr = rowtype[i] == FREE_ROW;
        double thr = 0.0;
        if (fr) {
            double m = 0.0;
            for (int32_t e = rp[i]; e < rp[i + 1]; e++)
                if (fabs(val[e]) > m) m = fabs(val[e]);
            thr = __dmul_rn(__dmul_rn(theta, m), omg);
        }
        int32_t c = 0, dst = FILL ? frp[i] : 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            bool keep = !fr || fabs(val[e]) >= thr || col[e] / mb == agg[i];  // own aggregate's block kept
            if (keep) {
                if (FILL) {
                    fcol[dst] = col[e];
                    fval[dst] = val[e];
                    dst++;
                }
                c++;
            }
        }
        if (!FILL) count[i] = c;
    }
}

// minimal-norm row fit (t + u) Bc = B_i on the row's pattern (eq. Tproj)
__global__ void enforce_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                               double *__restrict__ val, const int32_t *__restrict__ rowtype,
                               const double *__restrict__ B, const double *__restrict__ Bc) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (rowtype[i] != FREE_ROW) continue;
        double tb = 0.0, bb = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            const double b = Bc[col[e]];
            tb += val[e] * b;
            bb += b * b;
        }
        const double c = (B[i] - tb) / bb;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) val[e] = val[e] + c * Bc[col[e]];
    }
}

// ------------------------------------------------------------------ coarsest level: dense LU -> inverse
__global__ void csr_to_dense_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                    const double *__restrict__ val, double *__restrict__ M) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) M[(int64_t)i * n + col[e]] = val[e];
}

// One block: partial pivoting (largest |pivot|, lowest row on ties), in place.
__global__ void __launch_bounds__(1024) dense_lu_kernel(int n, double *M, int32_t *piv, int32_t *flag) {
    pdl_wait();
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ double amax;
    __shared__ int pivrow;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    double m = 0.0;
    for (int64_t q = tid; q < (int64_t)n * n; q += blockDim.x) m = fmax(m, fabs(M[q]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sv[w] = m;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < nw; k++) a = fmax(a, sv[k]);
        amax = a;
    }
    __syncthreads();
    for (int k = 0; k < n; k++) {
        double best = -1.0;
        int brow = n;
        for (int i = k + tid; i < n; i += blockDim.x) {
            double v = fabs(M[(int64_t)i * n + k]);
            if (v > best || (v == best && i < brow)) { best = v; brow = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, o);
            int orow = __shfl_xor_sync(0xffffffffu, brow, o);
            if (ov > best || (ov == best && orow < brow)) { best = ov; brow = orow; }
        }
        if (lane == 0) { sv[w] = best; si[w] = brow; }
        __syncthreads();
        if (tid == 0) {
            double b = -1.0;
            int r = n;
            for (int q = 0; q < nw; q++)
                if (sv[q] > b || (sv[q] == b && si[q] < r)) { b = sv[q]; r = si[q]; }
            pivrow = r;
            piv[k] = r;
            if (!(b >= 1e-14 * amax) || b == 0.0) flag[0] = 1;
        }
        __syncthreads();
        if (flag[0]) return;
        const int p = pivrow;
        if (p != k)
            for (int j = tid; j < n; j += blockDim.x) {
                double t = M[(int64_t)k * n + j];
                M[(int64_t)k * n + j] = M[(int64_t)p * n + j];
                M[(int64_t)p * n + j] = t;
            }
        __syncthreads();
        const double d = M[(int64_t)k * n + k];
        for (int i = k + 1 + tid; i < n; i += blockDim.x) M[(int64_t)i * n + k] = M[(int64_t)i * n + k] / d;
        __syncthreads();
        const int r = n - k - 1;
        for (int64_t q = tid; q < (int64_t)r * r; q += blockDim.x) {
            const int i = k + 1 + (int)(q / r), j = k + 1 + (int)(q % r);
            M[(int64_t)i * n + j] = M[(int64_t)i * n + j] - M[(int64_t)i * n + k] * M[(int64_t)k * n + j];
        }
        __syncthreads();
    }
}

// Coarsest levels of at most kLuSmall rows: densify, LU with partial pivoting
// (largest |pivot|, lowest row on ties; a pivot below 1e-14 max|A| sets
// *flag) and the explicit inverse, in one CTA with the matrix and the inverse
// in shared memory (the global-memory kernels above and below serve larger
// levels).  The same operations per entry as those kernels.
constexpr int kLuSmall = 96;
__global__ void __launch_bounds__(256)
dense_lu_small_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                      const double *__restrict__ val, double *__restrict__ Ainv, int32_t *__restrict__ flag) {
    pdl_wait();
    extern __shared__ __align__(16) double lu_sm[];
    double *M = lu_sm, *X = lu_sm + n * n;
    __shared__ double sv[8];
    __shared__ int si[8];
    __shared__ double amax;
    __shared__ int piv[kLuSmall];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    for (int q = tid; q < n * n; q += blockDim.x) M[q] = 0.0;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x)
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) M[i * n + col[e]] = val[e];
    __syncthreads();
    double m = 0.0;
    for (int q = tid; q < n * n; q += blockDim.x) m = fmax(m, fabs(M[q]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sv[w] = m;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < nw; k++) a = fmax(a, sv[k]);
        amax = a;
    }
    __syncthreads();
    for (int k = 0; k < n; k++) {
        if (w == 0) {  // pivot: one warp scans the column
            double best = -1.0;
            int brow = n;
            for (int i = k + lane; i < n; i += 32) {
                const double v = fabs(M[i * n + k]);
                if (v > best || (v == best && i < brow)) { best = v; brow = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
                if (ov > best || (ov == best && orow < brow)) { best = ov; brow = orow; }
            }
            if (lane == 0) {
                piv[k] = brow;
                if (!(best >= 1e-14 * amax) || best == 0.0) flag[0] = 1;
            }
        }
        __syncthreads();
        if (flag[0]) return;
        const int p = piv[k];
        if (p != k)
            for (int j = tid; j < n; j += blockDim.x) {
                const double t = M[k * n + j];
                M[k * n + j] = M[p * n + j];
                M[p * n + j] = t;
            }
        __syncthreads();
        const double d = M[k * n + k];
        for (int i = k + 1 + tid; i < n; i += blockDim.x) M[i * n + k] = M[i * n + k] / d;
        __syncthreads();
        const int r = n - k - 1;
        for (int q = tid; q < r * r; q += blockDim.x) {
            const int i = k + 1 + q / r, j = k + 1 + q % r;
            M[i * n + j] = M[i * n + j] - M[i * n + k] * M[k * n + j];
        }
        __syncthreads();
    }
    // inverse column c: L U x = P e_c, column c of X held by thread c
    for (int c = tid; c < n; c += blockDim.x) {
        for (int i = 0; i < n; i++) X[i * n + c] = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < n; k++)
            if (piv[k] != k) {
                const double t = X[k * n + c];
                X[k * n + c] = X[piv[k] * n + c];
                X[piv[k] * n + c] = t;
            }
        for (int i = 0; i < n; i++) {
            double s = X[i * n + c];
            for (int j = 0; j < i; j++) s -= M[i * n + j] * X[j * n + c];
            X[i * n + c] = s;
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = X[i * n + c];
            for (int j = i + 1; j < n; j++) s -= M[i * n + j] * X[j * n + c];
            X[i * n + c] = s / M[i * n + i];
        }
    }
    __syncthreads();
    for (int q = tid; q < n * n; q += blockDim.x) Ainv[q] = X[q];
}

// inverse column c: solve L U x = P e_c
__global__ void lu_inverse_kernel(int n, const double *__restrict__ LU, const int32_t *__restrict__ piv,
                                  double *__restrict__ X, double *__restrict__ work) {
    pdl_wait();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double *x = work + (int64_t)c * n;
        for (int i = 0; i < n; i++) x[i] = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < n; k++)
            if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
        for (int i = 0; i < n; i++) {
            double s = x[i];
            for (int j = 0; j < i; j++) s -= LU[(int64_t)i * n + j] * x[j];
            x[i] = s;
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = x[i];
            for (int j = i + 1; j < n; j++) s -= LU[(int64_t)i * n + j] * x[j];
            x[i] = s / LU[(int64_t)i * n + i];
        }
        for (int i = 0; i < n; i++) X[(int64_t)i * n + c] = x[i];
    }
}

// ================================================================== host orchestration
static int rows_grid(int64_t n) { return grid_for(n, kT, 8); }

static int pick_g(double avg) {
    if (avg <= 4.5) return 4;
    if (avg <= 10.0) return 8;
    if (avg <= 20.0) return 16;
    return 32;
}

#define RN_ROWG_LAUNCH(name, bytes, s, G, kern, n, ...)                                                   \
    do {                                                                                                  \
        const int grid_ = std::min(grid_for((n), kT / (G), 8), kReduceBlocks);                            \
        switch (G) {                                                                                      \
            case 4: RN_LAUNCH(name, bytes, s, (kern<4, TV>), grid_, kT, 0, n, __VA_ARGS__); break;        \
            case 8: RN_LAUNCH(name, bytes, s, (kern<8, TV>), grid_, kT, 0, n, __VA_ARGS__); break;        \
            case 16: RN_LAUNCH(name, bytes, s, (kern<16, TV>), grid_, kT, 0, n, __VA_ARGS__); break;      \
            default: RN_LAUNCH(name, bytes, s, (kern<32, TV>), grid_, kT, 0, n, __VA_ARGS__); break;      \
        }                                                                                                 \
    } while (0)

// CG energy minimisation of the values X (in/out, FP64) on pattern N, with
// sweeps in TV: double, or float for the mixed-precision setup (A, X and the
// CG vectors in FP32; the row projection and the scalar recurrences FP64).
// The steps are kept apart (start, direction, product, update, finish) so
// that the setup and the measurement hook (time_setup_op) run the same
// launches.
template <typename TV>
struct CgSweep {
    static constexpr bool f32 = sizeof(TV) == 4;
    const EmCtx &c;
    const CsrView &A;
    const Pattern &N;
    const int32_t *rowtype;
    const double *Bc;
    cudaStream_t s;
    DVec<TV> Rv, Dv, Wv, Xv, Av, Iv, Bcv, Rsv;
    DVec<double> Sv;
    TV *R = nullptr, *Dd = nullptr, *W = nullptr, *X = nullptr;
    const TV *aval = nullptr, *dinv_t = nullptr, *dinv = nullptr;
    double *rs2 = nullptr;
    KProj<TV> kp;
    ProjArgsT<TV> pa{};
    EpPlan<TV> plan;   // the sliced product and the elementwise kernels (when it can be built)
    EpMap em;          // otherwise: the gather map, else the scanning product
    bool vec = false;  // elementwise kernels with 16-byte vector accesses
    Fin fin;
    int G = 4;
    double nzb = 0, rpb = 0, db = 0;
    // independent problems set up together (c.seg): per-problem scalars
    SegCg sg;
    DVec<int32_t> sgi, sgf;
    DVec<double> sgd;
    DVec<unsigned> sgc;
    DVec<TV> sgde;
    const TV *de_s = nullptr;  // D^{-1} per pattern entry

    CgSweep(const EmCtx &c_, const CsrView &A_, const Pattern &N_, double *X64, const int32_t *rowtype_,
            const double *Bc_, const double *c_dinv)
        : c(c_), A(A_), N(N_), rowtype(rowtype_), Bc(Bc_), s(c_.s) {
        if constexpr (f32) {
            Rv.alloc(N.nnz, s); Dv.alloc(N.nnz, s); Wv.alloc(N.nnz, s); Xv.alloc(N.nnz, s);
            R = Rv.p; Dd = Dv.p; W = Wv.p; X = Xv.p;
            to_float(X64, X, N.nnz, s);
        } else {
            R = c.R; Dd = c.Dd; W = c.W; X = X64;
            if (!R) { Rv.alloc(N.nnz, s); R = Rv.p; }
            if (!Dd) { Dv.alloc(N.nnz, s); Dd = Dv.p; }
            if (!W) { Wv.alloc(N.nnz, s); W = Wv.p; }
        }
        fill_i32(c.fl, 0, 1, s);
        rs2 = c.rs2;
        if (!rs2) { Sv.alloc(N.n, s); rs2 = Sv.p; }
        kp.build(c.k, N, rowtype, Bc, s, c.u64, c.zero_row);
        if (c.k == 1) proj_scales(N.n, N.rp, N.col, N.nnz, rowtype, Bc, rs2, s);  // FP64
        else fill_f64(rs2, 0.0, N.n, s);  // products unprojected; the k-projection pass follows each
        pa.rowtype = rowtype;
        if constexpr (f32) {
            Bcv.alloc((size_t)N.nc * c.k, s);
            Rsv.alloc(N.n, s);
            to_float(Bc, Bcv.p, (int64_t)N.nc * c.k, s);
            to_float(rs2, Rsv.p, N.n, s);
            pa.Bc = Bcv.p;
            pa.rs2 = Rsv.p;
        } else {
            pa.Bc = Bc;
            pa.rs2 = rs2;
        }
        G = pick_g(N.n ? (double)N.nnz / N.n : 1.0);
        nzb = (double)sizeof(TV) * N.nnz;
        rpb = 4.0 * (N.n + 1);
        db = (double)sizeof(TV) * N.n;
        fin.partial = c.partial;
        fin.counter = c.counter;
        fin.sc = c.sc;
        fin.fl = c.fl;
        fin.stop = kCgStop;
        // the pattern is fixed for all sweeps: the sliced plan is built once
        // (it holds A's values in TV and D^{-1} per entry); rows of N too long
        // for it fall back to the gather map, then to the scanning product
        if (!c.scan_only)
            ep_plan_build<TV>(plan, A, N.rp, N.col, N.nnz, rowtype, Bc, c.precond ? c_dinv : nullptr, s);
        if (!plan.ok) {
            if constexpr (f32) {
                Av.alloc(A.nnz, s);
                Iv.alloc(N.n, s);
                to_float(A.val, Av.p, A.nnz, s);
                to_float(c_dinv, Iv.p, N.n, s);
                aval = Av.p;
                dinv_t = Iv.p;
            } else {
                aval = A.val;
                dinv_t = c_dinv;
            }
            dinv = c.precond ? dinv_t : nullptr;
            if (!c.scan_only) ep_map_build(em, A, N.rp, N.col, N.nnz, rowtype, s);
        } else {
            auto al = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
            vec = al(X) && al(R) && al(Dd) && al(W) && al(plan.de.p);
        }
        if (c.seg) seg_build(c_dinv);
    }
    // chunks of at most kSegChunk pattern entries, none across two problems
    void seg_build(const double *c_dinv) {
        if (c.k != 1) fail(RN_EINTERNAL, "per-problem energy minimisation needs one candidate");
        const int np = c.seg->np;
        DVec<int32_t> eo((size_t)np + 1, s);
        RN_LAUNCH("energy_seg", 8.0 * (np + 1), s, gather_i32_kernel, grid_for(np + 1, 256), 256, 0, np + 1, N.rp,
                  c.seg->ro_d, eo.p);
        std::vector<int32_t> eoh((size_t)np + 1);
        read_vec(eoh.data(), eo.p, (size_t)np + 1, s);
        std::vector<int32_t> lo, hi, pid, pc((size_t)np + 1, 0);
        for (int p = 0; p < np; p++) {
            pc[p] = (int32_t)lo.size();
            for (int64_t e = eoh[p]; e < eoh[p + 1]; e += kSegChunk) {
                lo.push_back((int32_t)e);
                hi.push_back((int32_t)std::min<int64_t>(e + kSegChunk, eoh[p + 1]));
                pid.push_back(p);
            }
        }
        pc[np] = (int32_t)lo.size();
        const int nch = (int)lo.size();
        std::vector<int32_t> all;
        all.reserve(3 * (size_t)nch + np + 1);
        all.insert(all.end(), lo.begin(), lo.end());
        all.insert(all.end(), hi.begin(), hi.end());
        all.insert(all.end(), pid.begin(), pid.end());
        all.insert(all.end(), pc.begin(), pc.end());
        sgi.alloc(all.size(), s);
        h2d(sgi.p, all.data(), all.size(), s);
        sgd.alloc((size_t)std::max(nch, 1) + 8 * (size_t)np, s);
        fill_f64(sgd.p, 0.0, (int64_t)sgd.n, s);
        sgf.alloc((size_t)np, s);
        fill_i32(sgf.p, 0, np, s);
        sgc.alloc(1, s);
        RN_CUDA_CHECK(cudaMemsetAsync(sgc.p, 0, sizeof(unsigned), s));
        sg.lo = sgi.p;
        sg.hi = sgi.p + nch;
        sg.pid = sgi.p + 2 * nch;
        sg.pc = sgi.p + 3 * nch;
        sg.nch = nch;
        sg.np = np;
        sg.part = sgd.p;
        sg.sc = sgd.p + std::max(nch, 1);
        sg.fl = sgf.p;
        sg.counter = sgc.p;
        sg.stop = kCgStop;
        if (plan.ok) {
            de_s = plan.de.p;
        } else {
            sgde.alloc((size_t)std::max<int64_t>(N.nnz, 1), s);
            RN_LAUNCH("energy_seg", 4.0 * N.n + 8.0 * N.n + (double)sizeof(TV) * N.nnz, s, entry_dinv_kernel<TV>,
                      rows_grid(N.n), kT, 0, N.n, N.rp, c.precond ? c_dinv : nullptr, sgde.p);
            de_s = sgde.p;
        }
    }
    int seg_grid() const { return std::max(1, std::min(sg.nch, 8 * num_sms())); }
    void product(const TV *Xin, TV *Wout, double scale, const TV *Y, const Fin &f) {
        const bool k1 = c.k == 1;
        const Fin none0;
        if (plan.ok)
            masked_product_plan<TV>(plan, N.n, N.rp, N.nnz, Xin, Wout, pa.rs2, k1 ? scale : 1.0, k1 ? Y : nullptr,
                                    k1 ? f : none0, s);
        else if (em.ok)
            masked_product_mapped<TV>(em, A, aval, N.rp, N.col, N.nnz, N.nc, Xin, Wout, pa, k1 ? scale : 1.0,
                                      k1 ? Y : nullptr, k1 ? f : none0, s);
        else
            masked_product_proj<TV>(A, aval, N.rp, N.col, N.nnz, N.nc, Xin, Wout, pa, k1 ? scale : 1.0,
                                    k1 ? Y : nullptr, k1 ? f : none0, s);
        if (!k1) kp.apply(N, rowtype, Wout, scale, Y, f, s);
    }
    int flat_grid(const void *fn) const {
        const int64_t chunks = (N.nnz + 3) / 4;
        int64_t need = (chunks + kT - 1) / kT;
        const int64_t wave = (int64_t)resident_blocks(fn, kT, 0) * num_sms();
        need = std::min<int64_t>(std::min<int64_t>(need, wave), kReduceBlocks);
        return (int)std::max<int64_t>(need, 1);
    }
#define RN_FLAT(name, bytes, kern, ...)                                                                     \
    do {                                                                                                    \
        if (vec) RN_LAUNCH(name, bytes, s, (kern<TV, true>), flat_grid((const void *)kern<TV, true>), kT, 0, \
                           __VA_ARGS__);                                                                    \
        else RN_LAUNCH(name, bytes, s, (kern<TV, false>), flat_grid((const void *)kern<TV, false>), kT, 0,   \
                       __VA_ARGS__);                                                                        \
    } while (0)
    // R = -Proj(Mask_N(A X)) and rho = <R, D^{-1} R>
    void start() {
        const Fin none;
        product(X, R, -1.0, nullptr, none);
        if (c.seg) {
            RN_LAUNCH("energy_cg_rho", 2 * nzb, s, seg_rho_kernel<TV>, seg_grid(), kT, 0, sg, R, de_s, 0);
            return;
        }
        fin.mode = FIN_CG_RHO;
        fin.it = 0;
        if (plan.ok) RN_FLAT("energy_cg_rho", 2 * nzb, cg_rho_flat_kernel, N.nnz, R, plan.de.p, fin);
        else RN_ROWG_LAUNCH("energy_cg_rho", rpb + nzb + db, s, G, cg_rho_kernel, N.n, N.rp, R, dinv, fin);
    }
    // Dd = D^{-1} R (+ beta Dd after the first sweep)
    void direction(int it) {
        if (c.seg)
            RN_LAUNCH("energy_cg_direction", (it == 0 ? 3 : 4) * nzb, s, seg_dd_kernel<TV>, seg_grid(), kT, 0, sg, R,
                      de_s, it == 0 ? 1 : 0, Dd);
        else if (plan.ok)
            RN_FLAT("energy_cg_direction", (it == 0 ? 3 : 4) * nzb, cg_dd_flat_kernel, N.nnz, R, plan.de.p, c.sc,
                    c.fl, it == 0 ? 1 : 0, Dd);
        else
            RN_ROWG_LAUNCH("energy_cg_direction", rpb + 3 * nzb + db, s, G, cg_dd_kernel, N.n, N.rp, R, dinv, c.sc,
                           c.fl, it == 0 ? 1 : 0, Dd);
    }
    // W = Proj(Mask_N(A Dd)), <Dd, W> and alpha
    void sweep_product() {
        if (c.seg) {  // the product unreduced, then <Dd, W> per problem
            product(Dd, W, 1.0, nullptr, Fin());
            RN_LAUNCH("energy_cg_dw", 2 * nzb, s, seg_dw_kernel<TV>, seg_grid(), kT, 0, sg, Dd, W);
            return;
        }
        fin.mode = FIN_CG_DW;
        product(Dd, W, 1.0, Dd, fin);
    }
    // X += alpha Dd, R -= alpha W, rho and beta
    void update(int it) {
        if (c.seg) {
            RN_LAUNCH("energy_cg_update", 7 * nzb, s, seg_update_kernel<TV>, seg_grid(), kT, 0, sg, X, R, Dd, W, de_s,
                      it + 1);
            return;
        }
        fin.mode = FIN_CG_RHO;
        fin.it = it + 1;
        if (plan.ok)
            RN_FLAT("energy_cg_update", 7 * nzb, cg_update_flat_kernel, N.nnz, X, R, Dd, W, plan.de.p, c.sc, c.fl,
                    fin);
        else
            RN_ROWG_LAUNCH("energy_cg_update", rpb + 6 * nzb + db, s, G, cg_update_kernel, N.n, N.rp, X, R, Dd, W,
                           dinv, c.sc, c.fl, fin);
    }
#undef RN_FLAT
    void sweep(int it) {
        direction(it);
        sweep_product();
        update(it);
    }
    void finish(double *X64) {
        if constexpr (f32) to_double(X, X64, N.nnz, s);
        else (void)X64;
    }
    // algorithmic bytes of one sweep: A once, the pattern once, eight passes
    // over the pattern's values (Dd read for the product and written by the
    // direction, W written and read, X and R read and written), D^{-1} and Bc
    double sweep_bytes() const {
        const double vb = sizeof(TV);
        return (4.0 + vb) * A.nnz + 4.0 * N.nnz + 8.0 * vb * N.nnz + vb * N.n + vb * c.k * N.nc;
    }
};

template <typename TV>
static void energy_min_cg_t(const EmCtx &c, const CsrView &A, const Pattern &N, double *X64,
                            const int32_t *rowtype, const double *Bc, const double *c_dinv, int sweeps) {
    CgSweep<TV> cg(c, A, N, X64, rowtype, Bc, c_dinv);
    cg.start();
    for (int it = 0; it < sweeps; it++) cg.sweep(it);
    cg.finish(X64);
}

void energy_min_cg(const EmCtx &c, const CsrView &A, const Pattern &N, double *X, const int32_t *rowtype,
                   const double *Bc, const double *c_dinv, int sweeps) {
    if (c.fp32) energy_min_cg_t<float>(c, A, N, X, rowtype, Bc, c_dinv, sweeps);
    else energy_min_cg_t<double>(c, A, N, X, rowtype, Bc, c_dinv, sweeps);
}

// GMRES energy minimisation (m Arnoldi steps, modified Gram-Schmidt), sweeps
// in TV (double; float in mixed precision: A, the basis and the projection's
// scales in FP32, the Hessenberg matrix, rotations and dot products FP64).
template <typename TV>
static void energy_min_gmres_t(const EmCtx &c, const CsrView &A, const Pattern &N, double *X64,
                               const int32_t *rowtype, const double *Bc, int m) {
    if (m <= 0) return;
    constexpr bool f32 = sizeof(TV) == 4;
    cudaStream_t s = c.s;
    const int64_t nz = N.nnz;
    DVec<TV> V((size_t)(m + 1) * (nz > 0 ? nz : 1), s), W(nz > 0 ? nz : 1, s), Xv, Av, Bcv, Rsv;
    DVec<double> Hm((size_t)(m + 1) * m + 4 * (m + 1), s);
    fill_f64(Hm.p, 0.0, (int64_t)Hm.n, s);
    double *H = Hm.p, *cs = H + (m + 1) * m, *sn = cs + (m + 1), *g = sn + (m + 1), *y = g + (m + 1);
    double *sc = c.sc;
    int32_t *fl = c.fl;
    DVec<double> Sv(c.rs2 ? 0 : N.n, s);
    double *rs2 = c.rs2 ? c.rs2 : Sv.p;
    KProj<TV> kp;
    kp.build(c.k, N, rowtype, Bc, s, c.u64, c.zero_row);
    if (c.k == 1) proj_scales(N.n, N.rp, N.col, N.nnz, rowtype, Bc, rs2, s);
    else fill_f64(rs2, 0.0, N.n, s);  // products unprojected; the k-projection pass follows each
    ProjArgsT<TV> pa{rowtype, nullptr, nullptr};
    TV *X;
    const TV *aval = nullptr;
    // the sliced plan holds A's values in TV; without it, A is converted
    EpPlan<TV> plan;
    if (!c.scan_only) ep_plan_build<TV>(plan, A, N.rp, N.col, N.nnz, rowtype, Bc, nullptr, s);
    if constexpr (f32) {
        Xv.alloc(nz > 0 ? nz : 1, s);
        Bcv.alloc((size_t)N.nc * c.k, s);
        Rsv.alloc(N.n, s);
        to_float(X64, Xv.p, nz, s);
        if (!plan.ok) {
            Av.alloc(A.nnz, s);
            to_float(A.val, Av.p, A.nnz, s);
            aval = Av.p;
        }
        to_float(Bc, Bcv.p, (int64_t)N.nc * c.k, s);
        to_float(rs2, Rsv.p, N.n, s);
        X = Xv.p;
        pa.Bc = Bcv.p;
        pa.rs2 = Rsv.p;
    } else {
        X = X64;
        aval = A.val;
        pa.Bc = Bc;
        pa.rs2 = rs2;
    }
    const int eg = grid_for(nz, 1024);
    const double nzb = (double)sizeof(TV) * nz;
    EpMap em;
    if (!plan.ok && !c.scan_only) ep_map_build(em, A, N.rp, N.col, N.nnz, rowtype, s);
    auto product = [&](const TV *Xin, TV *Wout, double scale) {
        const double sc0 = c.k == 1 ? scale : 1.0;
        if (plan.ok)
            masked_product_plan<TV>(plan, N.n, N.rp, N.nnz, Xin, Wout, pa.rs2, sc0, nullptr, Fin(), s);
        else if (em.ok)
            masked_product_mapped<TV>(em, A, aval, N.rp, N.col, N.nnz, N.nc, Xin, Wout, pa, sc0, nullptr, Fin(), s);
        else masked_product_proj<TV>(A, aval, N.rp, N.col, N.nnz, N.nc, Xin, Wout, pa, sc0, nullptr, Fin(), s);
        if (c.k > 1) kp.apply(N, rowtype, Wout, scale, nullptr, Fin(), s);
    };
    auto dot_t = [&](const TV *a, const TV *b, double *out) {
        Fin f;
        f.mode = FIN_STORE;
        f.partial = c.partial;
        f.counter = c.counter;
        f.out = out;
        RN_LAUNCH("energy_gmres_dot", 2 * nzb, s, gm_dot_kernel<TV>,
                  grid_resident(gm_dot_kernel<TV>, kT, 0, nz, kT * 4, kReduceBlocks), kT, 0, nz, a, b, f);
    };
    product(X, V.p, -1.0);
    dot_t(V.p, V.p, sc + 1);
    RN_LAUNCH("energy_gmres_scalar", 0, s, gm_start_kernel, 1, 1, 0, sc, fl, g);
    RN_LAUNCH("energy_gmres_vec", 2 * nzb, s, gm_scale_kernel<TV>, eg, 256, 0, nz, V.p, sc, fl);
    for (int j = 0; j < m; j++) {
        TV *vj = V.p + (int64_t)j * nz;
        product(vj, W.p, 1.0);
        for (int i = 0; i <= j; i++) {
            TV *vi = V.p + (int64_t)i * nz;
            dot_t(W.p, vi, H + i * m + j);
            RN_LAUNCH("energy_gmres_vec", 3 * nzb, s, gm_axpy_kernel<TV>, eg, 256, 0, nz, W.p, vi, H + i * m + j,
                      fl);
        }
        dot_t(W.p, W.p, sc + 1);
        RN_LAUNCH("energy_gmres_scalar", 0, s, gm_givens_kernel, 1, 1, 0, m, j, H, cs, sn, g, sc, fl, kGmresBreak);
        if (j + 1 < m + 1) {
            d2d(V.p + (int64_t)(j + 1) * nz, W.p, nz, s);
            RN_LAUNCH("energy_gmres_vec", 2 * nzb, s, gm_scale_kernel<TV>, eg, 256, 0, nz,
                      V.p + (int64_t)(j + 1) * nz, sc + 2, fl);
        }
    }
    RN_LAUNCH("energy_gmres_scalar", 0, s, gm_backsolve_kernel, 1, 1, 0, m, H, g, y, fl);
    RN_LAUNCH("energy_gmres_vec", (m + 2) * nzb, s, gm_combine_kernel<TV>, eg, 256, 0, nz, m, X, V.p, y, fl);
    if constexpr (f32) to_double(X, X64, nz, s);
}

void energy_min_gmres(const EmCtx &c, const CsrView &A, const Pattern &N, double *X, const int32_t *rowtype,
                      const double *Bc, int m) {
    if (c.fp32) energy_min_gmres_t<float>(c, A, N, X, rowtype, Bc, m);
    else energy_min_gmres_t<double>(c, A, N, X, rowtype, Bc, m);
}

void energy_min(const EmCtx &c, const CsrView &A, const Pattern &N, double *X, const int32_t *rowtype,
                const double *Bc, const double *dinv, int sweeps) {
    if (c.method == RN_ENERGY_GMRES) energy_min_gmres(c, A, N, X, rowtype, Bc, sweeps);
    else energy_min_cg(c, A, N, X, rowtype, Bc, dinv, sweeps);
}

static const SegRows *seg_of(const rn_hierarchy &h);

static EmCtx ctx_of(rn_hierarchy &h) {
    EmCtx c;
    c.s = h.s;
    c.partial = h.partial.p;
    c.counter = h.counters.p;
    c.sc = h.scal.p;
    c.fl = h.iflags.p;
    c.precond = h.p.energy_precond;
    c.method = h.p.energy_method;
    // FP32 sweeps (CG and GMRES) in the mixed-precision setup when k = 1; with
    // k > 1 candidates the row projection multiplies rounding by the
    // conditioning of each row's fit, so the sweeps stay FP64
    c.fp32 = h.p.precision == RN_MIXED && h.k == 1;
    c.k = h.k;
    c.seg = seg_of(h);
    return c;
}

static void coarsest_lu(rn_hierarchy &h, bool check = true);
static void coarsest_lu_check(rn_hierarchy &h);

// ================================================================== independent problems set up together
// The problems' level-l operators form one block-diagonal matrix (problem t of
// the active list owns rows [ro[t], ro[t + 1]) and the same columns), so every
// step of Alg. 3 runs once for all of them: strength, transfer patterns,
// energy minimisation, R and the Galerkin product never couple two blocks.
// What is per problem: the aggregation priorities (each node's index within
// its problem), the energy CG's step lengths (SegRows), and the end of
// coarsening; a problem whose level is its coarsest leaves the merged matrix,
// and every level is split into the problems' own hierarchies as it is
// finished.

// One block of a CSR copy: source rows [r0, r0 + nr) (entries [e0, e0 + ne))
// to destination rows from dr (entries from de), columns shifted by dc.
struct BlockCsr {
    int32_t r0, nr, e0, ne, dr, de, dc;
    int32_t *rp, *col;
    double *val;
    const int32_t *srp = nullptr, *scol = nullptr;  // source (filled from the copied matrix when null)
    const double *sval = nullptr;
};
__global__ void block_csr_kernel(const BlockCsr *__restrict__ blk) {
    pdl_wait();
    const BlockCsr b = blk[blockIdx.y];
    const int32_t t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    for (int32_t i = t0; i <= b.nr; i += st) b.rp[b.dr + i] = b.srp[b.r0 + i] - b.e0 + b.de;
    for (int32_t e = t0; e < b.ne; e += st) {
        b.col[b.de + e] = b.scol[b.e0 + e] + b.dc;
        b.val[b.de + e] = b.sval[b.e0 + e];
    }
}
// One block of a vector copy; with shift, values >= 0 get delta added (indices)
template <typename T>
struct BlockVec {
    int32_t s0, n, d0;
    T delta;
    T *dst;
};
template <typename T>
__global__ void block_vec_kernel(const BlockVec<T> *__restrict__ blk, const T *__restrict__ src, int shift) {
    pdl_wait();
    const BlockVec<T> b = blk[blockIdx.y];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        T v = src[b.s0 + i];
        if (shift && v >= T(0)) v += b.delta;
        b.dst[b.d0 + i] = v;
    }
}
// every row's problem offset: roff[i] = ro[t] for ro[t] <= i < ro[t + 1]
__global__ void row_offset_kernel(int32_t n, int np, const int32_t *__restrict__ ro, int32_t *__restrict__ roff) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = np - 1;
        while (lo < hi) {  // last t with ro[t] <= i
            const int mid = (lo + hi + 1) >> 1;
            if (ro[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        roff[i] = ro[lo];
    }
}

struct MergedSetup {
    std::vector<rn_hierarchy *> out;  // problem p's hierarchy
    std::vector<int> act;             // active problems, in merged order
    SegRows seg;                      // their row offsets at the current level
    DVec<int32_t> ro_d, roff;         // device: row offsets, every row's problem offset
    std::vector<int32_t> co;          // coarse row offsets (after aggregation)
    DVec<int32_t> co_d;
    std::vector<cudaEvent_t> ev;      // per problem: its stream's allocations are done
    cudaStream_t s = nullptr;

    ~MergedSetup() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    int np() const { return (int)act.size(); }
    void set_rows(std::vector<int32_t> ro, int32_t n) {
        seg.np = np();
        seg.ro = std::move(ro);
        ro_d.alloc(seg.ro.size(), s);
        h2d(ro_d.p, seg.ro.data(), seg.ro.size(), s);
        seg.ro_d = ro_d.p;
        roff.alloc(std::max<int32_t>(n, 1), s);
        RN_LAUNCH("merge_setup", 4.0 * n, s, row_offset_kernel, rows_grid(n), kT, 0, n, np(), ro_d.p, roff.p);
    }
    // values of a row-pointer array at the given block boundaries (one read)
    std::vector<int32_t> bounds(const int32_t *rp, const int32_t *rows_d, size_t m) {
        DVec<int32_t> g(m, s);
        RN_LAUNCH("merge_setup", 8.0 * m, s, gather_i32_kernel, grid_for((int64_t)m, 256), 256, 0, (int32_t)m, rp,
                  rows_d, g.p);
        std::vector<int32_t> v(m);
        read_vec(v.data(), g.p, m, s);
        return v;
    }
    // problem p's buffers come from its hierarchy's pool (or the caller's hooks)
    Allocator alloc_for(int p) const {
        Allocator a = current_allocator();
        a.pool = out[p]->pool;
        return a;
    }
    rn_level &level_of(int p, int l) {
        auto &lev = out[p]->lev;
        while ((int)lev.size() <= l) lev.push_back(std::make_unique<rn_level>());
        return *lev[l];
    }
    // the merged stream waits for every listed problem's allocations
    void wait_allocs(const std::vector<int> &ps) {
        for (int p : ps) {
            RN_CUDA_CHECK(cudaEventRecord(ev[p], out[p]->s));
            RN_CUDA_CHECK(cudaStreamWaitEvent(s, ev[p], 0));
        }
    }
    void launch_csr(std::vector<BlockCsr> b, const CsrView &M) {
        if (b.empty()) return;
        int32_t most = 1;
        for (BlockCsr &x : b) {
            most = std::max(most, std::max(x.nr + 1, x.ne));
            if (!x.srp) {
                x.srp = M.rowptr;
                x.scol = M.col;
                x.sval = M.val;
            }
        }
        DVec<BlockCsr> d(b.size(), s);
        h2d(d.p, b.data(), b.size(), s);
        const dim3 grid((unsigned)std::min<int64_t>((most + 255) / 256, 2048), (unsigned)b.size());
        RN_LAUNCH("merge_setup", 12.0 * M.nnz, s, block_csr_kernel, grid, 256, 0, d.p);
    }
    template <typename T>
    void launch_vec(const std::vector<BlockVec<T>> &b, const T *src, int shift) {
        if (b.empty()) return;
        int32_t most = 1;
        for (const BlockVec<T> &x : b) most = std::max(most, x.n);
        DVec<BlockVec<T>> d(b.size(), s);
        h2d(d.p, b.data(), b.size(), s);
        const dim3 grid((unsigned)std::min<int64_t>((most + 255) / 256, 2048), (unsigned)b.size());
        RN_LAUNCH("merge_setup", 0.0, s, block_vec_kernel<T>, grid, 256, 0, d.p, src, shift);
    }
    // problem blocks (merged index t) of a CSR with rows at rof and columns at cof,
    // each into level l of its problem's hierarchy (field f)
    void split_csr(const DCsr &M, const std::vector<int32_t> &rof, const int32_t *rof_d,
                   const std::vector<int32_t> &cof, const std::vector<int> &ts, int l, DCsr rn_level::*f,
                   std::vector<BlockCsr> &blk) {
        const std::vector<int32_t> eb = bounds(M.rowptr.p, rof_d, rof.size());
        for (int t : ts) {
            const int p = act[t];
            DCsr &X = level_of(p, l).*f;
            cudaStream_t ps = out[p]->s;
            const AllocScope scope(alloc_for(p));
            X.n = rof[t + 1] - rof[t];
            X.m = cof[t + 1] - cof[t];
            X.nnz = eb[t + 1] - eb[t];
            X.rowptr.alloc((size_t)X.n + 1, ps);
            X.col.alloc((size_t)X.nnz, ps);
            X.val.alloc((size_t)X.nnz, ps);
            blk.push_back(BlockCsr{rof[t], X.n, eb[t], (int32_t)X.nnz, 0, 0, -cof[t], X.rowptr.p, X.col.p, X.val.p});
        }
    }
    template <typename T>
    void split_vec(const std::vector<int32_t> &rof, const std::vector<int32_t> &dof, const std::vector<int> &ts,
                   int l, DVec<T> rn_level::*f, std::vector<BlockVec<T>> &blk) {
        for (int t : ts) {
            const int p = act[t];
            DVec<T> &X = level_of(p, l).*f;
            const int32_t n = rof[t + 1] - rof[t];
            const AllocScope scope(alloc_for(p));
            X.alloc((size_t)n, out[p]->s);
            blk.push_back(BlockVec<T>{rof[t], n, 0, (T)(dof.empty() ? 0 : -dof[t]), X.p});
        }
    }
    // level l is the coarsest of the listed problems: A, diag, B
    void split_coarsest(rn_level &L, const std::vector<int> &ts, int l) {
        if (ts.empty()) return;
        const std::vector<int32_t> &ro = seg.ro;
        std::vector<BlockCsr> ba;
        std::vector<BlockVec<double>> bd, bb;
        split_csr(L.A, ro, ro_d.p, ro, ts, l, &rn_level::A, ba);
        split_vec(ro, {}, ts, l, &rn_level::diag, bd);
        split_vec(ro, {}, ts, l, &rn_level::B, bb);
        std::vector<int> ps;
        for (int t : ts) ps.push_back(act[t]);
        wait_allocs(ps);
        launch_csr(ba, view(L.A));
        launch_vec(bd, L.diag.p, 0);
        launch_vec(bb, L.B.p, 0);
    }
    // keep only the listed problems in the merged level (A, B; diag is recomputed by the caller)
    void keep_only(rn_level &L, const std::vector<int> &ts) {
        const std::vector<int32_t> &ro = seg.ro;
        const std::vector<int32_t> eb = bounds(L.A.rowptr.p, ro_d.p, ro.size());
        std::vector<int32_t> nro(1, 0);
        int64_t nnz = 0;
        for (int t : ts) {
            nro.push_back(nro.back() + (ro[t + 1] - ro[t]));
            nnz += eb[t + 1] - eb[t];
        }
        const int32_t n = nro.back();
        DCsr A;
        A.n = A.m = n;
        A.nnz = nnz;
        A.rowptr.alloc((size_t)n + 1, s);
        A.col.alloc((size_t)nnz, s);
        A.val.alloc((size_t)nnz, s);
        DVec<double> B((size_t)n, s);
        std::vector<BlockCsr> ba;
        std::vector<BlockVec<double>> bb;
        int32_t de = 0;
        for (size_t u = 0; u < ts.size(); u++) {
            const int t = ts[u];
            const int32_t ne = eb[t + 1] - eb[t];
            ba.push_back(BlockCsr{ro[t], ro[t + 1] - ro[t], eb[t], ne, nro[u], de, nro[u] - ro[t], A.rowptr.p,
                                  A.col.p, A.val.p});
            bb.push_back(BlockVec<double>{ro[t], ro[t + 1] - ro[t], nro[u], 0.0, B.p});
            de += ne;
        }
        launch_csr(ba, view(L.A));
        launch_vec(bb, L.B.p, 0);
        std::vector<int> nact;
        for (int t : ts) nact.push_back(act[t]);
        act = std::move(nact);
        L.A = std::move(A);
        L.B = std::move(B);
        set_rows(std::move(nro), n);
    }
    std::vector<int> all_but(const std::vector<int> &ts) const {
        std::vector<char> drop((size_t)np(), 0);
        for (int t : ts) drop[t] = 1;
        std::vector<int> keep;
        for (int t = 0; t < np(); t++)
            if (!drop[t]) keep.push_back(t);
        return keep;
    }
    // hook after the level's diagonal: problems small enough (or at the level
    // limit) end here.  Returns true when no problem is left.
    bool end_small(rn_hierarchy &W, int l, int maxlev) {
        rn_level &L = *W.lev[l];
        std::vector<int> ending;
        for (int t = 0; t < np(); t++)
            if (seg.ro[t + 1] - seg.ro[t] <= W.p.max_coarse || l >= maxlev - 1) ending.push_back(t);
        if (ending.empty()) return false;
        split_coarsest(L, ending, l);
        if ((int)ending.size() == np()) return true;
        keep_only(L, all_but(ending));
        L.diag.alloc((size_t)L.A.n, s);
        fill_i32(W.iflags.p + 4, 0, 1, s);
        extract_diag(view(L.A), L.diag.p, W.iflags.p + 4, s);
        return false;
    }
    // hook after aggregation: problems whose coarsening stalled (no aggregate,
    // or as many aggregates as nodes) end at this level.  Returns 0 (go on:
    // co holds the coarse offsets), 1 (redo the level without them) or 2 (no
    // problem left).
    int stalled(rn_hierarchy &W, int l, const int32_t *cidx) {
        rn_level &L = *W.lev[l];
        const std::vector<int32_t> cb = bounds(cidx, ro_d.p, seg.ro.size());
        std::vector<int> st;
        for (int t = 0; t < np(); t++) {
            const int32_t nct = cb[t + 1] - cb[t];
            if (nct == 0 || nct >= seg.ro[t + 1] - seg.ro[t]) st.push_back(t);
        }
        if (st.empty()) {
            co.assign(cb.begin(), cb.end());
            for (auto &v : co) v -= cb[0];
            co_d.alloc(co.size(), s);
            h2d(co_d.p, co.data(), co.size(), s);
            return 0;
        }
        split_coarsest(L, st, l);
        if ((int)st.size() == np()) return 2;
        keep_only(L, all_but(st));
        return 1;
    }
    // hook after the Galerkin product: level l of every active problem (A,
    // diag, B, rowtype, Bc, P, R, and with keep_aux S, N, T, roots, agg); the
    // next level's rows are the coarse offsets
    void split_level(rn_hierarchy &W, int l) {
        rn_level &L = *W.lev[l];
        rn_level &Lc = *W.lev[l + 1];
        const std::vector<int32_t> &ro = seg.ro;
        std::vector<int> ts(np());
        for (int t = 0; t < np(); t++) ts[t] = t;
        std::vector<BlockCsr> ba, bp, br, bs, bn, bt;
        std::vector<BlockVec<double>> bd, bb, bc;
        std::vector<BlockVec<int32_t>> brt, bro, bag;
        split_csr(L.A, ro, ro_d.p, ro, ts, l, &rn_level::A, ba);
        split_csr(L.P, ro, ro_d.p, co, ts, l, &rn_level::P, bp);
        split_csr(L.R, co, co_d.p, ro, ts, l, &rn_level::R, br);
        split_vec(ro, {}, ts, l, &rn_level::diag, bd);
        split_vec(ro, {}, ts, l, &rn_level::B, bb);
        split_vec(co, {}, ts, l, &rn_level::Bc, bc);
        split_vec(ro, {}, ts, l, &rn_level::rowtype, brt);
        const bool aux = W.p.keep_aux != 0;
        if (aux) {
            split_csr(L.S, ro, ro_d.p, ro, ts, l, &rn_level::S, bs);
            split_csr(L.N, ro, ro_d.p, co, ts, l, &rn_level::N, bn);
            split_csr(L.T, ro, ro_d.p, co, ts, l, &rn_level::T, bt);
            split_vec(co, ro, ts, l, &rn_level::roots, bro);
            split_vec(ro, co, ts, l, &rn_level::agg, bag);
        }
        for (int t : ts) level_of(act[t], l).nc = co[t + 1] - co[t];
        wait_allocs(act);
        launch_csr(ba, view(L.A));
        launch_csr(bp, view(L.P));
        launch_csr(br, view(L.R));
        launch_vec(bd, L.diag.p, 0);
        launch_vec(bb, L.B.p, 0);
        launch_vec(bc, L.Bc.p, 0);
        launch_vec(brt, L.rowtype.p, 0);
        if (aux) {
            launch_csr(bs, view(L.S));
            launch_csr(bn, view(L.N));
            launch_csr(bt, view(L.T));
            launch_vec(bro, L.roots.p, 1);
            launch_vec(bag, L.agg.p, 1);
        }
        // the merged level is no longer needed once its copies have run (stream order)
        W.lev[l] = std::make_unique<rn_level>();
        set_rows(co, Lc.A.n);
    }
};

static const SegRows *seg_of(const rn_hierarchy &h) { return h.merged ? &h.merged->seg : nullptr; }

// A scan whose total comes back in the same read as the level's flags
// (iflags[0..16), the total in iflags[14..15]), so checks deferred to it cost
// no synchronisation of their own
static int64_t scan_with_flags(rn_hierarchy &h, const int32_t *counts, int32_t *out, int64_t n, int32_t (&fl)[16]) {
    scan_counts_dev(counts, out, n, reinterpret_cast<int64_t *>(h.iflags.p + 14), h.s);
    read_small(fl, h.iflags.p, 16, h.s);
    int64_t t;
    std::memcpy(&t, fl + 14, sizeof t);
    if (t > INT32_MAX) fail(RN_EINTERNAL, fmt("scan total %lld exceeds int32", (long long)t));
    return t;
}

static void check_flag(const int32_t *flag, cudaStream_t s, rn_status st, const char *what) {
    int32_t v = read_scalar(flag, s);
    if (v) fail(st, fmt("%s (index %d)", what, v - 1));
}

// Smooth candidates, build P (or R^T) on pattern N: Alg. 3 inject / improve /
// filter / enforce / improve.  Pout receives the final pattern and values.
// b_sweeps weighted-Jacobi sweeps on A B = 0 (exact) from B (read only),
// alternating between buf0 and buf1 on stream s; returns the buffer holding
// the smoothed candidates (B itself without sweeps)
static const double *smooth_candidates(const rn_hierarchy &h, const CsrView &A, const double *B, double *buf0,
                                       double *buf1, cudaStream_t s) {
    const int32_t n = A.n;
    const int k = h.k;
    const double *src = B;
    double *dst = buf0;
    for (int sw = 0; sw < h.p.b_sweeps; sw++) {
        if (k == 1)
            RN_LAUNCH("candidates", 12.0 * A.nnz + 24.0 * n, s, cand_jacobi_kernel, rows_grid(n), kT, 0, n, A.rowptr,
                      A.col, A.val, src, h.p.omega, dst);
        else
            RN_LAUNCH("candidates", 12.0 * A.nnz + 8.0 * k * (A.nnz + 2.0 * n), s, cand_jacobi_k_kernel, rows_grid(n),
                      kT, 0, n, k, A.rowptr, A.col, A.val, src, h.p.omega, dst);
        src = dst;
        dst = (dst == buf0) ? buf1 : buf0;
    }
    return src;
}

// This thread's side stream and fork/join events (kept for the thread's life):
// work of a level that needs only its operator (the candidate smoothing) runs
// there while the main stream aggregates, filling the main stream's gaps
// between its host synchronisations.  Nothing is allocated on it.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
static SideStream &side_stream() {
    thread_local SideStream ss;
    if (!ss.s) {
        RN_CUDA_CHECK(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
        RN_CUDA_CHECK(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
        RN_CUDA_CHECK(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming));
    }
    return ss;
}

// smoothed: Bsm already holds the smoothed candidates
static void build_transfer(rn_hierarchy &h, const CsrView &A, const DCsr &N, const int32_t *agg,
                           const int32_t *roots, int32_t nc, const int32_t *rowtype, double *Bsm, const double *diag,
                           double *Bc, DCsr &Pout, DCsr *Tkeep, bool smoothed = false) {
    cudaStream_t s = h.s;
    const int32_t n = A.n;
    const int k = h.k;
    // candidates (unless the caller smoothed them)
    if (!smoothed && h.p.b_sweeps > 0) {
        DVec<double> t0((size_t)n * k, s), t1((size_t)n * k, s);
        d2d(Bsm, smooth_candidates(h, A, Bsm, t0.p, t1.p, s), (size_t)n * k, s);
    }
    fill_i32(h.iflags.p + 2, 0, 1, s);
    if (k == 1)
        RN_LAUNCH("inject", 16.0 * nc, s, gather_kernel, rows_grid(nc), kT, 0, nc, roots, Bsm, Bc, h.iflags.p + 2);
    else
        RN_LAUNCH("inject", 16.0 * nc * k, s, gather_k_kernel, rows_grid(nc), kT, 0, nc, k, roots, Bsm, Bc,
                  h.iflags.p + 2);
    DVec<double> binv;
    if (h.mb > 1) {  // systems: the root node's m x m block of the first m candidates must be invertible
        fill_i32(h.iflags.p + 2, 0, 1, s);
        binv.alloc((size_t)nc * h.mb, s);  // (nc / m) blocks of m x m
        RN_LAUNCH("inject", 8.0 * nc * h.mb * 2, s, root_block_inverse_kernel, rows_grid(nc / h.mb), kT, 0,
                  nc / h.mb, h.mb, k, roots, Bsm, binv.p, h.iflags.p + 2);
        check_flag(h.iflags.p + 2, s, RN_EINVAL, "candidate block singular at a root node");
    } else {
        check_flag(h.iflags.p + 2, s, RN_EINVAL, "candidate vanishes at a root node");
    }
    // P = T on N
    Pout.n = n;
    Pout.m = nc;
    Pout.nnz = N.nnz;
    Pout.rowptr.alloc(n + 1, s);
    Pout.col.alloc(N.nnz, s);
    Pout.val.alloc(N.nnz, s);
    d2d(Pout.rowptr.p, N.rowptr.p, n + 1, s);
    d2d(Pout.col.p, N.col.p, N.nnz, s);
    if (h.mb > 1)
        RN_LAUNCH("tentative", 16.0 * N.nnz + 8.0 * k * n, s, tentative_block_kernel, rows_grid(n), kT, 0, n, h.mb,
                  k, N.rowptr.p, N.col.p, agg, rowtype, Bsm, binv.p, Pout.val.p);
    else
        RN_LAUNCH("tentative", 16.0 * N.nnz + 16.0 * n, s, tentative_kernel, rows_grid(n), kT, 0, n, N.rowptr.p,
                  N.col.p, agg, Bsm, Bc, Pout.val.p, k);
    // k > 1: every row's SVD of Bc_J on N, formed once for the row fits and the minimisation's projection
    DVec<double> uN, vsN;
    DVec<int32_t> zrN;
    if (k > 1) {
        uN.alloc((size_t)std::max<int64_t>(N.nnz, 1) * k, s);
        vsN.alloc((size_t)n * k * k, s);
        zrN.alloc(n, s);
        RN_K_SWITCH(k, RN_LAUNCH("energy_proj_scale", 4.0 * N.nnz + 16.0 * k * N.nnz + 8.0 * k * k * n, s,
                                 row_svd_kernel<KK>, rows_grid(n), kT, 0, n, N.rowptr.p, N.col.p, rowtype, Bc, uN.p,
                                 vsN.p, zrN.p));
    }
    if (k > h.mb)  // the other candidates: minimal-norm row fits (eq. Tproj)
        RN_K_SWITCH(k, RN_LAUNCH("tentative", 12.0 * N.nnz + 8.0 * k * (2.0 * N.nnz + n) + 8.0 * k * k * n, s,
                                 row_fit_u_kernel<KK>, rows_grid(n), kT, 0, n, Pout.rowptr.p, Pout.col.p, Pout.val.p,
                                 rowtype, Bsm, Bc, uN.p, vsN.p));
    if (Tkeep) {
        Tkeep->n = n; Tkeep->m = nc; Tkeep->nnz = N.nnz;
        Tkeep->rowptr.alloc(n + 1, s); Tkeep->col.alloc(N.nnz, s); Tkeep->val.alloc(N.nnz, s);
        d2d(Tkeep->rowptr.p, N.rowptr.p, n + 1, s);
        d2d(Tkeep->col.p, N.col.p, N.nnz, s);
        d2d(Tkeep->val.p, Pout.val.p, N.nnz, s);
    }
    Pattern pat{n, nc, N.nnz, Pout.rowptr.p, Pout.col.p};
    DVec<double> dinv(n, s);  // the energy CG's preconditioner D^{-1}
    reciprocal(diag, dinv.p, n, s);
    {
        EmCtx c = ctx_of(h);
        c.u64 = uN.p;  // the same pattern and Bc
        c.zero_row = zrN.p;
        energy_min(c, A, pat, Pout.val.p, rowtype, Bc, dinv.p, h.p.n_sweeps);
    }
    if (h.p.postfilter > 0.0) {
        const double omg = 1.0 - kGuard;
        DVec<int32_t> cnt(n + 1, s);
        RN_LAUNCH("postfilter", 24.0 * Pout.nnz, s, postfilter_kernel<false>, rows_grid(n), kT, 0, n, Pout.rowptr.p,
                  Pout.col.p, Pout.val.p, rowtype, agg, h.p.postfilter, omg, cnt.p, nullptr, nullptr, nullptr, h.mb);
        DCsr F;
        F.n = n; F.m = nc;
        F.rowptr.alloc(n + 1, s);
        F.nnz = scan_counts(cnt.p, F.rowptr.p, n, s);
        F.col.alloc(F.nnz, s);
        F.val.alloc(F.nnz, s);
        RN_LAUNCH("postfilter", 24.0 * Pout.nnz + 12.0 * F.nnz, s, postfilter_kernel<true>, rows_grid(n), kT, 0, n,
                  Pout.rowptr.p, Pout.col.p, Pout.val.p, rowtype, agg, h.p.postfilter, omg, nullptr, F.rowptr.p,
                  F.col.p, F.val.p, h.mb);
        if (k == 1)
            RN_LAUNCH("enforce", 28.0 * F.nnz + 8.0 * n, s, enforce_kernel, rows_grid(n), kT, 0, n, F.rowptr.p,
                      F.col.p, F.val.p, rowtype, Bsm, Bc);
        else {  // the fit on the filtered pattern, from that pattern's SVD of Bc_J
            DVec<double> uF((size_t)std::max<int64_t>(F.nnz, 1) * k, s), vsF((size_t)n * k * k, s);
            DVec<int32_t> zrF(n, s);
            RN_K_SWITCH(k, RN_LAUNCH("enforce", 4.0 * F.nnz + 16.0 * k * F.nnz + 8.0 * k * k * n, s,
                                     row_svd_kernel<KK>, rows_grid(n), kT, 0, n, F.rowptr.p, F.col.p, rowtype, Bc,
                                     uF.p, vsF.p, zrF.p));
            RN_K_SWITCH(k, RN_LAUNCH("enforce", 12.0 * F.nnz + 8.0 * k * (2.0 * F.nnz + n) + 8.0 * k * k * n, s,
                                     row_fit_u_kernel<KK>, rows_grid(n), kT, 0, n, F.rowptr.p, F.col.p, F.val.p,
                                     rowtype, Bsm, Bc, uF.p, vsF.p));
        }
        Pout = std::move(F);
        Pattern pf{n, nc, Pout.nnz, Pout.rowptr.p, Pout.col.p};
        energy_min(ctx_of(h), A, pf, Pout.val.p, rowtype, Bc, dinv.p, 1);
    }
}

void build_hierarchy(rn_hierarchy &h, const CsrView &A0, const double *B0, const double *Bhat0) {
    cudaStream_t s = h.s;
    const rn_params &p = h.p;
    const double omg = 1.0 - kGuard;
    h.partial.alloc(2 * kReduceBlocks, s);
    h.counters.alloc(4, s);
    RN_CUDA_CHECK(cudaMemsetAsync(h.counters.p, 0, 4 * sizeof(unsigned), s));
    h.scal.alloc(64, s);
    h.iflags.alloc(16, s);
    fill_f64(h.scal.p, 0.0, 64, s);
    fill_i32(h.iflags.p, 0, 16, s);
    // level 0: private copy of A, B (and B-hat)
    {
        auto L = std::make_unique<rn_level>();
        L->A.n = A0.n; L->A.m = A0.m; L->A.nnz = A0.nnz;
        L->A.rowptr.alloc(A0.n + 1, s); L->A.col.alloc(A0.nnz, s); L->A.val.alloc(A0.nnz, s);
        d2d(L->A.rowptr.p, A0.rowptr, A0.n + 1, s);
        d2d(L->A.col.p, A0.col, A0.nnz, s);
        d2d(L->A.val.p, A0.val, A0.nnz, s);
        L->B.alloc((size_t)A0.n * h.k, s);
        d2d(L->B.p, B0, (size_t)A0.n * h.k, s);
        if (!p.symmetric) {
            L->Bhat.alloc((size_t)A0.n * h.k, s);
            d2d(L->Bhat.p, Bhat0, (size_t)A0.n * h.k, s);
        }
        fill_i32(h.iflags.p + 3, 0, 1, s);
        RN_LAUNCH("validate", 12.0 * A0.nnz + 4.0 * A0.n, s, validate_kernel, rows_grid(A0.n), kT, 0, A0.n, A0.nnz,
                  L->A.rowptr.p, L->A.col.p, L->A.val.p, h.iflags.p + 3);
        check_flag(h.iflags.p + 3, s, RN_EINVAL, "CSR row malformed (bounds, unsorted/duplicate columns, no diagonal, "
                                                 "or non-finite value)");
        h.lev.push_back(std::move(L));
    }
    const int maxlev = std::max(1, std::min(p.max_levels, RN_MAX_LEVELS));
    MergedSetup *ms = h.merged;
    for (int l = 0;; l++) {
        rn_level &L = *h.lev[l];
        L.diag.alloc(L.A.n, s);
        fill_i32(h.iflags.p + 4, 0, 1, s);
        extract_diag(view(L.A), L.diag.p, h.iflags.p + 4, s);
        if (ms) {
            if (ms->end_small(h, l, maxlev)) break;  // every problem has reached its coarsest level
        } else if (L.A.n <= p.max_coarse || l >= maxlev - 1) {
            break;
        }
        const int32_t n = L.A.n;
        CsrView A = view(L.A);
        // the diagonal's flag is read with the strength pattern's size (a zero
        // diagonal only makes strength values non-finite until then)
        // ---- candidates smoothed on the side stream (they need only A and B)
        //      while this stream aggregates; joined after the aggregate count
        SideStream &ss = side_stream();
        DVec<double> cb0, cb1;
        const double *Bsmooth = nullptr;
        if (p.b_sweeps > 0) {
            cb0.alloc((size_t)n * h.k, s);
            cb1.alloc((size_t)n * h.k, s);
            RN_CUDA_CHECK(cudaEventRecord(ss.fork, s));
            RN_CUDA_CHECK(cudaStreamWaitEvent(ss.s, ss.fork, 0));
            Bsmooth = smooth_candidates(h, A, L.B.p, cb0.p, cb1.p, ss.s);
            RN_CUDA_CHECK(cudaEventRecord(ss.join, ss.s));
        }
        struct Join {  // the side stream's work is joined before this level's buffers can go
            cudaStream_t s;
            cudaEvent_t e;
            bool on;
            void operator()() {
                if (on) RN_CUDA_CHECK(cudaStreamWaitEvent(s, e, 0));
                on = false;
            }
            ~Join() {
                if (on) cudaStreamWaitEvent(s, e, 0);
            }
        } join{s, ss.join, p.b_sweeps > 0};
        const int32_t *roff = ms ? ms->roff.p : nullptr;  // aggregation priorities within each problem
        // ---- strength (line 'strength')
        const double theta = (l > 0 && p.soc_theta_coarse >= 0.0) ? p.soc_theta_coarse : p.soc_theta;
        const double thr = theta * omg;
        DCsr S;
        S.n = S.m = n;
        {
            DVec<int32_t> cnt(n + 1, s);
            DVec<double> vtmp(A.nnz, s), vmax(n, s);
            RN_LAUNCH("strength", 20.0 * A.nnz + 20.0 * n, s, strength_kernel<false>, rows_grid(n), kT, 0, n,
                      A.rowptr, A.col, A.val, L.diag.p, thr, cnt.p, vtmp.p, vmax.p, nullptr, nullptr, nullptr,
                      p.soc_kind == RN_SOC_CLASSICAL ? 1 : 0);
            S.rowptr.alloc(n + 1, s);
            int32_t fl[16];
            S.nnz = scan_with_flags(h, cnt.p, S.rowptr.p, n, fl);
            if (fl[4]) fail(RN_EINVAL, fmt("missing or zero diagonal (index %d)", fl[4] - 1));
            S.col.alloc(S.nnz, s);
            S.val.alloc(S.nnz, s);
            RN_LAUNCH("strength", 12.0 * A.nnz + 12.0 * n + 12.0 * S.nnz, s, strength_kernel<true>, rows_grid(n), kT,
                      0, n, A.rowptr, A.col, A.val, L.diag.p, thr, nullptr, vtmp.p, vmax.p, S.rowptr.p, S.col.p,
                      S.val.p, 0);
        }
        // ---- systems: S amalgamated to nodes (m unknowns each); scalar problems aggregate S itself
        const int mb = h.mb;
        const int32_t nn = n / mb;
        DCsr Sm;
        if (mb > 1) {
            DVec<int32_t> cnt(nn + 1, s);
            fill_i32(h.iflags.p + 6, 0, 1, s);
            RN_LAUNCH("amalgamate", 12.0 * S.nnz + 4.0 * n, s, amalgamate_kernel<false>, rows_grid(nn), kT, 0, nn, mb,
                      S.rowptr.p, S.col.p, S.val.p, cnt.p, nullptr, nullptr, nullptr, h.iflags.p + 6);
            check_flag(h.iflags.p + 6, s, RN_EINVAL, "a node row of S has too many entries to amalgamate");
            Sm.n = Sm.m = nn;
            Sm.rowptr.alloc(nn + 1, s);
            Sm.nnz = scan_counts(cnt.p, Sm.rowptr.p, nn, s);
            Sm.col.alloc(Sm.nnz, s);
            Sm.val.alloc(Sm.nnz, s);
            RN_LAUNCH("amalgamate", 12.0 * S.nnz + 12.0 * Sm.nnz, s, amalgamate_kernel<true>, rows_grid(nn), kT, 0, nn,
                      mb, S.rowptr.p, S.col.p, S.val.p, nullptr, Sm.rowptr.p, Sm.col.p, Sm.val.p, h.iflags.p + 6);
        }
        const DCsr &SG = mb > 1 ? Sm : S;  // the strength graph aggregation and the pattern run on
        // ---- aggregation graph and seeded MIS-2 (line 'aggregate'), on nodes
        DCsr Gr;
        {
            DCsr St;
            transpose(view(SG), false, St, s);
            DVec<int32_t> cnt(nn + 1, s);
            RN_LAUNCH("agg_graph", 8.0 * SG.nnz + 8.0 * nn, s, union_kernel<false>, rows_grid(nn), kT, 0, nn,
                      SG.rowptr.p, SG.col.p, St.rowptr.p, St.col.p, cnt.p, nullptr, nullptr);
            Gr.n = Gr.m = nn;
            Gr.rowptr.alloc(nn + 1, s);
            // only the row pointers are read from here on: the graph is allocated at
            // its bound (S and S^T without the diagonal) and its size never read back
            DVec<int64_t> tot(1, s);
            scan_counts_dev(cnt.p, Gr.rowptr.p, nn, tot.p, s);
            Gr.nnz = 2 * SG.nnz;
            Gr.col.alloc(Gr.nnz, s);
            RN_LAUNCH("agg_graph", 8.0 * SG.nnz + 8.0 * nn + 4.0 * Gr.nnz, s, union_kernel<true>, rows_grid(nn), kT, 0,
                      nn, SG.rowptr.p, SG.col.p, St.rowptr.p, St.col.p, nullptr, Gr.rowptr.p, Gr.col.p);
        }
        const uint64_t seed = p.seed + (uint64_t)l;
        DVec<int32_t> state(nn, s), m1(nn, s), r1(nn, s);
        const double gb = 4.0 * Gr.nnz + 8.0 * nn;
        RN_LAUNCH("mis2", gb, s, mis_init_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, state.p);
        int rounds = 0;
        for (;; rounds++) {
            if (rounds >= kMaxAggRounds) fail(RN_ETIMEOUT, fmt("aggregation did not finish in %d rounds", rounds));
            fill_i32(h.iflags.p + 5, 0, 1, s);
            RN_LAUNCH("mis2", gb + 8.0 * nn, s, mis_m1_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, Gr.col.p, state.p,
                      seed, roff, m1.p);
            RN_LAUNCH("mis2", gb + 8.0 * nn, s, mis_take_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, Gr.col.p, m1.p,
                      seed, roff, state.p);
            RN_LAUNCH("mis2", gb + 8.0 * nn, s, mis_r1_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, Gr.col.p, state.p,
                      r1.p);
            RN_LAUNCH("mis2", gb + 8.0 * nn, s, mis_remove_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, Gr.col.p, r1.p,
                      state.p, h.iflags.p + 5);
            // read the flag every second round: a round after the last is a no-op
            // (no undecided node), cheaper than a host synchronisation
            if ((rounds & 1) == 1 && read_scalar(h.iflags.p + 5, s) == 0) break;
        }
        h.agg_rounds += rounds + 1;
        DVec<int32_t> cidx(nn + 1, s);
        RN_LAUNCH("aggregate", 8.0 * nn, s, flag_taken_kernel, rows_grid(nn), kT, 0, nn, state.p, m1.p);
        const int32_t ncn = (int32_t)scan_counts(m1.p, cidx.p, nn, s);  // node aggregates
        join();  // before a stalled level's buffers are split off or replaced
        if (ms) {
            const int st = ms->stalled(h, l, cidx.p);
            if (st == 2) break;  // every remaining problem stalled here
            if (st == 1) {       // the level again without the problems that stalled
                l--;
                continue;
            }
        } else if (ncn == 0 || ncn >= nn) {
            break;  // stalled: this level is the coarsest
        }
        const int32_t nc = mb * ncn;       // coarse unknowns: m per root node
        L.nc = nc;
        L.roots.alloc(nc, s);
        L.agg.alloc(n, s);
        L.rowtype.alloc(n, s);
        DVec<int32_t> rootsN, aggN, rtN;  // node level (m > 1)
        if (mb > 1) {
            rootsN.alloc(ncn, s);
            aggN.alloc(nn, s);
            rtN.alloc(nn, s);
        }
        int32_t *roots_n = mb > 1 ? rootsN.p : L.roots.p, *agg_n = mb > 1 ? aggN.p : L.agg.p;
        int32_t *rt_n = mb > 1 ? rtN.p : L.rowtype.p;
        RN_LAUNCH("aggregate", 12.0 * nn, s, roots_kernel, rows_grid(nn), kT, 0, nn, state.p, cidx.p, roots_n);
        RN_LAUNCH("aggregate", gb + 12.0 * nn, s, agg_pass1_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, Gr.col.p,
                  state.p, cidx.p, seed, roff, r1.p);
        fill_i32(h.iflags.p + 6, 0, 1, s);
        RN_LAUNCH("aggregate", gb + 16.0 * nn, s, agg_pass2_kernel, rows_grid(nn), kT, 0, nn, Gr.rowptr.p, Gr.col.p,
                  state.p, r1.p, roots_n, seed, roff, agg_n, h.iflags.p + 6);
        // scalar problems read this flag with the pre-filter's size (an unassigned
        // node is only an unaggregated row until then); block systems at once
        if (mb > 1) check_flag(h.iflags.p + 6, s, RN_EINTERNAL, "aggregation pass 2 left a node unassigned");
        RN_LAUNCH("aggregate", 12.0 * nn, s, rowtype_kernel, rows_grid(nn), kT, 0, nn, state.p, agg_n, rt_n);
        if (mb > 1) {  // unamalgamate: aggregates, row types and roots of the unknowns
            RN_LAUNCH("aggregate", 16.0 * n, s, unamalgamate_nodes_kernel, rows_grid(n), kT, 0, n, mb, agg_n, rt_n,
                      L.agg.p, L.rowtype.p);
            RN_LAUNCH("aggregate", 8.0 * nc, s, unamalgamate_roots_kernel, rows_grid(ncn), kT, 0, ncn, mb, roots_n,
                      L.roots.p);
        }
        // ---- pattern N = S^d C, pre-filter, root-node pattern (on nodes; unamalgamated for m > 1)
        DCsr N, Nn;
        {
            DCsr cur;
            cur.n = nn;
            cur.m = ncn;
            cur.rowptr.alloc(nn + 1, s);
            RN_LAUNCH("pattern", 8.0 * nn, s, aggflag_kernel, rows_grid(nn), kT, 0, nn, agg_n, m1.p);
            // at most one entry per row, read through the row pointers only: allocated
            // at that bound, its size never read back
            DVec<int64_t> tot(1, s);
            scan_counts_dev(m1.p, cur.rowptr.p, nn, tot.p, s);
            cur.nnz = nn;
            cur.col.alloc(cur.nnz, s);
            cur.val.alloc(cur.nnz, s);
            RN_LAUNCH("pattern", 16.0 * nn, s, c_matrix_kernel, rows_grid(nn), kT, 0, nn, agg_n, cur.rowptr.p,
                      cur.col.p, cur.val.p);
            // each product's exact size stays on the device and comes back with the
            // next product's first read; a row past the block kernel's table is
            // reported with the pre-filter's read
            fill_i32(h.iflags.p + 12, 0, 1, s);
            for (int t = 0; t < p.degree; t++) {
                DCsr nxt;
                spgemm(view(SG), view(cur), nxt, s, false, cur.rowptr.p + cur.n, h.iflags.p + 12);
                cur = std::move(nxt);
            }
            DVec<int32_t> cnt(nn + 1, s);
            RN_LAUNCH("prefilter", 12.0 * cur.nnz + 12.0 * nn, s, prefilter_kernel<false>, rows_grid(nn), kT, 0, nn,
                      cur.rowptr.p, cur.col.p, cur.val.p, rt_n, agg_n, p.prefilter, omg, cnt.p, nullptr, nullptr,
                      nullptr);
            DCsr &NN = mb > 1 ? Nn : N;  // the node pattern: N itself for scalar problems
            NN.n = nn;
            NN.m = ncn;
            NN.rowptr.alloc(nn + 1, s);
            int32_t fl[16];
            NN.nnz = scan_with_flags(h, cnt.p, NN.rowptr.p, nn, fl);
            if (mb == 1 && fl[6])
                fail(RN_EINTERNAL, fmt("aggregation pass 2 left a node unassigned (index %d)", fl[6] - 1));
            if (fl[12]) fail(RN_EINTERNAL, fmt("pattern product row %d has more than 4096 distinct columns", fl[12] - 1));
            NN.col.alloc(NN.nnz, s);
            NN.val.alloc(NN.nnz, s);
            RN_LAUNCH("prefilter", 12.0 * cur.nnz + 12.0 * nn + 12.0 * NN.nnz, s, prefilter_kernel<true>,
                      rows_grid(nn), kT, 0, nn, cur.rowptr.p, cur.col.p, cur.val.p, rt_n, agg_n, p.prefilter, omg,
                      nullptr, NN.rowptr.p, NN.col.p, NN.val.p);
            if (mb > 1) {  // unamalgamate the pattern: m columns per node column, identity root rows
                DVec<int32_t> cn(n + 1, s);
                RN_LAUNCH("pattern", 8.0 * n + 4.0 * nn, s, unamalgamate_pattern_kernel<false>, rows_grid(n), kT, 0,
                          n, mb, Nn.rowptr.p, Nn.col.p, Nn.val.p, L.agg.p, L.rowtype.p, cn.p, nullptr, nullptr,
                          nullptr);
                N.n = n;
                N.m = nc;
                N.rowptr.alloc(n + 1, s);
                N.nnz = scan_counts(cn.p, N.rowptr.p, n, s);
                N.col.alloc(N.nnz, s);
                N.val.alloc(N.nnz, s);
                RN_LAUNCH("pattern", 12.0 * N.nnz + 12.0 * Nn.nnz, s, unamalgamate_pattern_kernel<true>, rows_grid(n),
                          kT, 0, n, mb, Nn.rowptr.p, Nn.col.p, Nn.val.p, L.agg.p, L.rowtype.p, nullptr, N.rowptr.p,
                          N.col.p, N.val.p);
            }
        }
        // ---- candidates, T, energy minimisation, filtering -> P
        L.Bc.alloc((size_t)nc * h.k, s);
        if (Bsmooth) d2d(L.B.p, Bsmooth, (size_t)n * h.k, s);
        build_transfer(h, A, N, L.agg.p, L.roots.p, nc, L.rowtype.p, L.B.p, L.diag.p, L.Bc.p, L.P,
                       p.keep_aux ? &L.T : nullptr, true);
        // ---- R
        if (p.symmetric) {
            transpose(view(L.P), true, L.R, s);
        } else {
            DCsr At, Rt;
            transpose(A, true, At, s);
            DVec<double> diagT(n, s);
            d2d(diagT.p, L.diag.p, n, s);  // the diagonal of A^T is the diagonal of A
            L.Bhatc.alloc((size_t)nc * h.k, s);
            build_transfer(h, view(At), N, L.agg.p, L.roots.p, nc, L.rowtype.p, L.Bhat.p, diagT.p, L.Bhatc.p, Rt,
                           nullptr);
            transpose(view(Rt), true, L.R, s);
        }
        // ---- Galerkin product A_{l+1} = R (A P)
        auto Lc = std::make_unique<rn_level>();
        {
            DCsr AP;
            spgemm(A, view(L.P), AP, s, true);
            spgemm(view(L.R), view(AP), Lc->A, s, true);
        }
        Lc->B.alloc((size_t)nc * h.k, s);
        d2d(Lc->B.p, L.Bc.p, (size_t)nc * h.k, s);
        if (!p.symmetric) {
            Lc->Bhat.alloc((size_t)nc * h.k, s);
            d2d(Lc->Bhat.p, L.Bhatc.p, (size_t)nc * h.k, s);
        }
        if (p.keep_aux) {
            L.S = std::move(S);
            L.N = std::move(N);
        }
        h.lev.push_back(std::move(Lc));
        if (ms) ms->split_level(h, l);  // releases the merged level l (L is not used past this point)
    }
    if (ms) return;  // every problem's coarsest level is factored by the caller
    coarsest_lu(h);
    if (!p.keep_aux) {
        for (auto &Lp : h.lev) {
            Lp->agg.release();
            Lp->roots.release();
        }
    }
}

// The coarsest level: dense LU with partial pivoting, kept as an explicit
// inverse.  Without check, the one-launch factorisation of a small level is
// only enqueued (a singular pivot leaves non-finite values, nothing out of
// bounds) and coarsest_lu_check reads the singularity flag later, so many
// problems' factorisations overlap.
static void coarsest_lu_check(rn_hierarchy &h) {
    check_flag(h.iflags.p + 7, h.s, RN_ESINGULAR, "coarsest-level LU pivot below 1e-14 max|A|");
}
static void coarsest_lu(rn_hierarchy &h, bool check) {
    cudaStream_t s = h.s;
    rn_level &C = *h.lev.back();
    const int32_t nL = C.A.n;
    if (nL > kMaxDense)
        fail(RN_ESTALL, fmt("coarsening stalled with %d rows (> %d for the dense solve)", nL, kMaxDense));
    h.nL = nL;
    if (nL <= kLuSmall) {  // one launch, the matrix and its inverse in shared memory
        const size_t smem = 2 * sizeof(double) * (size_t)nL * nL;
        static const bool configured = [] {  // once (thread-safe static initialisation)
            RN_CUDA_CHECK(cudaFuncSetAttribute(dense_lu_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(2 * sizeof(double) * kLuSmall * kLuSmall)));
            return true;
        }();
        (void)configured;
        fill_i32(h.iflags.p + 7, 0, 1, s);
        h.Ainv.alloc((size_t)nL * nL, s);
        RN_LAUNCH("coarse_lu", 12.0 * C.A.nnz + 8.0 * nL * nL, s, dense_lu_small_kernel, 1, 256, smem, nL,
                  C.A.rowptr.p, C.A.col.p, C.A.val.p, h.Ainv.p, h.iflags.p + 7);
        if (check) coarsest_lu_check(h);
    } else {
        DVec<double> M((size_t)nL * nL, s), work((size_t)nL * nL, s);
        DVec<int32_t> piv(nL, s);
        fill_f64(M.p, 0.0, (int64_t)nL * nL, s);
        RN_LAUNCH("coarse_lu", 12.0 * C.A.nnz, s, csr_to_dense_kernel, rows_grid(nL), kT, 0, nL, C.A.rowptr.p, C.A.col.p,
                  C.A.val.p, M.p);
        fill_i32(h.iflags.p + 7, 0, 1, s);
        RN_LAUNCH("coarse_lu", 16.0 * nL * nL, s, dense_lu_kernel, 1, 1024, 0, nL, M.p, piv.p, h.iflags.p + 7);
        // always checked here: a singular factorisation stops early and leaves
        // later pivot indices unset, which the inverse must not read
        coarsest_lu_check(h);
        h.Ainv.alloc((size_t)nL * nL, s);
        RN_LAUNCH("coarse_lu", 24.0 * nL * nL, s, lu_inverse_kernel, grid_for(nL, 64, 4), 64, 0, nL, M.p, piv.p, h.Ainv.p,
                  work.p);
    }
}

// Independent problems set up together (see MergedSetup): out[t] must hold
// problem t's params (CG energy minimisation, one candidate, scalar problems,
// R = P^T), stream and no levels; A[t] and B[t] are device data.
void build_hierarchies_merged(std::vector<rn_hierarchy *> &out, const std::vector<CsrView> &A,
                              const std::vector<const double *> &B, cudaStream_t s) {
    const int np = (int)out.size();
    if (np == 0) return;
    rn_hierarchy W;  // the working hierarchy of the merged matrices
    W.p = out[0]->p;
    W.k = 1;
    W.mb = 1;
    W.s = s;
    MergedSetup ms;
    ms.out = out;
    ms.s = s;
    ms.act.resize(np);
    ms.ev.assign(np, nullptr);
    for (int t = 0; t < np; t++) {
        ms.act[t] = t;
        RN_CUDA_CHECK(cudaEventCreateWithFlags(&ms.ev[t], cudaEventDisableTiming));
    }
    // every problem's scratch, as build_hierarchy allocates it
    for (int t = 0; t < np; t++) {
        rn_hierarchy *h = out[t];
        const AllocScope scope(ms.alloc_for(t));
        h->partial.alloc(2 * kReduceBlocks, h->s);
        h->counters.alloc(4, h->s);
        RN_CUDA_CHECK(cudaMemsetAsync(h->counters.p, 0, 4 * sizeof(unsigned), h->s));
        h->scal.alloc(64, h->s);
        h->iflags.alloc(16, h->s);
        fill_f64(h->scal.p, 0.0, 64, h->s);
        fill_i32(h->iflags.p, 0, 16, h->s);
    }
    // each problem's CSR checked on its own (a column past its own size is an error)
    {
        DVec<int32_t> bad((size_t)np, s);
        fill_i32(bad.p, 0, np, s);
        for (int t = 0; t < np; t++)
            RN_LAUNCH("validate", 12.0 * A[t].nnz + 4.0 * A[t].n, s, validate_kernel, rows_grid(A[t].n), kT, 0,
                      A[t].n, A[t].nnz, A[t].rowptr, A[t].col, A[t].val, bad.p + t);
        std::vector<int32_t> bh((size_t)np);
        read_vec(bh.data(), bad.p, (size_t)np, s);
        for (int t = 0; t < np; t++)
            if (bh[t])
                fail(RN_EINVAL, fmt("problem %d: CSR row %d malformed (bounds, unsorted/duplicate columns, no "
                                    "diagonal, or non-finite value)", t, bh[t] - 1));
    }
    // the merged level-0 operator and candidates
    std::vector<int32_t> ro(1, 0);
    std::vector<int64_t> eo(1, 0);
    for (int t = 0; t < np; t++) {
        ro.push_back(ro.back() + A[t].n);
        eo.push_back(eo.back() + A[t].nnz);
    }
    if (eo.back() > INT32_MAX - 1 || ro.back() > INT32_MAX - 1) fail(RN_EINVAL, "merged problems exceed int32 sizes");
    DCsr M;
    M.n = M.m = ro.back();
    M.nnz = eo.back();
    M.rowptr.alloc((size_t)M.n + 1, s);
    M.col.alloc((size_t)M.nnz, s);
    M.val.alloc((size_t)M.nnz, s);
    DVec<double> Bm((size_t)M.n, s);
    {
        std::vector<BlockCsr> blk;
        for (int t = 0; t < np; t++) {
            BlockCsr b{0, A[t].n, 0, (int32_t)A[t].nnz, ro[t], (int32_t)eo[t], ro[t], M.rowptr.p, M.col.p, M.val.p};
            b.srp = A[t].rowptr;
            b.scol = A[t].col;
            b.sval = A[t].val;
            blk.push_back(b);
            d2d(Bm.p + ro[t], B[t], (size_t)A[t].n, s);
        }
        ms.launch_csr(blk, view(M));
    }
    ms.set_rows(ro, M.n);
    W.merged = &ms;
    build_hierarchy(W, view(M), Bm.p, nullptr);
    W.merged = nullptr;
    cudaEvent_t done = ms.ev[0];
    RN_CUDA_CHECK(cudaEventRecord(done, s));
    for (rn_hierarchy *h : out) {
        RN_CUDA_CHECK(cudaStreamWaitEvent(h->s, done, 0));
        h->agg_rounds = W.agg_rounds;
    }
    // every problem's coarsest LU enqueued on its stream, then the flags read
    for (int t = 0; t < np; t++) {
        const AllocScope scope(ms.alloc_for(t));
        coarsest_lu(*out[t], false);
    }
    for (size_t t = 0; t < out.size(); t++) {
        try {
            coarsest_lu_check(*out[t]);
        } catch (const Error &e) {
            fail(e.status, fmt("problem %zu: %s", t, e.msg.c_str()));
        }
    }
}

// ================================================================== measurement hook
// Level 0's energy minimisation, one piece at a time: the state every timed
// run starts from is the one after the first sweep (restored before each
// run, outside the timed region), so every run times a general sweep (beta
// term included) on the minimisation's own pattern N, values and precision.
template <typename TV>
static void time_energy(rn_hierarchy &h, int op, int reps, int64_t flush_bytes, double *us, double *bytes,
                        std::string &name) {
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[0];
    const CsrView A = view(L.A);
    const int32_t n = A.n;
    const size_t nz = (size_t)L.N.nnz;
    Pattern pat{n, L.N.m, L.N.nnz, L.N.rowptr.p, L.N.col.p};
    DVec<double> x0(nz, s), dinv(n, s);
    d2d(x0.p, L.T.val.p, nz, s);
    reciprocal(L.diag.p, dinv.p, n, s);
    EmCtx c = ctx_of(h);
    CgSweep<TV> cg(c, A, pat, x0.p, L.rowtype.p, L.Bc.p, dinv.p);
    cg.start();
    cg.sweep(0);
    DVec<TV> sX(nz, s), sR(nz, s), sD(nz, s);
    DVec<double> ssc(8, s);
    d2d(sX.p, cg.X, nz, s);
    d2d(sR.p, cg.R, nz, s);
    d2d(sD.p, cg.Dd, nz, s);
    d2d(ssc.p, c.sc, 8, s);
    auto restore = [&]() {
        d2d(cg.X, sX.p, nz, s);
        d2d(cg.R, sR.p, nz, s);
        d2d(cg.Dd, sD.p, nz, s);
        d2d(c.sc, ssc.p, 8, s);
        fill_i32(c.fl, 0, 1, s);
    };
    const double vb = sizeof(TV);
    std::function<void()> before, timed;
    switch (op) {
        case RN_SOP_ENERGY_SWEEP:
            name = "energy_sweep_L0";
            before = restore;
            timed = [&]() { cg.sweep(1); };
            *bytes = cg.sweep_bytes();
            break;
        case RN_SOP_ENERGY_DIRECTION:
            name = "energy_direction_L0";
            before = restore;
            timed = [&]() { cg.direction(1); };
            *bytes = cg.rpb + 3.0 * cg.nzb + cg.db;
            break;
        case RN_SOP_ENERGY_PRODUCT:
            name = "energy_product_L0";
            before = [&]() { restore(); cg.direction(1); };
            timed = [&]() { cg.sweep_product(); };
            // A, both row-pointer arrays, row types, row scales, the pattern's
            // columns, X gathered once, W written, Y read, Bc (no gather map)
            *bytes = (4.0 + vb) * A.nnz + 8.0 * (n + 1) + 4.0 * n + vb * n + 4.0 * nz + 3.0 * vb * nz +
                     vb * h.k * L.N.m;
            break;
        case RN_SOP_ENERGY_UPDATE:
            name = "energy_update_L0";
            before = [&]() { restore(); cg.direction(1); cg.sweep_product(); };
            timed = [&]() { cg.update(1); };
            *bytes = cg.rpb + 6.0 * cg.nzb + cg.db;
            break;
        default: fail(RN_EINVAL, "unknown setup operation");
    }
    *us = time_launches(s, reps, flush_bytes, before, timed);
}

void time_setup_op(rn_hierarchy &h, int op, int reps, int64_t flush_bytes, double *us, double *bytes,
                   std::string &name) {
    if (op < 0 || op >= RN_SOP_COUNT) fail(RN_EINVAL, "unknown setup operation");
    if (h.lev.size() < 2) fail(RN_EINVAL, "a one-level hierarchy has no setup operation to time");
    cudaStream_t s = h.s;
    rn_level &L = *h.lev[0];
    const CsrView A = view(L.A);
    if (op <= RN_SOP_ENERGY_UPDATE) {
        if (!h.p.keep_aux || !L.N.rowptr.p || !L.T.val.p)
            fail(RN_EINVAL, "timing the energy minimisation needs a hierarchy built with keep_aux");
        if (h.p.energy_method != RN_ENERGY_CG) fail(RN_EINVAL, "the energy-minimisation timing covers CG sweeps");
        if (h.p.precision == RN_MIXED) time_energy<float>(h, op, reps, flush_bytes, us, bytes, name);
        else time_energy<double>(h, op, reps, flush_bytes, us, bytes, name);
        return;
    }
    const std::function<void()> none;
    if (op == RN_SOP_TRANSPOSE) {
        name = "transpose_P_L0";
        *bytes = 24.0 * L.P.nnz;
        *us = time_launches(s, reps, flush_bytes, none, [&]() {
            DCsr Pt;
            transpose(view(L.P), true, Pt, s);
        });
        return;
    }
    DCsr AP;
    spgemm(A, view(L.P), AP, s, true);  // untimed: its size, and the operand of R (A P)
    if (op == RN_SOP_GALERKIN_AP) {
        name = "galerkin_AP_L0";
        *bytes = 12.0 * (A.nnz + L.P.nnz) + 12.0 * AP.nnz;
        *us = time_launches(s, reps, flush_bytes, none, [&]() {
            DCsr C;
            spgemm(A, view(L.P), C, s, true);
        });
    } else {
        name = "galerkin_RAP_L0";
        *bytes = 12.0 * (L.R.nnz + AP.nnz) + 12.0 * h.lev[1]->A.nnz;
        *us = time_launches(s, reps, flush_bytes, none, [&]() {
            DCsr C;
            spgemm(view(L.R), view(AP), C, s, true);
        });
    }
}

}  // namespace rn
