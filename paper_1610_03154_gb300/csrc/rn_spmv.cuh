// rn_spmv.cuh - the staged SpMV family of the cycle and the outer iteration.
//
// SpMV-family kernels stream the CSR arrays through shared memory: each
// persistent CTA walks tiles of 256/G rows; thread 0 issues TMA bulk copies
// (cp.async.bulk, completion counted on an mbarrier) of the tile's column and
// value segments into a double buffer, so the next tile's matrix data is in
// flight while the current one is computed.  Only x is gathered from global
// memory (it is small enough to stay in L2).  Included by rn_solve.cu only.
#pragma once

#include "rn_hier.cuh"

namespace rn {

constexpr int kS = 256;           // threads per block, SpMV family
// matrix entries per shared-memory stage (four FP32 or three FP64 CTAs fit
// one SM; smaller FP64 stages with two lanes per row measured slower)
template <typename T>
constexpr int tile_nnz() {
    return 3072;
}
constexpr int kTileSlack = 8;     // room for 16-byte alignment of the bulk copies
constexpr uint32_t kMaxSpin = 1u << 24;  // bound on mbarrier polls before giving up

enum SpOp { OP_SPMV = 0, OP_SPMV_ADD = 1, OP_RESID = 2, OP_JACOBI = 3, OP_SPMV_DOT = 4, OP_JZ_RESID = 5,
            OP_JACOBI_RZ = 6 };
// OP_JZ_RESID: first relaxation from a zero guess fused with the residual:
//   xz = omega b / d,  y = b - A xz
// OP_JACOBI_RZ: the cycle's last sweep on level 0 (b = r of the outer CG,
//   y = z) fused with the outer CG's <r, z> and <z, r_old> (aux = r_old)
template <int OP>
struct OpNV {  // values reduced over the grid
    static constexpr int value = OP == OP_JACOBI_RZ ? 2 : 1;
};
template <int OP>
constexpr bool op_reduces() {
    return OP == OP_RESID || OP == OP_SPMV_DOT || OP == OP_JACOBI_RZ;
}

// ------------------------------------------------------------------ mbarrier / bulk-copy helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// An L2 policy that makes the lines it tags the first to be evicted: the
// matrix streams (read once per launch, and a cycle streams several times L2's
// capacity) then leave the vectors the gathers read resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_g2s_stream(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                                uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t k = 0; k < kMaxSpin; k++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The operand gathered at column j: x_j, or, for the fused first sweep from a
// zero guess, x_j = omega b_j / d_j computed on the fly (the same expression
// jacobi_zero_kernel stores, so the residual is bit-identical to the unfused
// pair of kernels).
template <typename T, typename TB, int OP>
__device__ __forceinline__ T xget(int32_t j, const T *__restrict__ x, const TB *__restrict__ b,
                                  const T *__restrict__ diag, T omega) {
    if (OP == OP_JZ_RESID) return diag[j] * (T)b[j];  // diag holds omega / a_jj
    return x[j];
}

template <typename T, typename TB, typename TO, int OP>
__device__ __forceinline__ void spmv_epilogue(int32_t i, T acc, const T *__restrict__ x, const TB *__restrict__ b,
                                              const T *__restrict__ diag, T omega, TO *__restrict__ y,
                                              T *__restrict__ xz, const double *__restrict__ aux, double *red) {
    if (OP == OP_SPMV) {
        y[i] = (TO)acc;
    } else if (OP == OP_SPMV_ADD) {
        y[i] = (TO)((T)y[i] + acc);
    } else if (OP == OP_RESID) {
        const T r = (T)b[i] - acc;
        y[i] = (TO)r;
        red[0] += (double)r * (double)r;
    } else if (OP == OP_JACOBI) {
        y[i] = (TO)(x[i] + diag[i] * ((T)b[i] - acc));
    } else if (OP == OP_JACOBI_RZ) {
        const TO z = (TO)(x[i] + diag[i] * ((T)b[i] - acc));
        y[i] = z;
        red[0] = fma((double)b[i], (double)z, red[0]);
        if (aux) red[1] = fma((double)z, aux[i], red[1]);
    } else if (OP == OP_JZ_RESID) {
        xz[i] = diag[i] * (T)b[i];
        y[i] = (TO)((T)b[i] - acc);
    } else {  // OP_SPMV_DOT
        y[i] = (TO)acc;
        red[0] += (double)x[i] * (double)acc;
    }
}

// Tile kernel: G lanes per row, RPT = 256/G rows per tile.  The tile's row
// pointers and its matrix segment (<= tile_nnz<T>() entries; guaranteed by the
// host's choice of G) are staged by bulk copies into a two-stage buffer.
// Thread 0 keeps the next tile's copies in flight and prefetches the bounds
// of the tile after that.  err[0] is set if an mbarrier wait gives up.
template <typename T, typename TB, typename TO, int G, int OP, bool TL>
__global__ void __launch_bounds__(kS)
spmv_tile_kernel(int32_t n, int32_t ntiles, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                 const T *__restrict__ val, const T *__restrict__ x, const TB *__restrict__ b,
                 const T *__restrict__ diag, T omega, TO *__restrict__ y, T *__restrict__ xz,
                 const double *__restrict__ aux, Fin fin, int32_t *__restrict__ err,
                 const int32_t *__restrict__ tlist, const int32_t *__restrict__ tcount) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NV = OpNV<OP>::value;
    constexpr int SL = tile_nnz<T>() + kTileSlack;
    constexpr int RPT = kS / G;
    constexpr int RL = RPT + 8;  // staged row pointers per stage (RPT + 1, rounded to 16 bytes)
    constexpr int VA = 16 / (int)sizeof(T);
    int32_t *scol = reinterpret_cast<int32_t *>(smem_raw);
    int32_t *srp = scol + 2 * SL;
    T *sval = reinterpret_cast<T *>(smem_raw + (2 * SL + 2 * RL) * sizeof(int32_t));
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double sm[32];
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t pend = 0u;             // thread 0: bit s = copies into stage s issued, not yet waited for
    const uint64_t pol = l2_evict_first_policy();
    int32_t be0 = 0, be1 = 0;       // thread 0: nnz bounds of the next tile to issue
    // the tiles to process: all, or (TL) the first *tcount entries of tlist
    // (which only change between launches, so they are read before pdl_wait)
    int32_t nt = ntiles;
    if constexpr (TL) nt = *tcount;
    auto tile_of = [&](int i) {
        if constexpr (TL) return tlist[i];
        else return i;
    };
    auto load_bounds = [&](int i) {
        if (i < nt) {
            const int32_t t = tile_of(i);
            be0 = rp[t * RPT];
            be1 = rp[min(n, t * RPT + RPT)];
        }
    };
    auto issue = [&](int stage, int i) {
        const int32_t r0 = tile_of(i) * RPT;
        const int32_t r1 = min(n, r0 + RPT);
        const int32_t c0 = be0 & ~3, c1 = (be1 + 3) & ~3;
        const int32_t v0 = be0 & ~(VA - 1), v1 = (be1 + VA - 1) & ~(VA - 1);
        const uint32_t cb = (uint32_t)(c1 - c0) * 4u, vb = (uint32_t)(v1 - v0) * (uint32_t)sizeof(T);
        const uint32_t rb = (uint32_t)(((r1 - r0 + 1) + 3) & ~3) * 4u;  // r0 is a multiple of 8: aligned
        mbar_expect_tx(&bar[stage], cb + vb + rb);
        bulk_g2s(srp + stage * RL, rp + r0, rb, &bar[stage]);
        if (cb) bulk_g2s_stream(scol + stage * SL, col + c0, cb, &bar[stage], pol);
        if (vb) bulk_g2s_stream(sval + stage * SL, val + v0, vb, &bar[stage], pol);
        pend |= 1u << stage;
    };
    double red[NV] = {};
    uint32_t parity = 0u;  // bit s = phase parity to wait for on stage s
    bool failed = false;
    int st = 0;
    int it = blockIdx.x;  // position in the tile sequence
    if (tid == 0 && it < nt) {  // the matrix is constant: stage it before the predecessor finishes
        load_bounds(it);
        issue(0, it);
        load_bounds(it + gridDim.x);
    }
    pdl_wait();
    pdl_trigger();
    for (; it < nt; it += gridDim.x, st ^= 1) {
        const int nxt = it + gridDim.x;
        if (tid == 0 && nxt < nt) {
            fence_proxy_async();  // earlier generic reads of that stage come before the async writes
            issue(st ^ 1, nxt);
            load_bounds(nxt + gridDim.x);  // lands while this tile is computed
        }
        const int32_t r0 = tile_of(it) * RPT;
        const int32_t row = r0 + tid / G;
        const int lane = tid % G;
        const bool live = row < min(n, r0 + RPT);
        // epilogue operands: issue their loads before waiting on the stage
        T xi = T(0), di = T(1);
        TB bi = TB(0);
        TO yi = TO(0);
        double ai = 0.0;
        if (live && lane == 0) {
            if (OP == OP_JACOBI || OP == OP_JACOBI_RZ || OP == OP_SPMV_DOT) xi = x[row];
            if (OP == OP_RESID || OP == OP_JACOBI || OP == OP_JACOBI_RZ || OP == OP_JZ_RESID) bi = b[row];
            if (OP == OP_JACOBI || OP == OP_JACOBI_RZ || OP == OP_JZ_RESID) di = diag[row];
            if (OP == OP_SPMV_ADD) yi = y[row];
            if (OP == OP_JACOBI_RZ && aux) ai = aux[row];
        }
        const bool ok = mbar_wait_bounded(&bar[st], (parity >> st) & 1u);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u << st;
        if (tid == 0) pend &= ~(1u << st);
        const int32_t *srow = srp + st * RL;
        const int32_t e0 = srow[0];
        const int32_t c0 = e0 & ~3, v0 = e0 & ~(VA - 1);
        const int32_t *sc = scol + st * SL;
        const T *sv = sval + st * SL;
        T acc = T(0);
        if (live) {
            // staged entry k of the matrix sits at sc[k - c0] / sv[k - v0]
            const int32_t s = srow[tid / G], e = srow[tid / G + 1];
            int32_t k = s + lane;
            for (; k + 3 * G < e; k += 4 * G) {  // four independent gathers in flight
                const int32_t j0 = sc[k - c0], j1 = sc[k + G - c0], j2 = sc[k + 2 * G - c0], j3 = sc[k + 3 * G - c0];
                const T a0 = sv[k - v0], a1 = sv[k + G - v0], a2 = sv[k + 2 * G - v0], a3 = sv[k + 3 * G - v0];
                const T x0 = xget<T, TB, OP>(j0, x, b, diag, omega), x1 = xget<T, TB, OP>(j1, x, b, diag, omega),
                        x2 = xget<T, TB, OP>(j2, x, b, diag, omega), x3 = xget<T, TB, OP>(j3, x, b, diag, omega);
                acc = fma(a0, x0, acc);
                acc = fma(a1, x1, acc);
                acc = fma(a2, x2, acc);
                acc = fma(a3, x3, acc);
            }
            for (; k < e; k += G) acc = fma(sv[k - v0], xget<T, TB, OP>(sc[k - c0], x, b, diag, omega), acc);
        }
        if (G > 1) {
            const unsigned mask = group_mask<G>();
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, G);
        }
        if (live && lane == 0) {
            if (OP == OP_SPMV) {
                y[row] = (TO)acc;
            } else if (OP == OP_SPMV_ADD) {
                y[row] = (TO)((T)yi + acc);
            } else if (OP == OP_RESID) {
                const T r = (T)bi - acc;
                y[row] = (TO)r;
                if (fin.mode != FIN_NONE) red[0] += (double)r * (double)r;
            } else if (OP == OP_JACOBI) {
                y[row] = (TO)(xi + di * ((T)bi - acc));
            } else if (OP == OP_JACOBI_RZ) {
                const TO z = (TO)(xi + di * ((T)bi - acc));
                y[row] = z;
                red[0] = fma((double)bi, (double)z, red[0]);
                red[NV - 1] = fma((double)z, ai, red[NV - 1]);  // ai = 0 without r_old
            } else if (OP == OP_JZ_RESID) {
                xz[row] = di * (T)bi;
                y[row] = (TO)((T)bi - acc);
            } else {
                y[row] = (TO)acc;
                red[0] += (double)xi * (double)acc;
            }
        }
        __syncthreads();  // this stage is fully read before it is refilled
    }
    if (failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int q = 0; q < 2; q++)
                if ((pend >> q) & 1u) mbar_wait_bounded(&bar[q], (parity >> q) & 1u);  // let our own copies land
        }
        __syncthreads();
    }
    if (op_reduces<OP>()) grid_finish<kS, NV>(red, fin, sm);
}

// Fallback for matrices with rows too long for a stage: G lanes per row
// straight from global memory.
template <typename T, typename TB, typename TO, int G, int OP>
__global__ void __launch_bounds__(kS)
spmv_group_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                  const T *__restrict__ val, const T *__restrict__ x, const TB *__restrict__ b,
                  const T *__restrict__ diag, T omega, TO *__restrict__ y, T *__restrict__ xz,
                  const double *__restrict__ aux, Fin fin) {
    __shared__ double sm[32];
    constexpr int NV = OpNV<OP>::value;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    double red[NV] = {};
    pdl_wait();
    pdl_trigger();
    for (int32_t i0 = blockIdx.x * (kS / G); i0 < n; i0 += gridDim.x * (kS / G)) {
        const int32_t i = i0 + g;
        T acc = T(0);
        if (i < n)
            for (int32_t e = rp[i] + lane; e < rp[i + 1]; e += G)
                acc = fma(val[e], xget<T, TB, OP>(col[e], x, b, diag, omega), acc);
        if (G > 1) {
            const unsigned mask = group_mask<G>();
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, G);
        }
        if (lane == 0 && i < n) spmv_epilogue<T, TB, TO, OP>(i, acc, x, b, diag, omega, y, xz, aux, red);
    }
    if (op_reduces<OP>()) grid_finish<kS, NV>(red, fin, sm);
}

}  // namespace rn
