// rn_device.cuh - device-side helpers shared by the kernels: programmatic
// dependent launch, warp and block sums, and the deterministic grid reduction
// with its scalar finishers.  Included by rn_internal.cuh.
#pragma once

// --------------------------------------------------------------- device helpers
namespace rn {
// Wait until the preceding grid in the stream has completed and its memory
// is visible (programmatic dependent launch); a no-op for ordinary launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Allow the next grid in the stream to be scheduled (it still waits in
// pdl_wait until this grid has completed).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}
template <int G>
__device__ __forceinline__ float group_sumf(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    const int lane = threadIdx.x & 31;
    return ((1u << (G & 31)) - 1u) << (lane & ~(G - 1));
}
// SplitMix64 (Steele, Lea, Flood 2014), from its published definition.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
// Block-level sum of one double per thread; result valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double *smem32) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem32[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (lane < BLOCK / 32) ? smem32[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// What the last block does with the finished sums of a grid reduction.
enum FinMode { FIN_NONE = 0, FIN_STORE = 1, FIN_CG_RHO = 2, FIN_CG_DW = 3, FIN_RZ = 4, FIN_PQ = 5, FIN_XR = 6 };
// Outer CG scalars in sc: [8] ||r||^2, [9] <r,z>, [10] <p,Ap>, [11] <z,r_old>,
// [12] alpha, [13] beta, [14] previous <r,z>, [17] ||b||^2, [18] ||b|| (1 when
// b = 0), [19] rtol; int flags fl: [9] iterations done, [10] iteration limit,
// [11] converged.
struct Fin {
    int mode = FIN_NONE;
    double *partial = nullptr;   // >= 2 * kReduceBlocks slots
    unsigned *counter = nullptr; // zero between launches (the last block resets it)
    double *out = nullptr;       // FIN_STORE: out[0] = s0 (and out[1] = s1 when two sums)
    double *sc = nullptr;        // scalar block of the CG recurrences
    int32_t *fl = nullptr;       // fl[0]: energy-minimisation "done"
    int it = 0;                  // energy CG: iteration; FIN_RZ: bit 0 first, bit 1 flexible
    double stop = 0.0;
    // FIN_XR inside the solve graph: conditional handles of the next
    // iteration and of this iteration's preconditioning half (0: none)
    unsigned long long cond_loop = 0, cond_body = 0;
};

__device__ __forceinline__ void apply_fin(const Fin &f, const double *s, int nv) {
    switch (f.mode) {
        case FIN_STORE:
            f.out[0] = s[0];
            if (nv > 1) f.out[1] = s[1];
            break;
        case FIN_CG_RHO: {  // energy CG: rho = <R, D^-1 R>; stop test; beta
            if (f.fl[0]) return;
            const double r = s[0];
            if (f.it == 0) f.sc[1] = r;
            if (r == 0.0 || r <= f.stop * f.sc[1]) {
                f.fl[0] = 1;
                return;
            }
            f.sc[2] = (f.it == 0) ? 0.0 : r / f.sc[0];
            f.sc[0] = r;
            break;
        }
        case FIN_CG_DW: {  // energy CG: <D, W>; breakdown test; alpha
            if (f.fl[0]) return;
            f.sc[3] = s[0];
            if (!(s[0] > 0.0)) {
                f.fl[0] = 1;
                return;
            }
            f.sc[4] = f.sc[0] / s[0];
            break;
        }
        case FIN_RZ: {  // outer CG: keep the previous <r,z>, store <r,z> and <z, r_old>; beta
            f.sc[14] = f.sc[9];
            f.sc[9] = s[0];
            const double zro = nv > 1 ? s[1] : 0.0;
            f.sc[11] = zro;
            // beta = <z,r>/<z,r>_prev, or (<z,r> - <z,r_old>)/<z,r>_prev for the flexible variant
            f.sc[13] = (f.it & 1) ? 0.0 : ((f.it & 2) ? s[0] - zro : s[0]) / f.sc[14];
            break;
        }
        case FIN_PQ:  // outer CG: <p, Ap> and alpha = <r,z> / <p, Ap>
            f.sc[10] = s[0];
            f.sc[12] = f.sc[9] / s[0];
            break;
        case FIN_XR: {  // outer CG: ||r||^2, iteration count, stopping test
            f.sc[8] = s[0];
            const int it = ++f.fl[9];
            const bool conv = sqrt(s[0]) / f.sc[18] < f.sc[19];
            const bool stop = conv || it >= f.fl[10];
            f.fl[11] = conv ? 1 : 0;
            if (f.cond_loop) cudaGraphSetConditional(f.cond_loop, stop ? 0u : 1u);
            if (f.cond_body) cudaGraphSetConditional(f.cond_body, stop ? 0u : 1u);
            break;
        }
        default: break;
    }
}

// Deterministic grid reduction of NV per-thread values.  Every block writes
// its totals to f.partial[k * kReduceBlocks + block]; the block that arrives
// last sums them in block order (a fixed order, whichever block is last) and
// applies the finisher in thread 0.  All threads of every block must call it.
template <int BLOCK, int NV>
__device__ __forceinline__ void grid_finish(const double (&v)[NV], const Fin &f, double *smem32) {
    if (f.mode == FIN_NONE) return;
    __shared__ int am_last;
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) t[k] = block_sum<BLOCK>(v[k], smem32);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) f.partial[k * kReduceBlocks + blockIdx.x] = t[k];
        __threadfence();
        const unsigned prev = atomicAdd(f.counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) {
        __threadfence();
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double a = 0.0;
            for (int i = threadIdx.x; i < (int)gridDim.x; i += BLOCK) a += __ldcg(&f.partial[k * kReduceBlocks + i]);
            s[k] = block_sum<BLOCK>(a, smem32);
        }
        if (threadIdx.x == 0) {
            apply_fin(f, s, NV);
            *f.counter = 0u;
            __threadfence();
        }
    }
}

}  // namespace rn
