// rn_internal.cuh - shared internals of the root-node AMG CUDA library.
//
// Error model: internal code throws rn::Error (status + message); every C-ABI
// entry point catches it and returns the status.  Device buffers are RAII
// objects freed with cudaFreeAsync on the stream they were allocated on, so an
// exception anywhere in setup releases everything.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rn.h"

namespace rn {

struct Error {
    rn_status status;
    std::string msg;
};

[[noreturn]] void fail(rn_status s, const std::string &msg);
void set_last_error(const std::string &msg);

#define RN_CUDA_CHECK(call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (e_ == cudaErrorMemoryAllocation)                                              \
                ::rn::fail(RN_ENOMEM, std::string(#call) + ": " + cudaGetErrorString(e_));    \
            ::rn::fail(RN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
        }                                                                                     \
    } while (0)

// --------------------------------------------------------------- device memory
// Where device memory comes from: the caller's hooks (rn_params alloc /
// dealloc / alloc_ctx), or the stream-ordered pool when alloc is null.
struct Allocator {
    void *(*alloc)(size_t, void *, void *) = nullptr;
    void (*dealloc)(void *, size_t, void *, void *) = nullptr;
    void *ctx = nullptr;
    int pool = -1;  // without hooks: the library's device pool of this slot (-1: the thread's)
};
// The allocator new buffers take on this thread; the API entry points set it
// for the duration of a call (AllocScope) from the call's parameters.
Allocator &current_allocator();
void set_thread_pool(int slot);  // worker threads of batched calls: a device pool per worker (-1: default)
// Merged setups: problem streams kMergedPoolBase + k .. with pools of the same
// index (see merged_stream); the working stream is merged_stream(kMergedStreams).
constexpr int kMergedStreams = 64;
constexpr int kMergedPoolBase = 16;  // above the batched calls' worker slots
cudaStream_t merged_stream(int k);
struct AllocScope {
    Allocator saved;
    explicit AllocScope(const Allocator &a) : saved(current_allocator()) { current_allocator() = a; }
    ~AllocScope() { current_allocator() = saved; }
    AllocScope(const AllocScope &) = delete;
    AllocScope &operator=(const AllocScope &) = delete;
};
// bytes is rounded up (with tail slack) inside; *got receives the size asked of the allocator
void *dmalloc(size_t bytes, cudaStream_t s, const Allocator &a, size_t *got);
void dfree(void *p, size_t got, cudaStream_t s, const Allocator &a);
int64_t allocation_count();  // allocations made so far (dmalloc and page-locked scratch)

// A device buffer; it is freed by the allocator it came from, whatever the
// thread's allocator is at that time.
template <typename T>
struct DVec {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    Allocator a;
    size_t got = 0;
    DVec() = default;
    DVec(size_t n_, cudaStream_t s_) { alloc(n_, s_); }
    void alloc(size_t n_, cudaStream_t s_) {
        release();
        s = s_;
        a = current_allocator();
        p = n_ ? static_cast<T *>(dmalloc(n_ * sizeof(T), s, a, &got)) : nullptr;
        n = n_;
    }
    void release() {
        if (p) dfree(p, got, s, a);
        p = nullptr;
        n = 0;
        got = 0;
    }
    ~DVec() { release(); }
    DVec(const DVec &) = delete;
    DVec &operator=(const DVec &) = delete;
    DVec(DVec &&o) noexcept : p(o.p), n(o.n), s(o.s), a(o.a), got(o.got) { o.p = nullptr; o.n = 0; o.got = 0; }
    DVec &operator=(DVec &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s; a = o.a; got = o.got;
            o.p = nullptr; o.n = 0; o.got = 0;
        }
        return *this;
    }
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// Device CSR owned by the library.  val32 is the FP32 shadow used by the
// mixed-precision cycle.
struct DCsr {
    int32_t n = 0, m = 0;
    int64_t nnz = 0;
    DVec<int32_t> rowptr, col;
    DVec<double> val;
    DVec<float> val32;
    int32_t maxlen = 0;     // longest row (set before solving)
    int tile_group = 0;     // lanes per row of the staged SpMV, FP32 values (0: rows too long, unstaged kernel)
    int tile_group64 = 0;   // the same for FP64 values (smaller stages)
    // optional lists of the staged tiles to process (FP32 / FP64 stages) and
    // their lengths tcnt[0], tcnt[1]; empty: every tile
    DVec<int32_t> tl32, tl64, tcnt;
};

// Borrowed view of a CSR (device pointers).
struct CsrView {
    int32_t n, m;
    int64_t nnz;
    const int32_t *rowptr, *col;
    const double *val;
};
inline CsrView view(const DCsr &a) { return CsrView{a.n, a.m, a.nnz, a.rowptr.p, a.col.p, a.val.p}; }

// --------------------------------------------------------------- launches
int num_sms();
int grid_for(int64_t work_items, int items_per_block, int blocks_per_sm = 8);
// Blocks of `fn` (with this block size and dynamic shared memory) resident on
// one SM, from the occupancy calculator (registers included); cached.
int resident_blocks(const void *fn, int block, size_t smem);
// Grid for a grid-stride kernel: enough blocks for the work, at most one wave
// of resident blocks (and at most cap).
template <typename K>
int grid_resident(K kernel, int block, size_t smem, int64_t work_items, int items_per_block,
                  int cap = 1 << 30) {
    int64_t need = (work_items + items_per_block - 1) / items_per_block;
    const int64_t wave = (int64_t)resident_blocks((const void *)kernel, block, smem) * num_sms();
    if (need > wave) need = wave;
    if (need > cap) need = cap;
    return (int)(need < 1 ? 1 : need);
}

// Profiled launch: records CUDA events around the kernel when profiling is on
// and attributes `bytes` of algorithmic traffic to `name`.
struct ProfScope {
    const char *name;
    double bytes;
    cudaStream_t s;
    int slot = -1;
    ProfScope(const char *name_, double bytes_, cudaStream_t s_);
    ~ProfScope() noexcept(false);
};
void check_launch(const char *name);
bool profiling_enabled();
void add_launches(int64_t k);      // kernels replayed inside a CUDA graph
int64_t launches_so_far();


// Launch with programmatic dependent launch (PDL): the kernel may be
// scheduled while its predecessor in the stream (or graph) is still draining.
// Such kernels call pdl_wait() before they read anything the predecessor
// writes and before their own first global write; on a launch without the
// attribute pdl_wait() returns at once.
template <typename... K, typename... A>
void launch_pdl(const char *name, double bytes, cudaStream_t s, void (*kernel)(K...), dim3 grid, dim3 block,
                size_t smem, A &&...args) {
    ProfScope ps(name, bytes, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
    if (e != cudaSuccess) fail(RN_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
}
#define RN_LAUNCH_PDL(name, bytes, stream, kernel, grid, block, smem, ...) \
    ::rn::launch_pdl((name), (double)(bytes), (stream), kernel, dim3(grid), dim3(block), (size_t)(smem), __VA_ARGS__)
// Every kernel of the library starts with pdl_wait() (or reads nothing a
// predecessor writes before it), so every launch may use programmatic
// dependent launch: in a stream of dependent kernels the next grid is set up
// while the previous one drains (measured on GB300: 4.5 -> 2.3 us per
// dependent launch of a small kernel).
#define RN_LAUNCH(name, bytes, stream, kernel, grid, block, smem, ...) \
    RN_LAUNCH_PDL(name, bytes, stream, kernel, grid, block, smem, __VA_ARGS__)

template <typename T>
void h2d(T *dst, const T *src, size_t n, cudaStream_t s) {
    if (n) RN_CUDA_CHECK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
}
template <typename T>
void d2h(T *dst, const T *src, size_t n, cudaStream_t s) {
    if (n) RN_CUDA_CHECK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, s));
}
template <typename T>
void d2d(T *dst, const T *src, size_t n, cudaStream_t s) {
    if (n) RN_CUDA_CHECK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
}
// This thread's page-locked host scratch (kPinnedBytes): small device->host
// reads land there by DMA, with no staging through the driver's pageable
// buffer, so threads driving independent setups do not serialise on it.
constexpr size_t kPinnedBytes = 1024;
void *pinned_scratch();
// Read n elements (n * sizeof(T) <= kPinnedBytes) and wait for them.
template <typename T>
void read_small(T *dst, const T *dptr, size_t n, cudaStream_t s) {
    if (n * sizeof(T) > kPinnedBytes) fail(RN_EINTERNAL, "read_small: more than the pinned scratch holds");
    T *h = static_cast<T *>(pinned_scratch());
    RN_CUDA_CHECK(cudaMemcpyAsync(h, dptr, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    std::memcpy(dst, h, n * sizeof(T));
}
// Read n elements and wait (through the pinned scratch when they fit, else a
// plain copy into dst).
template <typename T>
void read_vec(T *dst, const T *dptr, size_t n, cudaStream_t s) {
    if (n * sizeof(T) <= kPinnedBytes) {
        read_small(dst, dptr, n, s);
        return;
    }
    RN_CUDA_CHECK(cudaMemcpyAsync(dst, dptr, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
}
template <typename T>
T read_scalar(const T *dptr, cudaStream_t s) {
    T v;
    read_small(&v, dptr, 1, s);
    return v;
}

// --------------------------------------------------------------- primitives (rn_prims.cu)
// Exclusive scan of n int32 counts into out[0..n] (out[n] = total); returns
// the total (one device->host read).  Fails with RN_EINTERNAL if the total
// does not fit in int32.
int64_t scan_counts(const int32_t *counts, int32_t *out, int64_t n, cudaStream_t s);
// The same without the host read: the total goes to *total (device).
void scan_counts_dev(const int32_t *counts, int32_t *out, int64_t n, int64_t *total, cudaStream_t s);
// Deterministic grid reductions: per-block partial sums, summed in block order
// by the last block (see grid_finish).  Grids of reducing kernels never exceed
// kReduceBlocks blocks.
constexpr int kReduceBlocks = 1216;   // partial-sum slots per value (8 x 152 SMs)
struct Fin;
// *result = <x, y>
// y -= (*h) x, then *result = <y, xn> (xn null: <y, y>), bit-identical to the
// axpy and dot() launched apart
void axpy_dot(double *y, const double *x, const double *h, const double *xn, int64_t n, double *result,
              cudaStream_t s, double *partial, unsigned *counter);
void dot(const double *x, const double *y, int64_t n, double *result, cudaStream_t s, double *partial,
         unsigned *counter);
void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s);
void fill_f64(double *p, double v, int64_t n, cudaStream_t s);
// diag[i] = a_ii (fails RN_EINVAL through *bad when a diagonal is missing or zero)
void extract_diag(const CsrView &A, double *diag, int32_t *bad, cudaStream_t s);
// Transpose with sorted rows (values optional).
void transpose(const CsrView &A, bool with_val, DCsr &At, cudaStream_t s);
void to_float(const double *x, float *y, int64_t n, cudaStream_t s);
void to_double(const float *x, double *y, int64_t n, cudaStream_t s);
// g_e = -lam_i x_j for every stored entry e = (i, j) of A (values unused)
void adjoint_grad(const CsrView &A, const double *lam, const double *x, double *g, cudaStream_t s);
// y = 1 / x elementwise (y may be x)
void reciprocal(const double *x, double *y, int64_t n, cudaStream_t s);

// --------------------------------------------------------------- products (rn_spgemm.cu)
// C = A*B in one hash pass per row: the symbolic pattern (explicit zeros kept,
// rows sorted) and the values, each summed in ascending k with a rounded
// multiply then a rounded add (bit-identical to a sequential evaluation).
// fused: each further term added by a fused multiply-add instead (one FP64
// instruction instead of two; the Galerkin products, held to 1e-12 rather
// than bit-exactness), still in ascending k; rows of the sorting kernel keep
// the separate operations.
// b_nnz_dev (optional): B's size on the device (B.nnz then need only bound it:
// the exact value comes back with the first read); err_dev (optional): no
// second read - C is allocated at its bound (C.nnz = the product count, the
// exact size in C.rowptr[n]) and a row past the block kernel's table is
// reported in *err_dev (row + 1, atomic max) for the caller to read later
void spgemm(const CsrView &A, const CsrView &B, DCsr &C, cudaStream_t s, bool fused = false,
            const int32_t *b_nnz_dev = nullptr, int32_t *err_dev = nullptr);

// Energy-minimisation operator on the fixed pattern N shared by X and W:
//   W = scale * Proj(Mask_N(A X)) with A's values aval (TV = double, or float
//   for the mixed-precision sweeps), plus, when Y != nullptr, the Frobenius
//   product <Y, W> reduced into fin.
template <typename TV>
struct ProjArgsT {
    const int32_t *rowtype;  // 0 free, 1 root, 2 unaggregated
    const TV *Bc;            // coarse candidates
    const TV *rs2;           // per row 1 / sum_{j in N_i} Bc_j^2 (proj_scales, FP64; rounded for float)
};
using ProjArgs = ProjArgsT<double>;
// The energy product's gather map for a fixed pattern N (see rn_spgemm.cu):
// built once per minimisation, then each product gathers directly.
struct EpMap {
    DVec<int32_t> base;        // per-row byte offsets (n + 1)
    DVec<unsigned char> map;   // per row: [position in A_i] x [entry of N_i] offsets into N_k
    int64_t bytes = 0;
    int G = 4;
    bool ok = false;
};
// false (and m unusable) when a row of N is too long for byte offsets or the
// map would exceed int32 offsets; the scanning product is then used
bool ep_map_build(EpMap &m, const CsrView &A, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN,
                  const int32_t *rowtype, cudaStream_t s);
template <typename TV>
void masked_product_mapped(const EpMap &m, const CsrView &A, const TV *aval, const int32_t *nrowptr,
                           const int32_t *ncol, int64_t nnzN, int32_t nc, const TV *X, TV *W, const ProjArgsT<TV> &pa,
                           double scale, const TV *Y, const Fin &fin, cudaStream_t s);
// The energy product on a sliced plan (see rn_spgemm.cu), built once per
// minimisation.  Rows go in slices of 32 / G consecutive rows, one warp per
// slice and G lanes per row; lane l of row i owns A_i's entries l, l + G, ...
// Per slice the plan stores, interleaved so that the warp's 32 lanes read 32
// consecutive words: A's values in the sweeps' type (pa), the start of the
// neighbour's pattern row nrp[k] (pb), and the positions of row i's pattern
// columns in N_k (pm): `bits` bits each (4 when every row of N has at most 15
// entries, else 8; all ones: absent), wps[s] words per A entry, the same for
// the whole slice (enough for its longest row), so that entry q of a row is
// always bit field q % (32 / bits) of word q / (32 / bits).
// rinfo[i] = steps | len << 16 (steps = ceil(|A_i| / G), 0 for rows the
// operator zeroes; len = |N_i|); bq[q] = Bc at the entry's column and de[q] =
// the row's D^{-1} (or 1 without preconditioning), per pattern entry, for the
// projection and for the elementwise CG kernels.
template <typename TV>
struct EpPlan {
    DVec<int32_t> aoff, moff, wps, slen, rinfo, pb;  // slen: per slice, the longest kept row of N
    DVec<TV> pa, bq, de;
    DVec<uint32_t> pm;
    int G = 1, S = 4, bits = 8;
    int64_t slots = 0, words = 0;
    bool ok = false;
};
// false (plan unusable) when a row of N is longer than 16 entries, a row N_k
// longer than 254, or the plan's offsets would pass int32: the caller then
// uses the gather map or the scanning product.  dinv may be null (no
// preconditioning: de = 1).
template <typename TV>
bool ep_plan_build(EpPlan<TV> &p, const CsrView &A, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN,
                   const int32_t *rowtype, const double *Bc, const double *dinv, cudaStream_t s);
// W = scale * Proj(Mask_N(A X)) (and <Y, W> into fin when Y != null) on the plan
template <typename TV>
void masked_product_plan(const EpPlan<TV> &p, int32_t n, const int32_t *nrowptr, int64_t nnzN, const TV *X, TV *W,
                         const TV *rs2, double scale, const TV *Y, const Fin &fin, cudaStream_t s);
// rs2 for ProjArgs: the row projection's scale on pattern N (n rows)
void proj_scales(int32_t n, const int32_t *nrowptr, const int32_t *ncol, int64_t nnzN, const int32_t *rowtype,
                 const double *Bc, double *rs2, cudaStream_t s);
template <typename TV>
void masked_product_proj(const CsrView &A, const TV *aval, const int32_t *nrowptr, const int32_t *ncol,
                         int64_t nnzN, int32_t nc, const TV *X, TV *W, const ProjArgsT<TV> &pa, double scale,
                         const TV *Y, const Fin &fin, cudaStream_t s);

// --------------------------------------------------------------- misc
std::string fmt(const char *f, ...);
double now_ms();

}  // namespace rn

#include "rn_device.cuh"
