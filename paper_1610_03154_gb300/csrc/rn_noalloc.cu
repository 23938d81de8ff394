// rn_noalloc.cu - rn_energy_min_noalloc: the CG energy minimisation of
// rn_energy_min with all of its scratch memory in one statically allocated
// device array instead of the stream-ordered allocator.
//
// Who needs it: callers that must not allocate device memory while they run.
// Examples are a host framework whose own caching allocator has reserved the
// GPU's memory (a library cudaMalloc would fail or fragment that reserve), a
// latency-critical loop in which an allocation's implicit synchronisation or
// pool growth is not acceptable, and plugin hosts that forbid libraries from
// allocating.  Such a caller still passes every input and output buffer; this
// entry point then makes no allocation call of any kind.
//
// The array below is created when the library is loaded and every GPU that
// loads the library keeps it until the process exits.  All calls share it:
// calls whose GPU work overlaps (on different streams, or from different
// threads) race on it and must be serialised by the caller.  The call reads
// one flag back to the host and synchronises its stream before it returns.
#include <mutex>

#include "rn_hier.cuh"

namespace rn {
namespace {

// Limits of the static scratch (stated in include/rn.h as well).
constexpr int64_t kNaMaxRows = 1 << 18;      // rows of A
constexpr int64_t kNaMaxPattern = 1 << 19;   // entries of the pattern N

// Layout (bytes, each region 256-byte aligned): the inverted diagonal D^{-1}
// (one double per row), CG's residual R, direction Dd and product W (one
// double per pattern entry each), the row projection's scales (one double per
// row), the reduction partials (two per reducing block), the CG scalars, the
// reduction's arrival counters and the flags.  This is the only device memory
// the call uses besides the caller's buffers: the minimisation runs with FP64
// sweeps, k = 1 and products that scan the pattern rows (no gather map), a
// path that allocates nothing once these workspaces are supplied.
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffDiag = 0;
constexpr size_t kOffR = align_up(kOffDiag + sizeof(double) * kNaMaxRows);
constexpr size_t kOffD = align_up(kOffR + sizeof(double) * kNaMaxPattern);
constexpr size_t kOffW = align_up(kOffD + sizeof(double) * kNaMaxPattern);
constexpr size_t kOffS2 = align_up(kOffW + sizeof(double) * kNaMaxPattern);
constexpr size_t kOffPartial = align_up(kOffS2 + sizeof(double) * kNaMaxRows);
constexpr size_t kOffSc = align_up(kOffPartial + sizeof(double) * 2 * kReduceBlocks);
constexpr size_t kOffCounter = align_up(kOffSc + sizeof(double) * 64);
constexpr size_t kOffFlags = align_up(kOffCounter + sizeof(unsigned) * 4);
constexpr size_t kScratchBytes = align_up(kOffFlags + sizeof(int32_t) * 16) + kAlign;  // + tail slack

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, resolved on the first call made
// with that device current.
std::mutex g_mu;
void *g_addr[64] = {nullptr};

unsigned char *scratch_address() {
    int dev = 0;
    RN_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(RN_EINVAL, "device index out of range for the static scratch table");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            fail(RN_ECUDA, fmt("cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e)));
        g_addr[dev] = p;
    }
    return static_cast<unsigned char *>(g_addr[dev]);
}

}  // namespace
}  // namespace rn

extern "C" rn_status rn_energy_min_noalloc(const rn_csr *A, const rn_csr *N, const int32_t *rowtype, const double *Bc,
                                           double *P, int sweeps, int precond, void *stream) {
    try {
        using namespace rn;
        if (!A || !N || !rowtype || !Bc || !P) fail(RN_EINVAL, "null argument");
        if (A->n_rows <= 0 || A->n_rows != A->n_cols || !A->rowptr || !A->col || !A->val) fail(RN_EINVAL, "A");
        if (A->nnz <= 0 || A->nnz > INT32_MAX - 1) fail(RN_EINVAL, "nnz(A) out of range");
        if (N->n_rows != A->n_rows || N->n_cols < 1 || N->nnz < 0 || !N->rowptr || (N->nnz > 0 && !N->col))
            fail(RN_EINVAL, "pattern N does not match A");
        if (A->n_rows > kNaMaxRows)
            fail(RN_EINVAL, fmt("rn_energy_min_noalloc: %d rows exceed the static scratch limit of %lld rows",
                                A->n_rows, (long long)kNaMaxRows));
        if (N->nnz > kNaMaxPattern)
            fail(RN_EINVAL, fmt("rn_energy_min_noalloc: %lld pattern entries exceed the static scratch limit of "
                                "%lld entries", (long long)N->nnz, (long long)kNaMaxPattern));
        if (sweeps < 0 || sweeps > 1000) fail(RN_EINVAL, "sweeps must be in [0, 1000]");
        // NULL means the legacy default stream here: creating a stream is
        // also something this entry point does not do.
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        unsigned char *base = scratch_address();
        double *diag = reinterpret_cast<double *>(base + kOffDiag);
        double *sc = reinterpret_cast<double *>(base + kOffSc);
        unsigned *counter = reinterpret_cast<unsigned *>(base + kOffCounter);
        int32_t *fl = reinterpret_cast<int32_t *>(base + kOffFlags);
        // the array keeps the previous call's contents: zero what must start at zero
        RN_CUDA_CHECK(cudaMemsetAsync(base + kOffSc, 0, kOffFlags + sizeof(int32_t) * 16 - kOffSc, s));
        const int32_t n = A->n_rows;
        CsrView Av{n, n, A->nnz, A->rowptr, A->col, A->val};
        extract_diag(Av, diag, fl + 4, s);
        // the flag is read into this stack variable (pageable: the library's
        // page-locked read slots may not exist yet on this thread)
        int32_t bad = 0;
        RN_CUDA_CHECK(cudaMemcpyAsync(&bad, fl + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        RN_CUDA_CHECK(cudaStreamSynchronize(s));
        if (bad) fail(RN_EINVAL, "missing or zero diagonal");
        EmCtx c;
        c.s = s;
        c.partial = reinterpret_cast<double *>(base + kOffPartial);
        c.counter = counter;
        c.sc = sc;
        c.fl = fl;
        c.precond = precond ? 1 : 0;
        c.method = RN_ENERGY_CG;
        c.R = reinterpret_cast<double *>(base + kOffR);
        c.Dd = reinterpret_cast<double *>(base + kOffD);
        c.W = reinterpret_cast<double *>(base + kOffW);
        c.rs2 = reinterpret_cast<double *>(base + kOffS2);
        c.scan_only = true;  // no gather map: the products scan the pattern rows
        Pattern pat{n, N->n_cols, N->nnz, N->rowptr, N->col};
        reciprocal(diag, diag, n, s);  // the preconditioner D^{-1}, in place
        energy_min(c, Av, pat, P, rowtype, Bc, diag, sweeps);
        RN_CUDA_CHECK(cudaStreamSynchronize(s));
        return RN_OK;
    } catch (const rn::Error &e) {
        rn::set_last_error(e.msg);
        return e.status;
    } catch (...) {
        rn::set_last_error("unexpected internal exception");
        return RN_EINTERNAL;
    }
}
