// rn_prims.cu - allocator, profiling, scan, deterministic reductions,
// transpose and small elementwise kernels.
#include <atomic>
#include <cstdarg>
#include <chrono>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "rn_internal.cuh"

namespace rn {

// --------------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }
const std::string &last_error_ref() { return g_last_error; }

[[noreturn]] void fail(rn_status s, const std::string &msg) { throw Error{s, msg}; }

std::string fmt(const char *f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return std::string(buf);
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// --------------------------------------------------------------------- memory

// Allocations the library has made in this process (device buffers through
// dmalloc, page-locked host scratch through pinned_scratch); read by
// rn_allocation_count.
static std::atomic<int64_t> g_allocations{0};
int64_t allocation_count() { return g_allocations.load(); }

// Pinned scratch: slots of one page-locked pool (allocated once, kept for the
// process), one per thread; threads past the pool's slots get their own.
void *pinned_scratch() {
    constexpr int kSlots = 256;
    static unsigned char *pool = nullptr;
    static std::once_flag once;
    static std::atomic<int> next{0};
    thread_local void *mine = nullptr;
    if (mine) return mine;
    std::call_once(once, [] {
        void *p = nullptr;
        g_allocations++;
        if (cudaMallocHost(&p, kSlots * kPinnedBytes) == cudaSuccess) pool = static_cast<unsigned char *>(p);
    });
    const int k = next++;
    if (pool && k < kSlots) {
        mine = pool + (size_t)k * kPinnedBytes;
    } else {
        void *p = nullptr;  // kept for the thread's life (and the process's: a few bytes)
        g_allocations++;
        RN_CUDA_CHECK(cudaMallocHost(&p, kPinnedBytes));
        mine = p;
    }
    return mine;
}

Allocator &current_allocator() {
    thread_local Allocator a;
    return a;
}

// Host threads driving independent setups allocate from pools of their own
// (slot = worker index), so they do not contend on the default pool.
static thread_local int t_pool_slot = -1;
void set_thread_pool(int slot) { t_pool_slot = slot; }
static cudaMemPool_t slot_pool(int slot) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    while ((int)pools.size() <= slot) {
        int dev = 0;
        RN_CUDA_CHECK(cudaGetDevice(&dev));
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t mp;
        RN_CUDA_CHECK(cudaMemPoolCreate(&mp, &props));
        uint64_t thr = UINT64_MAX;
        RN_CUDA_CHECK(cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr));
        pools.push_back(mp);
    }
    return pools[slot];
}

// Streams of the hierarchies that merged setups build, kept for the process:
// stream k is used with pool kMergedPoolBase + k and no other, because a
// stream-ordered pool holding blocks freed on many streams is slow to
// allocate from (measured on GB300: 43 us per allocation after frees on 64
// streams, 5.7 us on 8, 1.0 us on one).
cudaStream_t merged_stream(int k) {
    static std::mutex mu;
    static std::vector<cudaStream_t> st;
    std::lock_guard<std::mutex> lk(mu);
    while ((int)st.size() <= k) {
        cudaStream_t s = nullptr;
        RN_CUDA_CHECK(cudaStreamCreate(&s));
        st.push_back(s);
    }
    return st[k];
}

void *dmalloc(size_t bytes, cudaStream_t s, const Allocator &a, size_t *got) {
    // every buffer gets >= 256 bytes of tail slack: the tile kernels copy CSR
    // segments with 16-byte-granular bulk copies that may end up to 15 bytes
    // past the last element (the slack is never interpreted)
    bytes = ((bytes + 255) / 256) * 256 + 256;
    *got = bytes;
    g_allocations++;
    if (a.alloc) {
        void *p = a.alloc(bytes, (void *)s, a.ctx);
        if (!p) fail(RN_ENOMEM, fmt("the caller's allocator returned NULL for %zu bytes", bytes));
        if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {  // bulk copies and vector loads need alignment
            a.dealloc(p, bytes, (void *)s, a.ctx);
            fail(RN_EINVAL, "the caller's allocator returned memory not aligned to 256 bytes");
        }
        return p;
    }
    static const bool pool_configured = [] {
        // keep freed blocks cached in the device's default pool: setup makes
        // many short-lived allocations (once; thread-safe static initialisation)
        int dev = 0;
        RN_CUDA_CHECK(cudaGetDevice(&dev));
        cudaMemPool_t pool;
        RN_CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t thr = UINT64_MAX;
        RN_CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        return true;
    }();
    (void)pool_configured;
    void *p = nullptr;
    const int slot = a.pool >= 0 ? a.pool : t_pool_slot;
    cudaError_t e = slot >= 0 ? cudaMallocFromPoolAsync(&p, bytes, slot_pool(slot), s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? RN_ENOMEM : RN_ECUDA,
             fmt("cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e)));
    }
    return p;
}

void dfree(void *p, size_t got, cudaStream_t s, const Allocator &a) {
    if (!p) return;
    if (a.alloc) a.dealloc(p, got, (void *)s, a.ctx);
    else cudaFreeAsync(p, s);
}

// --------------------------------------------------------------------- launch helpers
int num_sms() {
    static const int sms = [] {  // thread-safe static initialisation
        int dev = 0, v = 0;
        RN_CUDA_CHECK(cudaGetDevice(&dev));
        RN_CUDA_CHECK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        return v;
    }();
    return sms;
}

int grid_for(int64_t work_items, int items_per_block, int blocks_per_sm) {
    int64_t need = (work_items + items_per_block - 1) / items_per_block;
    int64_t cap = (int64_t)num_sms() * blocks_per_sm;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

int resident_blocks(const void *fn, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t, int>, int> cache;
    int dev = 0;
    RN_CUDA_CHECK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(fn, block, smem, dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    RN_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem));
    if (per_sm < 1) per_sm = 1;
    cache[key] = per_sm;
    return per_sm;
}

void check_launch(const char *name) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(RN_ECUDA, fmt("launch of %s: %s", name, cudaGetErrorString(e)));
}

// --------------------------------------------------------------------- profiling
struct Pending {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
};
struct KStat {
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
};
static bool g_prof_on = false;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_event_pool;
static std::map<std::string, KStat> g_stats;
static std::mutex g_prof_mu;

bool profiling_enabled() { return g_prof_on; }

static cudaEvent_t get_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    RN_CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

static void drain_pending() {
    for (auto &p : g_pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        KStat &k = g_stats[p.name];
        k.launches++;
        k.ms += ms;
        k.bytes += p.bytes;
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
}

static std::atomic<int64_t> g_launches{0};
void add_launches(int64_t k) { g_launches += k; }
int64_t launches_so_far() { return g_launches.load(); }

ProfScope::ProfScope(const char *name_, double bytes_, cudaStream_t s_) : name(name_), bytes(bytes_), s(s_) {
    g_launches++;
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    Pending p{name, bytes, get_event(), get_event()};
    cudaEventRecord(p.a, s);
    g_pending.push_back(p);
    slot = (int)g_pending.size() - 1;
    if (g_pending.size() > 4096) {
        // keep the pending list bounded (this synchronises the recorded events)
        cudaEventRecord(g_pending.back().b, s);
        Pending last = g_pending.back();
        g_pending.pop_back();
        drain_pending();
        g_pending.push_back(last);
        slot = 0;
    }
}

ProfScope::~ProfScope() noexcept(false) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].b, s);
}

}  // namespace rn

extern "C" int64_t rn_kernel_launches(void) { return rn::launches_so_far(); }
extern "C" int64_t rn_allocation_count(void) { return rn::allocation_count(); }

extern "C" rn_status rn_profile_enable(int on) {
    rn::g_prof_on = (on != 0);
    return RN_OK;
}

extern "C" rn_status rn_profile_reset(void) {
    std::lock_guard<std::mutex> lk(rn::g_prof_mu);
    rn::drain_pending();
    rn::g_stats.clear();
    return RN_OK;
}

extern "C" rn_status rn_profile_read(rn_kernel_stat *out, int max, int *count) {
    std::lock_guard<std::mutex> lk(rn::g_prof_mu);
    rn::drain_pending();
    int c = 0;
    for (auto &kv : rn::g_stats) {
        if (out && c < max) {
            snprintf(out[c].name, sizeof out[c].name, "%s", kv.first.c_str());
            out[c].launches = kv.second.launches;
            out[c].ms = kv.second.ms;
            out[c].bytes = kv.second.bytes;
        }
        c++;
    }
    if (count) *count = c;
    return RN_OK;
}

namespace rn {

// --------------------------------------------------------------------- scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

// exclusive block scan of one int64 per thread; returns the block total
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *out_excl, int64_t *smem) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        smem[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    int64_t warp_off = (w > 0) ? smem[w - 1] : 0;
    int64_t total = smem[(blockDim.x >> 5) - 1];
    *out_excl = warp_off + x - v;
    __syncthreads();
    return total;
}

// Single-pass exclusive scan with decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016): tiles of
// kScanChunk counts are claimed in order through a ticket, so every tile a
// block waits on belongs to a block that is already running; each tile
// publishes its sum, then its inclusive prefix, in one word of tile_state
// (flag in the top two bits).  A block that has waited kScanMaxSpin polls
// for a predecessor sums the raw counts before its tile instead, so the scan
// always ends.
constexpr unsigned long long kScanAgg = 1ull << 62, kScanPre = 2ull << 62, kScanVal = (1ull << 62) - 1;
constexpr uint32_t kScanMaxSpin = 1u << 22;

__global__ void __launch_bounds__(kScanThreads)
scan_onepass_kernel(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ out, int64_t *__restrict__ total,
                    unsigned long long *__restrict__ state, unsigned int *__restrict__ ticket, int64_t ntiles) {
    pdl_wait();
    __shared__ int64_t smem[32];
    __shared__ unsigned int tile_sh;
    __shared__ int64_t excl_sh;
    __shared__ int gave_up;
    if (threadIdx.x == 0) {
        tile_sh = atomicAdd(ticket, 1u);
        gave_up = 0;
    }
    __syncthreads();
    const int64_t tile = tile_sh;
    const int64_t base = tile * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int32_t vals[kScanItems];
    int64_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        vals[k] = (base + k < n) ? in[base + k] : 0;
        v += vals[k];
    }
    int64_t ex;
    const int64_t agg = block_exclusive_scan(v, &ex, smem);
    if (threadIdx.x == 0) {
        int64_t pre = 0;
        if (tile == 0) {
            atomicExch(&state[0], kScanPre | (unsigned long long)agg);
        } else {
            atomicExch(&state[tile], kScanAgg | (unsigned long long)agg);
            const volatile unsigned long long *st = state;
            for (int64_t j = tile - 1; j >= 0; j--) {
                unsigned long long w = st[j];
                for (uint32_t spin = 0; (w >> 62) == 0 && spin < kScanMaxSpin; spin++) {
                    __nanosleep(64);
                    w = st[j];
                }
                if ((w >> 62) == 0) {
                    gave_up = 1;
                    break;
                }
                pre += (int64_t)(w & kScanVal);
                if ((w >> 62) == 2) break;
            }
            if (!gave_up) atomicExch(&state[tile], kScanPre | (unsigned long long)(pre + agg));
        }
        excl_sh = pre;
    }
    __syncthreads();
    if (gave_up) {  // sum every count before this tile directly
        int64_t t = 0;
        for (int64_t i = threadIdx.x; i < tile * kScanChunk; i += blockDim.x) t += in[i];
        int64_t dummy;
        const int64_t pre = block_exclusive_scan(t, &dummy, smem);
        if (threadIdx.x == 0) {
            excl_sh = pre;
            atomicExch(&state[tile], kScanPre | (unsigned long long)(pre + agg));
        }
        __syncthreads();
    }
    int64_t run = excl_sh + ex;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = (int32_t)run;
        run += vals[k];
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) {
        out[n] = (int32_t)(excl_sh + agg);
        *total = excl_sh + agg;
    }
}

void scan_counts_dev(const int32_t *counts, int32_t *out, int64_t n, int64_t *total, cudaStream_t s) {
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb < 1) nb = 1;
    DVec<unsigned long long> st(nb + 1, s);  // tile words, then the ticket
    RN_CUDA_CHECK(cudaMemsetAsync(st.p, 0, st.bytes(), s));
    RN_LAUNCH("scan", 8.0 * n, s, scan_onepass_kernel, (int)nb, kScanThreads, 0, counts, n, out, total, st.p,
              reinterpret_cast<unsigned int *>(st.p + nb), nb);
}

int64_t scan_counts(const int32_t *counts, int32_t *out, int64_t n, cudaStream_t s) {
    DVec<int64_t> total(1, s);
    scan_counts_dev(counts, out, n, total.p, s);
    int64_t t = read_scalar(total.p, s);
    if (t > INT32_MAX) fail(RN_EINTERNAL, fmt("scan total %lld exceeds int32", (long long)t));
    return t;
}

// --------------------------------------------------------------------- reductions
constexpr int kRedThreads = 256;

__global__ void dot_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n, Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    double v[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[0] = fma(x[i], y[i], v[0]);
    grid_finish<kRedThreads, 1>(v, fin, sm);
}

void dot(const double *x, const double *y, int64_t n, double *result, cudaStream_t s, double *partial,
         unsigned *counter) {
    const int nb = grid_resident((const void *)dot_kernel, kRedThreads, 0, n, kRedThreads * 4, kReduceBlocks);
    Fin f;
    f.mode = FIN_STORE;
    f.partial = partial;
    f.counter = counter;
    f.out = result;
    RN_LAUNCH("dot", 16.0 * n, s, dot_kernel, nb, kRedThreads, 0, x, y, n, f);
}

// y -= (*h) x, then <y, xn> of the updated y (xn null: <y, y>): one step of
// modified Gram-Schmidt fused with the next projection (or the norm).  The update is the same
// expression as a separate axpy and the sum is formed as dot() forms it (same
// grid, per-thread order and block-order finish), so the results are the
// same bits as the two launches.
__global__ void axpy_dot_kernel(double *__restrict__ y, const double *__restrict__ x, const double *__restrict__ h,
                                const double *__restrict__ xn, int64_t n, Fin fin) {
    pdl_wait();
    __shared__ double sm[32];
    const double c = *h;
    double v[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double yi = y[i] - c * x[i];
        y[i] = yi;
        v[0] = fma(yi, xn ? xn[i] : yi, v[0]);
    }
    grid_finish<kRedThreads, 1>(v, fin, sm);
}

void axpy_dot(double *y, const double *x, const double *h, const double *xn, int64_t n, double *result,
              cudaStream_t s, double *partial, unsigned *counter) {
    const int nb = grid_resident((const void *)dot_kernel, kRedThreads, 0, n, kRedThreads * 4, kReduceBlocks);
    Fin f;
    f.mode = FIN_STORE;
    f.partial = partial;
    f.counter = counter;
    f.out = result;
    RN_LAUNCH("outer_gmres_vec", 32.0 * n, s, axpy_dot_kernel, nb, kRedThreads, 0, y, x, h, xn, n, f);
}

// --------------------------------------------------------------------- elementwise
__global__ void fill_i32_kernel(int32_t *p, int32_t v, int64_t n) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void fill_f64_kernel(double *p, double v, int64_t n) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void to_float_kernel(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    RN_LAUNCH("fill", 4.0 * n, s, fill_i32_kernel, grid_for(n, 1024), 256, 0, p, v, n);
}
void fill_f64(double *p, double v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    RN_LAUNCH("fill", 8.0 * n, s, fill_f64_kernel, grid_for(n, 1024), 256, 0, p, v, n);
}
// Gradient of a loss through x = A^{-1} b with respect to A's stored values:
// dL/dA_ij = -lambda_i x_j (lambda = A^{-T} dL/dx), one value per stored
// entry.  Warp per row; the row's entries are contiguous, so the lanes'
// stores coalesce.
__global__ void adjoint_grad_kernel(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                    const double *__restrict__ lam, const double *__restrict__ x,
                                    double *__restrict__ g) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int32_t i = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < n;
         i += (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5)) {
        const double li = lam[i];
        for (int32_t e = rp[i] + lane; e < rp[i + 1]; e += 32) g[e] = -li * x[col[e]];
    }
}
void adjoint_grad(const CsrView &A, const double *lam, const double *x, double *g, cudaStream_t s) {
    if (A.n <= 0) return;
    RN_LAUNCH("adjoint_grad", 16.0 * A.nnz + 4.0 * (A.n + 1) + 16.0 * A.n, s, adjoint_grad_kernel,
              grid_for((int64_t)A.n * 32, 256), 256, 0, A.n, A.rowptr, A.col, lam, x, g);
}

__global__ void to_double_kernel(int64_t n, const float *x, double *y) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}
void to_double(const float *x, double *y, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    RN_LAUNCH("to_double", 12.0 * n, s, to_double_kernel, grid_for(n, 1024), 256, 0, n, x, y);
}

__global__ void reciprocal_kernel(int64_t n, const double *x, double *y) {
    pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = 1.0 / x[i];
}
void reciprocal(const double *x, double *y, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    RN_LAUNCH("reciprocal", 16.0 * n, s, reciprocal_kernel, grid_for(n, 1024), 256, 0, n, x, y);
}

void to_float(const double *x, float *y, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    RN_LAUNCH("to_float", 12.0 * n, s, to_float_kernel, grid_for(n, 1024), 256, 0, x, y, n);
}

__global__ void extract_diag_kernel(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                    const double *__restrict__ val, double *__restrict__ diag, int32_t *bad) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        int found = 0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (col[e] == i) { d = val[e]; found = 1; }
        diag[i] = d;
        if (!found || d == 0.0) atomicMax(bad, i + 1);
    }
}

void extract_diag(const CsrView &A, double *diag, int32_t *bad, cudaStream_t s) {
    RN_LAUNCH("extract_diag", 12.0 * A.nnz + 12.0 * A.n, s, extract_diag_kernel, grid_for(A.n, 256), 256, 0, A.n,
              A.rowptr, A.col, A.val, diag, bad);
}

// --------------------------------------------------------------------- transpose
__global__ void count_cols_kernel(int64_t nnz, const int32_t *__restrict__ col, int32_t *__restrict__ cnt) {
    pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[e]], 1);
}

__global__ void transpose_scatter_kernel(int32_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                         const double *__restrict__ val, int32_t *__restrict__ next,
                                         int32_t *__restrict__ tcol, double *__restrict__ tval) {
    pdl_wait();
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int32_t pos = atomicAdd(&next[col[e]], 1);
            tcol[pos] = i;
            if (val) tval[pos] = val[e];
        }
    }
}

// warp per output row: rank sort of the (unique) row indices of the segment
__global__ void segment_rank_sort_kernel(int32_t m, const int32_t *__restrict__ rowptr,
                                         const int32_t *__restrict__ kin, const double *__restrict__ vin,
                                         int32_t *__restrict__ kout, double *__restrict__ vout) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += (gridDim.x * blockDim.x) >> 5) {
        int32_t s = rowptr[r], t = rowptr[r + 1];
        for (int32_t e = s + lane; e < t; e += 32) {
            int32_t key = kin[e];
            int32_t rank = 0;
            for (int32_t f = s; f < t; f++) rank += (kin[f] < key);
            kout[s + rank] = key;
            if (vin) vout[s + rank] = vin[e];
        }
    }
}

void transpose(const CsrView &A, bool with_val, DCsr &At, cudaStream_t s) {
    At.n = A.m;
    At.m = A.n;
    At.nnz = A.nnz;
    DVec<int32_t> cnt(A.m + 1, s);
    fill_i32(cnt.p, 0, A.m + 1, s);
    if (A.nnz)
        RN_LAUNCH("transpose", 4.0 * A.nnz, s, count_cols_kernel, grid_for(A.nnz, 1024), 256, 0, A.nnz, A.col, cnt.p);
    At.rowptr.alloc(A.m + 1, s);
    DVec<int64_t> tot(1, s);  // the total is A.nnz: nothing to read back
    scan_counts_dev(cnt.p, At.rowptr.p, A.m, tot.p, s);
    DVec<int32_t> next(A.m, s), tcol(A.nnz, s);
    DVec<double> tval;
    if (with_val) tval.alloc(A.nnz, s);
    d2d(next.p, At.rowptr.p, A.m, s);
    if (A.nnz)
        RN_LAUNCH("transpose", 16.0 * A.nnz, s, transpose_scatter_kernel, grid_for(A.n, 256), 256, 0, A.n, A.rowptr,
                  A.col, with_val ? A.val : nullptr, next.p, tcol.p, tval.p);
    At.col.alloc(A.nnz, s);
    if (with_val) At.val.alloc(A.nnz, s);
    if (A.nnz)
        RN_LAUNCH("transpose", 24.0 * A.nnz, s, segment_rank_sort_kernel, grid_for((int64_t)A.m * 32, 256), 256, 0,
                  A.m, At.rowptr.p, tcol.p, with_val ? tval.p : nullptr, At.col.p, with_val ? At.val.p : nullptr);
}

}  // namespace rn
