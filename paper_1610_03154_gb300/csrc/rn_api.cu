// rn_api.cu - the extern "C" entry points declared in include/rn.h.
// Each entry point converts internal errors (rn::Error) into status codes and
// records a thread-local message; nothing aborts.
#include <cstring>
#include <string>
#include <vector>
#include <atomic>
#include <thread>

#include "rn_hier.cuh"

namespace rn {
const std::string &last_error_ref();
}

rn_hierarchy::~rn_hierarchy() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    if (cg_exec) cudaGraphExecDestroy(cg_exec);
    if (cg_graph) cudaGraphDestroy(cg_graph);
}

#define RN_API_BEGIN try {
#define RN_API_END                                                          \
    }                                                                       \
    catch (const rn::Error &e) {                                            \
        rn::set_last_error(e.msg);                                          \
        return e.status;                                                    \
    }                                                                       \
    catch (const std::bad_alloc &) {                                        \
        rn::set_last_error("host allocation failed");                       \
        return RN_ENOMEM;                                                   \
    }                                                                       \
    catch (...) {                                                           \
        rn::set_last_error("unexpected internal exception");                \
        return RN_EINTERNAL;                                                \
    }

extern "C" rn_status rn_default_params(rn_params *p) {
    if (!p) return RN_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->soc_theta = 0.25;
    p->soc_theta_coarse = -1.0;
    p->degree = 2;
    p->n_sweeps = 4;
    p->energy_method = RN_ENERGY_CG;
    p->energy_precond = 1;
    p->prefilter = 0.0;
    p->postfilter = 0.0;
    p->max_coarse = 64;
    p->max_levels = 25;
    p->b_sweeps = 4;
    p->omega = 2.0 / 3.0;
    p->seed = 12345;
    p->symmetric = 1;
    p->nu_pre = 1;
    p->nu_post = 1;
    p->precision = RN_FP64;
    p->outer = RN_OUTER_CG;
    p->restart = 30;
    p->use_graphs = 1;
    p->keep_aux = 0;
    p->coarse_cluster = 0;
    p->gamma = 1;
    p->soc_kind = RN_SOC_SYMMETRIC;
    p->block_size = 1;
    p->autotune = 0;
    p->stream = nullptr;
    return RN_OK;
}

static void check_params(const rn_params *p) {
    using rn::fail;
    if (p->degree < 0 || p->degree > 16) fail(RN_EINVAL, "degree must be in [0, 16]");
    if (p->n_sweeps < 0 || p->n_sweeps > 1000) fail(RN_EINVAL, "n_sweeps must be in [0, 1000]");
    if (p->energy_method != RN_ENERGY_CG && p->energy_method != RN_ENERGY_GMRES) fail(RN_EINVAL, "energy_method");
    if (p->max_levels < 1) fail(RN_EINVAL, "max_levels must be >= 1");
    if (p->max_coarse < 1) fail(RN_EINVAL, "max_coarse must be >= 1");
    if (p->b_sweeps < 0) fail(RN_EINVAL, "b_sweeps must be >= 0");
    if (p->nu_pre < 0 || p->nu_post < 0) fail(RN_EINVAL, "nu_pre/nu_post must be >= 0");
    if (p->precision != RN_FP64 && p->precision != RN_MIXED) fail(RN_EINVAL, "precision");
    if (p->outer < RN_OUTER_STATIONARY || p->outer > RN_OUTER_FGMRES) fail(RN_EINVAL, "outer");
    if (p->outer == RN_OUTER_FGMRES && (p->restart < 1 || p->restart > 1000)) fail(RN_EINVAL, "restart");
    if (!(p->omega > 0.0)) fail(RN_EINVAL, "omega must be > 0");
    if (p->coarse_cluster < 0) fail(RN_EINVAL, "coarse_cluster must be >= 0");
    if (p->autotune != 0 && p->autotune != 1) fail(RN_EINVAL, "autotune must be 0 or 1");
    if (p->gamma != 1 && p->gamma != 2) fail(RN_EINVAL, "gamma must be 1 (V-cycle) or 2 (W-cycle)");
    if (p->soc_kind != RN_SOC_SYMMETRIC && p->soc_kind != RN_SOC_CLASSICAL) fail(RN_EINVAL, "soc_kind");
    if (p->block_size < 1 || p->block_size > RN_MAX_BLOCK) fail(RN_EINVAL, "block_size must be in [1, RN_MAX_BLOCK]");
    if ((p->alloc == nullptr) != (p->dealloc == nullptr))
        fail(RN_EINVAL, "alloc and dealloc must both be set or both be NULL");
}

static rn::Allocator alloc_of(const rn_params &p) {
    rn::Allocator a;
    a.alloc = p.alloc;
    a.dealloc = p.dealloc;
    a.ctx = p.alloc_ctx;
    return a;
}
// a hierarchy's allocator: its params' hooks, else its device pool
static rn::Allocator alloc_of(const rn_hierarchy &h) {
    rn::Allocator a = alloc_of(h.p);
    a.pool = h.pool;
    return a;
}

extern "C" rn_status rn_setup(const rn_csr *A, const double *B, const double *Bhat, int k, int location,
                              const rn_params *p, rn_hierarchy **out) {
    if (out) *out = nullptr;
    RN_API_BEGIN
    using rn::fail;
    if (!A || !B || !p || !out) fail(RN_EINVAL, "null argument");
    if (k < 1 || k > RN_MAX_CANDIDATES) fail(RN_EINVAL, "k must be in [1, RN_MAX_CANDIDATES]");
    if (p && (p->block_size > k || (p->block_size >= 1 && A->n_rows % p->block_size != 0)))
        fail(RN_EINVAL, "block_size must divide n and not exceed k");
    if (location != RN_DEVICE && location != RN_HOST) fail(RN_EINVAL, "location");
    if (A->n_rows <= 0 || A->n_rows != A->n_cols) fail(RN_EINVAL, "A must be square and non-empty");
    if (A->nnz <= 0 || A->nnz > INT32_MAX - 1) fail(RN_EINVAL, "nnz out of range");
    if (!A->rowptr || !A->col || !A->val) fail(RN_EINVAL, "null CSR array");
    check_params(p);
    if (!p->symmetric && !Bhat) fail(RN_EINVAL, "nonsymmetric setup needs Bhat");
    const rn::AllocScope alloc_scope(alloc_of(*p));  // every buffer of the hierarchy comes from p's hooks
    // With no stream given, work goes to a stream the hierarchy creates: a
    // blocking stream, so it stays ordered with the legacy default stream,
    // and unlike that stream it can be captured into a CUDA graph.
    struct StreamGuard {
        cudaStream_t s = nullptr;
        ~StreamGuard() {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
        }
    } own;
    cudaStream_t s = static_cast<cudaStream_t>(p->stream);
    if (!s) {
        RN_CUDA_CHECK(cudaStreamCreate(&own.s));
        s = own.s;
    }
    std::unique_ptr<rn_hierarchy> h(new rn_hierarchy());
    h->p = *p;
    h->k = k;
    h->mb = p->block_size;
    h->s = s;
    h->own_stream = (own.s != nullptr);
    const double t0 = rn::now_ms();
    const int32_t n = A->n_rows;
    rn::DVec<int32_t> rp, ci;
    rn::DVec<double> va, Bd, Bhd;
    rn::CsrView Av{n, n, A->nnz, A->rowptr, A->col, A->val};
    const double *Bp = B, *Bhp = Bhat;
    if (location == RN_HOST) {
        rp.alloc(n + 1, s);
        ci.alloc(A->nnz, s);
        va.alloc(A->nnz, s);
        Bd.alloc((size_t)n * k, s);
        rn::h2d(rp.p, A->rowptr, n + 1, s);
        rn::h2d(ci.p, A->col, A->nnz, s);
        rn::h2d(va.p, A->val, A->nnz, s);
        rn::h2d(Bd.p, B, (size_t)n * k, s);
        Av.rowptr = rp.p;
        Av.col = ci.p;
        Av.val = va.p;
        Bp = Bd.p;
        if (!p->symmetric) {
            Bhd.alloc((size_t)n * k, s);
            rn::h2d(Bhd.p, Bhat, (size_t)n * k, s);
            Bhp = Bhd.p;
        }
    }
    rn::build_hierarchy(*h, Av, Bp, Bhp);
    rn::prepare_solve(*h);
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    h->setup_ms = rn::now_ms() - t0;
    rp.release(); ci.release(); va.release(); Bd.release(); Bhd.release();
    *out = h.release();
    own.s = nullptr;  // the hierarchy owns it now; rn_free destroys it
    return RN_OK;
    RN_API_END
}

namespace {
// Run work(i) for i < count on up to `threads` host threads (0: one per
// hardware thread, at most 16); each item's status and error message are
// kept; returns the first non-OK status in index order and makes its message
// this thread's last error.
template <typename F>
rn_status run_batch(int count, int threads, F &&work) {
    std::vector<rn_status> st((size_t)count, RN_OK);
    std::vector<std::string> msg((size_t)count);
    int nt = threads > 0 ? threads : (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    nt = std::max(1, std::min(nt, count));
    std::atomic<int> next{0};
    auto body = [&](int t) {
        rn::set_thread_pool(nt > 1 ? t : -1);
        for (int i = next++; i < count; i = next++) {
            st[i] = work(i);
            if (st[i] != RN_OK) msg[i] = rn_last_error();
        }
        rn::set_thread_pool(-1);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; t++) pool.emplace_back(body, t);
    body(0);
    for (auto &t : pool) t.join();
    for (int i = 0; i < count; i++)
        if (st[i] != RN_OK) {
            rn::set_last_error(rn::fmt("problem %d: %s", i, msg[i].c_str()));
            return st[i];
        }
    return RN_OK;
}
}  // namespace

extern "C" rn_status rn_setup_batched(int count, const rn_csr *A, const double *const *B, const double *const *Bhat,
                                      const rn_params *p, int threads, rn_hierarchy **out) {
    if (!out || count < 0) {
        rn::set_last_error("null argument or negative count");
        return RN_EINVAL;
    }
    for (int i = 0; i < count; i++) out[i] = nullptr;
    if (count == 0) return RN_OK;
    if (!A || !B || !p) {
        rn::set_last_error("null argument");
        return RN_EINVAL;
    }
    if (p->stream) {
        rn::set_last_error("batched setup: params.stream must be NULL (every problem gets its own stream)");
        return RN_EINVAL;
    }
    const rn_status st = run_batch(count, threads, [&](int i) {
        return rn_setup(&A[i], B[i], Bhat ? Bhat[i] : nullptr, 1, RN_DEVICE, p, &out[i]);
    });
    if (st != RN_OK) {
        for (int i = 0; i < count; i++) {
            rn_free(out[i]);
            out[i] = nullptr;
        }
    }
    return st;
}

extern "C" rn_status rn_setup_merged(int count, const rn_csr *A, const double *const *B, const rn_params *p,
                                     rn_hierarchy **out) {
    if (!out || count < 0) {
        rn::set_last_error("null argument or negative count");
        return RN_EINVAL;
    }
    for (int i = 0; i < count; i++) out[i] = nullptr;
    if (count == 0) return RN_OK;
    std::vector<rn_hierarchy *> hs;  // freed with rn_free unless handed out
    struct Guard {
        std::vector<rn_hierarchy *> &hs;
        cudaStream_t ws = nullptr;
        ~Guard() {
            if (ws) cudaStreamSynchronize(ws);
            for (rn_hierarchy *h : hs) rn_free(h);
        }
    } guard{hs};
    RN_API_BEGIN
    using rn::fail;
    if (!A || !B || !p) fail(RN_EINVAL, "null argument");
    check_params(p);
    if (p->stream) fail(RN_EINVAL, "merged setup: params.stream must be NULL (every problem gets its own stream)");
    if (!p->symmetric) fail(RN_EINVAL, "merged setup: symmetric problems only (R = P^T)");
    if (p->energy_method != RN_ENERGY_CG) fail(RN_EINVAL, "merged setup: CG energy minimisation only");
    if (p->block_size != 1) fail(RN_EINVAL, "merged setup: scalar problems only (block_size 1)");
    std::vector<rn::CsrView> views;
    std::vector<const double *> bs;
    for (int i = 0; i < count; i++) {
        const rn_csr &a = A[i];
        if (a.n_rows <= 0 || a.n_rows != a.n_cols) fail(RN_EINVAL, rn::fmt("problem %d: A must be square and non-empty", i));
        if (a.nnz <= 0 || a.nnz > INT32_MAX - 1) fail(RN_EINVAL, rn::fmt("problem %d: nnz out of range", i));
        if (!a.rowptr || !a.col || !a.val || !B[i]) fail(RN_EINVAL, rn::fmt("problem %d: null array", i));
        views.push_back(rn::CsrView{a.n_rows, a.n_cols, a.nnz, a.rowptr, a.col, a.val});
        bs.push_back(B[i]);
    }
    // Streams and device pools kept for the process: problem i works on stream
    // k = i mod kMergedStreams with pool kMergedPoolBase + k, the merged
    // matrices on the next stream and pool, so no pool sees frees from more
    // than one stream (rn_free leaves these streams alone)
    rn::Allocator wa = alloc_of(*p);
    wa.pool = rn::kMergedPoolBase + rn::kMergedStreams;
    const rn::AllocScope alloc_scope(wa);
    const double t0 = rn::now_ms();
    guard.ws = rn::merged_stream(rn::kMergedStreams);
    for (int i = 0; i < count; i++) {
        rn_hierarchy *h = new rn_hierarchy();
        h->p = *p;
        h->k = 1;
        h->mb = 1;
        h->s = rn::merged_stream(i % rn::kMergedStreams);
        h->own_stream = false;
        h->pool = rn::kMergedPoolBase + i % rn::kMergedStreams;
        hs.push_back(h);
    }
    rn::build_hierarchies_merged(hs, views, bs, guard.ws);
    for (rn_hierarchy *h : hs) {  // every problem's launches before any read
        const rn::AllocScope scope(alloc_of(*h));
        rn::prepare_solve_begin(*h);
    }
    for (rn_hierarchy *h : hs) {
        const rn::AllocScope scope(alloc_of(*h));
        rn::prepare_solve_end(*h);
    }
    for (rn_hierarchy *h : hs) RN_CUDA_CHECK(cudaStreamSynchronize(h->s));
    const double ms = rn::now_ms() - t0;
    for (int i = 0; i < count; i++) {
        hs[i]->setup_ms = ms;
        out[i] = hs[i];
    }
    hs.clear();
    return RN_OK;
    RN_API_END
}

extern "C" rn_status rn_solve_batched(int count, rn_hierarchy *const *h, const double *const *b, double *const *x,
                                      double rtol, int maxit, int threads, rn_solve_info *info) {
    if (count < 0 || (count > 0 && (!h || !b || !x))) {
        rn::set_last_error("null argument or negative count");
        return RN_EINVAL;
    }
    return run_batch(count, threads, [&](int i) {
        return rn_solve(h[i], b[i], x[i], RN_DEVICE, rtol, maxit, info ? &info[i] : nullptr);
    });
}

extern "C" rn_status rn_batch_merge(int count, rn_hierarchy *const *h, void *stream, rn_batch **out) {
    if (out) *out = nullptr;
    RN_API_BEGIN
    using rn::fail;
    if (!out || !h || count < 1) fail(RN_EINVAL, "null argument or count < 1");
    for (int i = 0; i < count; i++)
        if (!h[i]) fail(RN_EINVAL, rn::fmt("hierarchy %d is NULL", i));
    // With no stream given, the batch works on a stream the library keeps for
    // the process, with a device pool of its own (a stream-ordered pool that
    // holds blocks freed on many streams is slow to allocate from).
    rn::Allocator a = alloc_of(h[0]->p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!s) {
        s = rn::merged_stream(rn::kMergedStreams + 1);
        a.pool = rn::kMergedPoolBase + rn::kMergedStreams + 1;
    }
    const rn::AllocScope alloc_scope(a);
    for (int i = 0; i < count; i++) RN_CUDA_CHECK(cudaStreamSynchronize(h[i]->s));
    rn_batch *b = rn::batch_merge(count, h, s);
    b->own_stream = false;
    b->M->pool = a.pool;
    *out = b;
    return RN_OK;
    RN_API_END
}

extern "C" rn_status rn_batch_solve(rn_batch *b, const double *const *bvec, double *const *x, double rtol, int maxit,
                                    rn_solve_info *info) {
    RN_API_BEGIN
    using rn::fail;
    if (!b || !bvec || !x) fail(RN_EINVAL, "null argument");
    for (int i = 0; i < b->np; i++)
        if (!bvec[i] || !x[i]) fail(RN_EINVAL, rn::fmt("vector of problem %d is NULL", i));
    if (maxit < 0 || !(rtol >= 0.0)) fail(RN_EINVAL, "maxit/rtol");
    const rn::AllocScope alloc_scope(alloc_of(*b->M));
    const rn_status st = rn::batch_solve(*b, bvec, x, rtol, maxit, info);
    if (st == RN_ENOTCONV) rn::set_last_error("a problem did not reach the tolerance within maxit");
    return st;
    RN_API_END
}

extern "C" rn_status rn_batch_cycle(rn_batch *b, const double *const *bvec, double *const *x) {
    RN_API_BEGIN
    using rn::fail;
    if (!b || !bvec || !x) fail(RN_EINVAL, "null argument");
    const rn::AllocScope alloc_scope(alloc_of(*b->M));
    rn::batch_cycle(*b, bvec, x);
    return RN_OK;
    RN_API_END
}

extern "C" void rn_batch_free(rn_batch *b) {
    if (!b) return;
    cudaStream_t s = b->M->s;
    const bool own = b->own_stream;
    try {
        delete b;
    } catch (...) {
    }
    cudaStreamSynchronize(s);
    if (own) cudaStreamDestroy(s);
}

extern "C" rn_status rn_solve(rn_hierarchy *h, const double *b, double *x, int location, double rtol, int maxit,
                              rn_solve_info *info) {
    RN_API_BEGIN
    using rn::fail;
    if (!h || !b || !x) fail(RN_EINVAL, "null argument");
    if (location != RN_DEVICE && location != RN_HOST) fail(RN_EINVAL, "location");
    if (maxit < 0 || !(rtol >= 0.0)) fail(RN_EINVAL, "maxit/rtol");
    const rn::AllocScope alloc_scope(alloc_of(*h));
    cudaStream_t s = h->s;
    const int64_t n = h->lev[0]->A.n;
    const double t0 = rn::now_ms();
    rn_status st;
    if (location == RN_HOST) {
        rn::DVec<double> bd(n, s), xd(n, s);
        rn::h2d(bd.p, b, n, s);
        rn::h2d(xd.p, x, n, s);
        st = rn::solve(*h, bd.p, xd.p, rtol, maxit, info);
        rn::d2h(x, xd.p, n, s);
        RN_CUDA_CHECK(cudaStreamSynchronize(s));
    } else {
        st = rn::solve(*h, b, x, rtol, maxit, info);
    }
    if (info) info->solve_ms = rn::now_ms() - t0;
    if (st == RN_ENOTCONV) rn::set_last_error("solve did not reach the tolerance within maxit");
    return st;
    RN_API_END
}

extern "C" rn_status rn_solve_multi(rn_hierarchy *h, const double *B, double *X, int s, int location, double rtol,
                                    int maxit, rn_solve_info *info) {
    RN_API_BEGIN
    using rn::fail;
    if (!h || !B || !X) fail(RN_EINVAL, "null argument");
    if (s < 1 || s > 2048) fail(RN_EINVAL, "s must be in [1, 2048]");
    if (h->p.gamma != 1) fail(RN_EINVAL, "the many-right-hand-side cycle is a V-cycle (gamma 1)");
    if (location != RN_DEVICE && location != RN_HOST) fail(RN_EINVAL, "location");
    if (maxit < 0 || !(rtol >= 0.0)) fail(RN_EINVAL, "maxit/rtol");
    const rn::AllocScope alloc_scope(alloc_of(*h));
    cudaStream_t st = h->s;
    const int64_t tot = (int64_t)h->lev[0]->A.n * s;
    const double t0 = rn::now_ms();
    rn_status r;
    if (location == RN_HOST) {
        rn::DVec<double> bd(tot, st), xd(tot, st);
        rn::h2d(bd.p, B, tot, st);
        rn::h2d(xd.p, X, tot, st);
        r = rn::solve_multi(*h, bd.p, xd.p, s, rtol, maxit, info);
        rn::d2h(X, xd.p, tot, st);
    } else {
        r = rn::solve_multi(*h, B, X, s, rtol, maxit, info);
    }
    RN_CUDA_CHECK(cudaStreamSynchronize(st));
    if (info) info->solve_ms = rn::now_ms() - t0;
    if (r == RN_ENOTCONV) rn::set_last_error("a column did not reach the tolerance within maxit");
    return r;
    RN_API_END
}

extern "C" rn_status rn_vcycle(rn_hierarchy *h, const double *b, double *x) {
    RN_API_BEGIN
    if (!h || !b || !x) rn::fail(RN_EINVAL, "null argument");
    const rn::AllocScope alloc_scope(alloc_of(*h));
    rn::cycle_checked(*h, b, x);
    RN_CUDA_CHECK(cudaStreamSynchronize(h->s));
    return RN_OK;
    RN_API_END
}

extern "C" rn_status rn_time_op(rn_hierarchy *h, int op, int reps, int64_t flush_bytes, double *us, double *bytes,
                                char *name) {
    RN_API_BEGIN
    if (!h || !us || !bytes) rn::fail(RN_EINVAL, "null argument");
    const rn::AllocScope alloc_scope(alloc_of(*h));
    std::string nm;
    rn::time_op(*h, op, reps, flush_bytes, us, bytes, nm);
    if (name) {
        std::strncpy(name, nm.c_str(), 47);
        name[47] = '\0';
    }
    return RN_OK;
    RN_API_END
}

extern "C" rn_status rn_time_setup_op(rn_hierarchy *h, int op, int reps, int64_t flush_bytes, double *us,
                                      double *bytes, char *name) {
    RN_API_BEGIN
    if (!h || !us || !bytes) rn::fail(RN_EINVAL, "null argument");
    const rn::AllocScope alloc_scope(alloc_of(*h));
    std::string nm;
    rn::time_setup_op(*h, op, reps, flush_bytes, us, bytes, nm);
    if (name) {
        std::strncpy(name, nm.c_str(), 47);
        name[47] = '\0';
    }
    return RN_OK;
    RN_API_END
}

namespace {
// A stream the call owns when the caller passes none (blocking, so it stays
// ordered with the legacy default stream).
struct CallStream {
    cudaStream_t s = nullptr;
    bool own = false;
    explicit CallStream(void *given) {
        s = static_cast<cudaStream_t>(given);
        if (!s) {
            RN_CUDA_CHECK(cudaStreamCreate(&s));
            own = true;
        }
    }
    ~CallStream() {
        if (own) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};
}  // namespace

extern "C" rn_status rn_adjoint_grad(const rn_csr *A, const double *lambda, const double *x, double *grad,
                                     void *stream) {
    RN_API_BEGIN
    using rn::fail;
    if (!A || !lambda || !x || !grad) fail(RN_EINVAL, "null argument");
    if (A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0 || A->nnz > INT32_MAX - 1) fail(RN_EINVAL, "A");
    if (A->n_rows > 0 && (!A->rowptr || (A->nnz > 0 && !A->col))) fail(RN_EINVAL, "null CSR array");
    CallStream cs(stream);
    rn::CsrView Av{A->n_rows, A->n_cols, A->nnz, A->rowptr, A->col, A->val};
    rn::adjoint_grad(Av, lambda, x, grad, cs.s);
    RN_CUDA_CHECK(cudaStreamSynchronize(cs.s));
    return RN_OK;
    RN_API_END
}

extern "C" rn_status rn_energy_min(const rn_csr *A, const rn_csr *N, const int32_t *rowtype, const double *Bc,
                                   double *P, int sweeps, int method, int precond, void *stream) {
    RN_API_BEGIN
    using rn::fail;
    if (!A || !N || !rowtype || !Bc || !P) fail(RN_EINVAL, "null argument");
    if (A->n_rows <= 0 || A->n_rows != A->n_cols || !A->rowptr || !A->col || !A->val) fail(RN_EINVAL, "A");
    if (A->nnz <= 0 || A->nnz > INT32_MAX - 1) fail(RN_EINVAL, "nnz(A) out of range");
    if (N->n_rows != A->n_rows || N->n_cols < 1 || N->nnz < 0 || N->nnz > INT32_MAX - 1 || !N->rowptr ||
        (N->nnz > 0 && !N->col))
        fail(RN_EINVAL, "pattern N does not match A");
    if (sweeps < 0 || sweeps > 1000) fail(RN_EINVAL, "sweeps must be in [0, 1000]");
    if (method != RN_ENERGY_CG && method != RN_ENERGY_GMRES) fail(RN_EINVAL, "method");
    CallStream cs(stream);
    cudaStream_t s = cs.s;
    const int32_t n = A->n_rows;
    rn::DVec<double> diag(n, s), partial(2 * rn::kReduceBlocks, s), sc(64, s);
    rn::DVec<unsigned> counter(4, s);
    rn::DVec<int32_t> fl(16, s);
    RN_CUDA_CHECK(cudaMemsetAsync(counter.p, 0, 4 * sizeof(unsigned), s));
    RN_CUDA_CHECK(cudaMemsetAsync(fl.p, 0, 16 * sizeof(int32_t), s));
    RN_CUDA_CHECK(cudaMemsetAsync(sc.p, 0, 64 * sizeof(double), s));
    rn::CsrView Av{n, n, A->nnz, A->rowptr, A->col, A->val};
    rn::extract_diag(Av, diag.p, fl.p + 4, s);
    if (rn::read_scalar(fl.p + 4, s)) fail(RN_EINVAL, "missing or zero diagonal");
    rn::EmCtx c;
    c.s = s;
    c.partial = partial.p;
    c.counter = counter.p;
    c.sc = sc.p;
    c.fl = fl.p;
    c.precond = precond ? 1 : 0;
    c.method = method;
    rn::Pattern pat{n, N->n_cols, N->nnz, N->rowptr, N->col};
    rn::reciprocal(diag.p, diag.p, n, s);  // the preconditioner D^{-1}
    rn::energy_min(c, Av, pat, P, rowtype, Bc, diag.p, sweeps);
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    return RN_OK;
    RN_API_END
}

extern "C" void rn_free(rn_hierarchy *h) {
    if (!h) return;
    cudaStream_t s = h->s;
    const bool own = h->own_stream;
    try {
        delete h;
    } catch (...) {
    }
    cudaStreamSynchronize(s);
    if (own) cudaStreamDestroy(s);
}

extern "C" rn_status rn_hierarchy_stats(const rn_hierarchy *h, rn_stats *st) {
    if (!h || !st) return RN_EINVAL;
    std::memset(st, 0, sizeof *st);
    st->levels = (int)h->lev.size();
    const double nnz0 = (double)h->lev[0]->A.nnz;
    double oc = 0.0, cc = 0.0;
    const int nu = h->p.nu_pre + h->p.nu_post;
    for (size_t l = 0; l < h->lev.size() && l < RN_MAX_LEVELS; l++) {
        const rn_level &L = *h->lev[l];
        st->n[l] = L.A.n;
        st->nnz_A[l] = L.A.nnz;
        st->nnz_P[l] = L.P.nnz;
        st->nnz_R[l] = L.R.nnz;
        oc += L.A.nnz / nnz0;
        if (l + 1 < h->lev.size()) cc += ((nu + 1) * (double)L.A.nnz + L.P.nnz + L.R.nnz) / nnz0;
    }
    st->oc = oc;
    st->cc = cc;
    st->setup_ms = h->setup_ms;
    st->agg_rounds = h->agg_rounds;
    return RN_OK;
}

extern "C" rn_status rn_export_csr(const rn_hierarchy *h, int lvl, int which, int32_t *n_rows, int32_t *n_cols,
                                   int64_t *nnz, int32_t *rowptr, int32_t *col, double *val) {
    RN_API_BEGIN
    using rn::fail;
    if (!h || lvl < 0 || lvl >= (int)h->lev.size()) fail(RN_EINVAL, "level out of range");
    const rn_level &L = *h->lev[lvl];
    const rn::DCsr *M = nullptr;
    switch (which) {
        case 0: M = &L.A; break;
        case 1: M = &L.S; break;
        case 2: M = &L.N; break;
        case 3: M = &L.T; break;
        case 4: M = &L.P; break;
        case 5: M = &L.R; break;
        default: fail(RN_EINVAL, "which");
    }
    if (!M->rowptr.p) fail(RN_EINVAL, "matrix not present on this level (keep_aux off or coarsest level)");
    if (n_rows) *n_rows = M->n;
    if (n_cols) *n_cols = M->m;
    if (nnz) *nnz = M->nnz;
    cudaStream_t s = h->s;
    if (rowptr) rn::d2h(rowptr, M->rowptr.p, M->n + 1, s);
    if (col) rn::d2h(col, M->col.p, M->nnz, s);
    if (val && M->val.p) rn::d2h(val, M->val.p, M->nnz, s);
    RN_CUDA_CHECK(cudaStreamSynchronize(s));
    return RN_OK;
    RN_API_END
}

extern "C" rn_status rn_export_vec(const rn_hierarchy *h, int lvl, int which, int64_t *len, void *out) {
    RN_API_BEGIN
    using rn::fail;
    if (!h || !len || lvl < 0 || lvl >= (int)h->lev.size()) fail(RN_EINVAL, "bad argument");
    const rn_level &L = *h->lev[lvl];
    const void *src = nullptr;
    size_t elt = 4;
    int64_t n = 0;
    switch (which) {
        case 0: src = L.agg.p; n = L.agg.n; break;
        case 1: src = L.roots.p; n = L.roots.n; break;
        case 2: src = L.rowtype.p; n = L.rowtype.n; break;
        case 3: src = L.B.p; n = L.B.n; elt = 8; break;
        case 4: src = L.Bc.p; n = L.Bc.n; elt = 8; break;
        case 5: src = L.Bhat.p; n = L.Bhat.n; elt = 8; break;
        case 6: src = L.Bhatc.p; n = L.Bhatc.n; elt = 8; break;
        default: fail(RN_EINVAL, "which");
    }
    if (!src) fail(RN_EINVAL, "vector not present on this level");
    *len = n;
    if (out) {
        RN_CUDA_CHECK(cudaMemcpyAsync(out, src, (size_t)n * elt, cudaMemcpyDeviceToHost, h->s));
        RN_CUDA_CHECK(cudaStreamSynchronize(h->s));
    }
    return RN_OK;
    RN_API_END
}

extern "C" const char *rn_last_error(void) { return rn::last_error_ref().c_str(); }

extern "C" const char *rn_status_string(rn_status s) {
    switch (s) {
        case RN_OK: return "RN_OK";
        case RN_EINVAL: return "RN_EINVAL";
        case RN_ENOMEM: return "RN_ENOMEM";
        case RN_ESINGULAR: return "RN_ESINGULAR";
        case RN_ESTALL: return "RN_ESTALL";
        case RN_ENOTCONV: return "RN_ENOTCONV";
        case RN_ETIMEOUT: return "RN_ETIMEOUT";
        case RN_ECUDA: return "RN_ECUDA";
        case RN_EINTERNAL: return "RN_EINTERNAL";
    }
    return "unknown";
}
