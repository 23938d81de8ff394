"""Python binding of the C ABI in include/rn.h (argument marshalling only).

Every step of setup and solve runs in ``librn.so``'s CUDA kernels.  The
functions ``rn_setup``, ``rn_solve``, ``rn_free``, ... carry the C names; the
``Hierarchy`` class is a thin owner around them that accepts torch tensors
(device) or numpy arrays (host).  Importing this module fails loudly when the
library has not been built or cannot be loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librn.so")

RN_OK, RN_EINVAL, RN_ENOMEM, RN_ESINGULAR, RN_ESTALL, RN_ENOTCONV, RN_ETIMEOUT, RN_ECUDA, RN_EINTERNAL = range(9)
RN_DEVICE, RN_HOST = 0, 1
RN_ENERGY_CG, RN_ENERGY_GMRES = 0, 1
RN_FP64, RN_MIXED = 0, 1
RN_OUTER_STATIONARY, RN_OUTER_CG, RN_OUTER_FGMRES = 0, 1, 2
RN_MAX_LEVELS = 32
RN_SOC_SYMMETRIC, RN_SOC_CLASSICAL = 0, 1
(RN_OP_OUTER_SPMV, RN_OP_RELAX0_RESIDUAL, RN_OP_JACOBI_OUT, RN_OP_RESTRICT, RN_OP_PROLONG, RN_OP_CG_XR,
 RN_OP_CG_RZ, RN_OP_CG_P, RN_OP_COARSE_CLUSTER, RN_OP_COUNT) = range(10)
(RN_SOP_ENERGY_SWEEP, RN_SOP_ENERGY_DIRECTION, RN_SOP_ENERGY_PRODUCT, RN_SOP_ENERGY_UPDATE, RN_SOP_GALERKIN_AP,
 RN_SOP_GALERKIN_RAP, RN_SOP_TRANSPOSE, RN_SOP_COUNT) = range(8)
STATUS_NAMES = ["RN_OK", "RN_EINVAL", "RN_ENOMEM", "RN_ESINGULAR", "RN_ESTALL", "RN_ENOTCONV", "RN_ETIMEOUT",
                "RN_ECUDA", "RN_EINTERNAL"]


class rn_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
DEALLOC_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class rn_params(C.Structure):
    _fields_ = [("soc_theta", C.c_double), ("soc_theta_coarse", C.c_double), ("degree", C.c_int),
                ("n_sweeps", C.c_int), ("energy_method", C.c_int), ("energy_precond", C.c_int),
                ("prefilter", C.c_double), ("postfilter", C.c_double), ("max_coarse", C.c_int),
                ("max_levels", C.c_int), ("b_sweeps", C.c_int), ("omega", C.c_double), ("seed", C.c_uint64),
                ("symmetric", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int), ("precision", C.c_int),
                ("outer", C.c_int), ("restart", C.c_int), ("use_graphs", C.c_int), ("keep_aux", C.c_int),
                ("coarse_cluster", C.c_int), ("gamma", C.c_int), ("soc_kind", C.c_int), ("block_size", C.c_int),
                ("autotune", C.c_int), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("dealloc", DEALLOC_FN),
                ("alloc_ctx", C.c_void_p)]


class rn_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_res", C.c_double), ("rho", C.c_double), ("solve_ms", C.c_double),
                ("status", C.c_int)]


class rn_stats(C.Structure):
    _fields_ = [("levels", C.c_int), ("n", C.c_int32 * RN_MAX_LEVELS), ("nnz_A", C.c_int64 * RN_MAX_LEVELS),
                ("nnz_P", C.c_int64 * RN_MAX_LEVELS), ("nnz_R", C.c_int64 * RN_MAX_LEVELS), ("oc", C.c_double),
                ("cc", C.c_double), ("setup_ms", C.c_double), ("agg_rounds", C.c_int)]


class rn_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("ms", C.c_double), ("bytes", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                          "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    L.rn_default_params.argtypes = [P(rn_params)]
    L.rn_setup.argtypes = [P(rn_csr), C.c_void_p, C.c_void_p, C.c_int, C.c_int, P(rn_params), P(C.c_void_p)]
    L.rn_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, P(rn_solve_info)]
    L.rn_vcycle.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.rn_solve_multi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                                 P(rn_solve_info)]
    L.rn_setup_batched.argtypes = [C.c_int, P(rn_csr), P(C.c_void_p), P(C.c_void_p), P(rn_params), C.c_int,
                                   P(C.c_void_p)]
    L.rn_setup_merged.argtypes = [C.c_int, P(rn_csr), P(C.c_void_p), P(rn_params), P(C.c_void_p)]
    L.rn_solve_batched.argtypes = [C.c_int, P(C.c_void_p), P(C.c_void_p), P(C.c_void_p), C.c_double, C.c_int,
                                   C.c_int, P(rn_solve_info)]
    L.rn_free.argtypes = [C.c_void_p]
    L.rn_free.restype = None
    L.rn_batch_merge.argtypes = [C.c_int, P(C.c_void_p), C.c_void_p, P(C.c_void_p)]
    L.rn_batch_solve.argtypes = [C.c_void_p, P(C.c_void_p), P(C.c_void_p), C.c_double, C.c_int, P(rn_solve_info)]
    L.rn_batch_cycle.argtypes = [C.c_void_p, P(C.c_void_p), P(C.c_void_p)]
    L.rn_batch_free.argtypes = [C.c_void_p]
    L.rn_batch_free.restype = None
    L.rn_energy_min.argtypes = [P(rn_csr), P(rn_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                C.c_void_p]
    L.rn_energy_min_noalloc.argtypes = [P(rn_csr), P(rn_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                        C.c_void_p]
    L.rn_hierarchy_stats.argtypes = [C.c_void_p, P(rn_stats)]
    L.rn_export_csr.argtypes = [C.c_void_p, C.c_int, C.c_int, P(C.c_int32), P(C.c_int32), P(C.c_int64),
                                C.c_void_p, C.c_void_p, C.c_void_p]
    L.rn_export_vec.argtypes = [C.c_void_p, C.c_int, C.c_int, P(C.c_int64), C.c_void_p]
    L.rn_profile_enable.argtypes = [C.c_int]
    L.rn_profile_reset.argtypes = []
    L.rn_profile_read.argtypes = [P(rn_kernel_stat), C.c_int, P(C.c_int)]
    L.rn_kernel_launches.argtypes = []
    L.rn_kernel_launches.restype = C.c_int64
    L.rn_allocation_count.argtypes = []
    L.rn_allocation_count.restype = C.c_int64
    L.rn_time_op.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, P(C.c_double), P(C.c_double), C.c_char_p]
    L.rn_time_setup_op.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, P(C.c_double), P(C.c_double),
                                   C.c_char_p]
    L.rn_adjoint_grad.argtypes = [P(rn_csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.rn_last_error.restype = C.c_char_p
    L.rn_status_string.argtypes = [C.c_int]
    L.rn_status_string.restype = C.c_char_p
    return L


lib = _load()

# ----------------------------------------------------------------- C names
rn_default_params = lib.rn_default_params
rn_setup = lib.rn_setup
rn_solve = lib.rn_solve
rn_vcycle = lib.rn_vcycle
rn_solve_multi = lib.rn_solve_multi
rn_setup_batched = lib.rn_setup_batched
rn_setup_merged = lib.rn_setup_merged
rn_solve_batched = lib.rn_solve_batched
rn_free = lib.rn_free
rn_batch_merge = lib.rn_batch_merge
rn_batch_solve = lib.rn_batch_solve
rn_batch_cycle = lib.rn_batch_cycle
rn_batch_free = lib.rn_batch_free
rn_hierarchy_stats = lib.rn_hierarchy_stats
rn_export_csr = lib.rn_export_csr
rn_export_vec = lib.rn_export_vec
rn_profile_enable = lib.rn_profile_enable
rn_profile_reset = lib.rn_profile_reset
rn_profile_read = lib.rn_profile_read
rn_last_error = lib.rn_last_error
rn_status_string = lib.rn_status_string
rn_kernel_launches = lib.rn_kernel_launches
rn_allocation_count = lib.rn_allocation_count
rn_time_op = lib.rn_time_op
rn_time_setup_op = lib.rn_time_setup_op
rn_adjoint_grad = lib.rn_adjoint_grad
rn_energy_min = lib.rn_energy_min
rn_energy_min_noalloc = lib.rn_energy_min_noalloc


def energy_min_noalloc(A_rowptr, A_col, A_val, N_rowptr, N_col, n_c, rowtype, Bc, P, sweeps, precond=1, stream=None):
    """Run rn_energy_min_noalloc (CG, no device allocation) on device tensors; P is updated in place."""
    n = int(A_rowptr.shape[0]) - 1
    A = rn_csr(n, n, int(A_col.shape[0]), _ptr(A_rowptr), _ptr(A_col), _ptr(A_val))
    N = rn_csr(n, int(n_c), int(N_col.shape[0]), _ptr(N_rowptr), _ptr(N_col) if N_col.shape[0] else None, None)
    _check(rn_energy_min_noalloc(C.byref(A), C.byref(N), _ptr(rowtype), _ptr(Bc), _ptr(P), sweeps, precond, stream),
           "rn_energy_min_noalloc")


def energy_min(A_rowptr, A_col, A_val, N_rowptr, N_col, n_c, rowtype, Bc, P, sweeps, method=RN_ENERGY_CG,
               precond=1, stream=None):
    """Run rn_energy_min on device tensors; P (float64, nnz(N)) is updated in place."""
    n = int(A_rowptr.shape[0]) - 1
    A = rn_csr(n, n, int(A_col.shape[0]), _ptr(A_rowptr), _ptr(A_col), _ptr(A_val))
    N = rn_csr(n, int(n_c), int(N_col.shape[0]), _ptr(N_rowptr), _ptr(N_col) if N_col.shape[0] else None, None)
    _check(rn_energy_min(C.byref(A), C.byref(N), _ptr(rowtype), _ptr(Bc), _ptr(P), sweeps, method, precond,
                         stream), "rn_energy_min")


def adjoint_grad(rowptr, col, lam, x, grad, n_cols=None, stream=None):
    """grad[e] = -lam[i] * x[col[e]] on the CSR pattern (rn_adjoint_grad); device tensors, grad written."""
    n = int(rowptr.shape[0]) - 1
    A = rn_csr(n, int(n if n_cols is None else n_cols), int(col.shape[0]), _ptr(rowptr), _ptr(col), None)
    _check(rn_adjoint_grad(C.byref(A), _ptr(lam), _ptr(x), _ptr(grad), stream), "rn_adjoint_grad")


def setup_batched(problems, params=None, threads=0):
    """Hierarchies for many problems at once (rn_setup_batched).  problems: a
    list of (rowptr, col, val, B) or (rowptr, col, val, B, Bhat) device
    tensors; returns a list of Hierarchy."""
    if params is None:
        params = default_params()
    k = len(problems)
    A = (rn_csr * k)()
    Bp = (C.c_void_p * k)()
    Bh = (C.c_void_p * k)()
    for i, pr in enumerate(problems):
        rp, ci, va, B = pr[:4]
        n = int(rp.shape[0]) - 1
        A[i] = rn_csr(n, n, int(ci.shape[0]), _ptr(rp), _ptr(ci), _ptr(va))
        Bp[i] = _ptr(B)
        Bh[i] = _ptr(pr[4]) if len(pr) > 4 and pr[4] is not None else None
    out = (C.c_void_p * k)()
    _check(rn_setup_batched(k, A, Bp, Bh, C.byref(params), threads, out), "rn_setup_batched")
    hs = []
    for i in range(k):
        h = Hierarchy.__new__(Hierarchy)
        h.n = int(problems[i][0].shape[0]) - 1
        h.params = params
        h._keep = None
        h._h = C.c_void_p(out[i])
        hs.append(h)
    return hs


def setup_merged(problems, params=None):
    """Hierarchies for many problems built in one merged pass (rn_setup_merged).
    problems: a list of (rowptr, col, val, B) device tensors (symmetric, one
    candidate); returns a list of Hierarchy."""
    if params is None:
        params = default_params()
    k = len(problems)
    A = (rn_csr * k)()
    Bp = (C.c_void_p * k)()
    for i, pr in enumerate(problems):
        rp, ci, va, B = pr[:4]
        n = int(rp.shape[0]) - 1
        A[i] = rn_csr(n, n, int(ci.shape[0]), _ptr(rp), _ptr(ci), _ptr(va))
        Bp[i] = _ptr(B)
    out = (C.c_void_p * k)()
    _check(rn_setup_merged(k, A, Bp, C.byref(params), out), "rn_setup_merged")
    hs = []
    for i in range(k):
        h = Hierarchy.__new__(Hierarchy)
        h.n = int(problems[i][0].shape[0]) - 1
        h.params = params
        h._keep = None
        h._h = C.c_void_p(out[i])
        hs.append(h)
    return hs


def solve_batched(hierarchies, bs, xs, rtol=1e-8, maxit=500, threads=0, raise_on_notconv=True):
    """Solve every (hierarchy, b, x) at once (rn_solve_batched); x updated in place."""
    k = len(hierarchies)
    H = (C.c_void_p * k)(*[h._h.value for h in hierarchies])
    Bv = (C.c_void_p * k)(*[_ptr(b) for b in bs])
    Xv = (C.c_void_p * k)(*[_ptr(x) for x in xs])
    infos = (rn_solve_info * k)()
    st = rn_solve_batched(k, H, Bv, Xv, rtol, maxit, threads, infos)
    if st != RN_OK and (st != RN_ENOTCONV or raise_on_notconv):
        raise RNError(st, "rn_solve_batched")
    return [dict(iters=i.iters, rel_res=i.rel_res, rho=i.rho, solve_ms=i.solve_ms, status=i.status) for i in infos]


class RNError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.rn_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


def _check(st: int, where: str):
    if st != RN_OK:
        raise RNError(st, where)


def default_params(**overrides) -> rn_params:
    p = rn_params()
    _check(rn_default_params(C.byref(p)), "rn_default_params")
    for k, v in overrides.items():
        if k in ("outer_name",):
            continue
        if not hasattr(p, k):
            continue
        setattr(p, k, v)
    return p


def params_from_config(cfg: dict, **overrides) -> rn_params:
    """Map a workload parameter dict (see problems.PARAMS_*) to rn_params."""
    m = dict(cfg)
    m.update(overrides)
    kw = dict(soc_theta=m.get("soc_theta", 0.25), soc_theta_coarse=m.get("soc_theta_coarse", -1.0),
              degree=m.get("degree", 2), n_sweeps=m.get("n_sweeps", 4), energy_method=m.get("method", 0),
              energy_precond=m.get("precond", 1), prefilter=m.get("prefilter", 0.0),
              postfilter=m.get("postfilter", 0.0), max_coarse=m.get("max_coarse", 64),
              max_levels=m.get("max_levels", 25), b_sweeps=m.get("b_sweeps", 4), omega=m.get("omega", 2.0 / 3.0),
              seed=m.get("seed", 12345), symmetric=m.get("symmetric", 1), nu_pre=m.get("nu_pre", 1),
              nu_post=m.get("nu_post", 1), precision=m.get("precision", RN_FP64), outer=m.get("outer", RN_OUTER_CG),
              restart=m.get("restart", 30), use_graphs=m.get("use_graphs", 1), keep_aux=m.get("keep_aux", 0),
              coarse_cluster=m.get("coarse_cluster", 0), gamma=m.get("gamma", 1), soc_kind=m.get("soc_kind", 0),
              block_size=m.get("block_size", 1), autotune=m.get("autotune", 0))
    return default_params(**kw)


def _ptr(a) -> int:
    """Device pointer of a contiguous torch tensor, or host pointer of a numpy array."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _is_host(a) -> bool:
    return isinstance(a, np.ndarray) or (hasattr(a, "is_cuda") and not a.is_cuda)


def _torch_alloc(nbytes, stream, ctx):
    try:
        import torch

        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
    except Exception:  # out of memory or no CUDA: the library reports RN_ENOMEM
        return None


def _torch_dealloc(ptr, nbytes, stream, ctx):
    try:
        import torch

        torch.cuda.caching_allocator_delete(ptr)
    except Exception:  # interpreter shutdown: the process is releasing the device anyway
        pass


# module-level callback objects: they must outlive every hierarchy that uses them
TORCH_ALLOC = ALLOC_FN(_torch_alloc)
TORCH_DEALLOC = DEALLOC_FN(_torch_dealloc)


def use_torch_allocator(p: rn_params, stream=None) -> rn_params:
    """Route every device allocation of a hierarchy set up with p through
    torch's caching allocator (rn_params alloc/dealloc hooks), on `stream`
    (default: torch's current stream), so the library shares torch's memory
    pool instead of holding a pool of its own."""
    import torch

    p.alloc = TORCH_ALLOC
    p.dealloc = TORCH_DEALLOC
    p.alloc_ctx = None
    if stream is None and not p.stream:
        stream = torch.cuda.current_stream().cuda_stream
    if stream is not None:
        p.stream = C.c_void_p(stream)
    return p


class Batch:
    """Independent problems merged into one block-diagonal hierarchy
    (rn_batch_merge): every cycle and CG step is one launch for all of them.
    hierarchies: Hierarchy objects (only read; they may be closed afterwards)."""

    def __init__(self, hierarchies, stream=None):
        k = len(hierarchies)
        H = (C.c_void_p * k)(*[h._h.value for h in hierarchies])
        self._b = C.c_void_p()
        self.count = k
        _check(rn_batch_merge(k, H, C.c_void_p(stream) if stream else None, C.byref(self._b)), "rn_batch_merge")

    def close(self):
        if getattr(self, "_b", None):
            rn_batch_free(self._b)
            self._b = None

    def __del__(self):
        self.close()

    def solve(self, bs, xs, rtol=1e-8, maxit=500, raise_on_notconv=True):
        """CG on every problem (device vectors); xs updated in place; one record per problem."""
        k = self.count
        Bv = (C.c_void_p * k)(*[_ptr(b) for b in bs])
        Xv = (C.c_void_p * k)(*[_ptr(x) for x in xs])
        infos = (rn_solve_info * k)()
        st = rn_batch_solve(self._b, Bv, Xv, rtol, maxit, infos)
        if st != RN_OK and (st != RN_ENOTCONV or raise_on_notconv):
            raise RNError(st, "rn_batch_solve")
        return [dict(iters=i.iters, rel_res=i.rel_res, rho=i.rho, solve_ms=i.solve_ms, status=i.status) for i in infos]

    def cycle(self, bs, xs):
        """xs[i] = M_i^{-1} bs[i]: one cycle per problem."""
        k = self.count
        Bv = (C.c_void_p * k)(*[_ptr(b) for b in bs])
        Xv = (C.c_void_p * k)(*[_ptr(x) for x in xs])
        _check(rn_batch_cycle(self._b, Bv, Xv), "rn_batch_cycle")


class Hierarchy:
    """Owns an rn_hierarchy.  A, B, Bhat: torch CUDA tensors or numpy arrays;
    B (and Bhat) is n or n x k (k candidate vectors, row-major)."""

    def __init__(self, rowptr, col, val, B, Bhat=None, params: rn_params | None = None, stream=None):
        host = _is_host(val)
        n = int(rowptr.shape[0]) - 1
        k = 1 if len(B.shape) == 1 else int(B.shape[1])
        if host:
            rowptr = np.ascontiguousarray(rowptr, np.int32)
            col = np.ascontiguousarray(col, np.int32)
            val = np.ascontiguousarray(val, np.float64)
            B = np.ascontiguousarray(B, np.float64).reshape(-1)
            Bhat = None if Bhat is None else np.ascontiguousarray(Bhat, np.float64).reshape(-1)
        else:
            B = B.contiguous()
            Bhat = None if Bhat is None else Bhat.contiguous()
        self.k = k
        self.n = n
        self.params = params if params is not None else default_params()
        if stream is not None:
            self.params.stream = C.c_void_p(stream)
        A = rn_csr(n, n, int(col.shape[0]), _ptr(rowptr), _ptr(col), _ptr(val))
        h = C.c_void_p()
        self._keep = (rowptr, col, val, B, Bhat)
        st = rn_setup(C.byref(A), _ptr(B), _ptr(Bhat) if Bhat is not None else None, k,
                      RN_HOST if host else RN_DEVICE, C.byref(self.params), C.byref(h))
        self._keep = None
        _check(st, "rn_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            rn_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def solve(self, b, x, rtol=1e-8, maxit=500, raise_on_notconv=True):
        host = _is_host(b)
        info = rn_solve_info()
        st = rn_solve(self._h, _ptr(b), _ptr(x), RN_HOST if host else RN_DEVICE, rtol, maxit, C.byref(info))
        if st != RN_OK and (st != RN_ENOTCONV or raise_on_notconv):
            raise RNError(st, "rn_solve")
        return dict(iters=info.iters, rel_res=info.rel_res, rho=info.rho, solve_ms=info.solve_ms, status=st)

    def solve_multi(self, B, X, rtol=1e-8, maxit=500, raise_on_notconv=True):
        """Solve for the s columns of B (n x s, row-major) at once; X (n x s) is updated in place."""
        host = _is_host(B)
        s = int(B.shape[1])
        info = rn_solve_info()
        st = rn_solve_multi(self._h, _ptr(B), _ptr(X), s, RN_HOST if host else RN_DEVICE, rtol, maxit,
                            C.byref(info))
        if st != RN_OK and (st != RN_ENOTCONV or raise_on_notconv):
            raise RNError(st, "rn_solve_multi")
        return dict(iters=info.iters, rel_res=info.rel_res, rho=info.rho, solve_ms=info.solve_ms, status=st)

    def vcycle(self, b, x):
        _check(rn_vcycle(self._h, _ptr(b), _ptr(x)), "rn_vcycle")

    def time_op(self, op: int, reps: int = 20, flush_bytes: int = 256 << 20):
        """(name, mean device us per launch, algorithmic bytes) of one level-0 launch of the solve
        timed in isolation (rn_time_op); None when this hierarchy does not run it."""
        us, by = C.c_double(), C.c_double()
        nm = C.create_string_buffer(48)
        st = rn_time_op(self._h, op, reps, flush_bytes, C.byref(us), C.byref(by), nm)
        if st == RN_EINVAL:
            return None
        _check(st, "rn_time_op")
        return nm.value.decode(), us.value, by.value

    def time_setup_op(self, op: int, reps: int = 10, flush_bytes: int = 256 << 20):
        """(name, mean device us per run, algorithmic bytes) of one level-0 setup operation timed in
        isolation (rn_time_setup_op); raises RNError when the hierarchy lacks what it needs."""
        us, by = C.c_double(), C.c_double()
        nm = C.create_string_buffer(48)
        _check(rn_time_setup_op(self._h, op, reps, flush_bytes, C.byref(us), C.byref(by), nm), "rn_time_setup_op")
        return nm.value.decode(), us.value, by.value

    def stats(self) -> dict:
        s = rn_stats()
        _check(rn_hierarchy_stats(self._h, C.byref(s)), "rn_hierarchy_stats")
        L = s.levels
        return dict(levels=L, n=list(s.n[:L]), nnz_A=list(s.nnz_A[:L]), nnz_P=list(s.nnz_P[:L]),
                    nnz_R=list(s.nnz_R[:L]), oc=s.oc, cc=s.cc, setup_ms=s.setup_ms, agg_rounds=s.agg_rounds)

    def export_csr(self, lvl: int, which: int):
        """(rowptr, col, val, shape) numpy copies of matrix `which` (0 A, 1 S, 2 N, 3 T, 4 P, 5 R) on level lvl."""
        nr, nc, nz = C.c_int32(), C.c_int32(), C.c_int64()
        _check(rn_export_csr(self._h, lvl, which, C.byref(nr), C.byref(nc), C.byref(nz), None, None, None),
               "rn_export_csr")
        rp = np.zeros(nr.value + 1, np.int32)
        ci = np.zeros(max(nz.value, 1), np.int32)
        va = np.zeros(max(nz.value, 1), np.float64)
        _check(rn_export_csr(self._h, lvl, which, C.byref(nr), C.byref(nc), C.byref(nz), rp.ctypes.data,
                             ci.ctypes.data, va.ctypes.data), "rn_export_csr")
        return rp, ci[: nz.value], va[: nz.value], (nr.value, nc.value)

    def export_vec(self, lvl: int, which: int):
        """0 agg, 1 roots, 2 row types (int32); 3 B, 4 Bc, 5 Bhat, 6 Bhat_c (float64; n x k when k > 1)."""
        ln = C.c_int64()
        _check(rn_export_vec(self._h, lvl, which, C.byref(ln), None), "rn_export_vec")
        out = np.zeros(max(ln.value, 1), np.int32 if which <= 2 else np.float64)
        _check(rn_export_vec(self._h, lvl, which, C.byref(ln), out.ctypes.data), "rn_export_vec")
        out = out[: ln.value]
        k = getattr(self, "k", 1)
        return out.reshape(-1, k) if which >= 3 and k > 1 else out


def profile_enable(on: bool = True):
    _check(rn_profile_enable(1 if on else 0), "rn_profile_enable")


def profile_reset():
    _check(rn_profile_reset(), "rn_profile_reset")


def profile_read() -> dict:
    cnt = C.c_int()
    _check(rn_profile_read(None, 0, C.byref(cnt)), "rn_profile_read")
    arr = (rn_kernel_stat * max(cnt.value, 1))()
    _check(rn_profile_read(arr, cnt.value, C.byref(cnt)), "rn_profile_read")
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes)
            for i in range(cnt.value)}
