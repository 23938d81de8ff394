"""ctypes binding of the plain-C FP64 root-node AMG oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never uses it.

``build()`` compiles ``liboracle.so`` from the C sources in this directory with
``-O2 -ffp-contract=off`` (no fused multiply-add, so every a*b+c is a rounded
multiply then a rounded add, as the oracle's docstrings assume).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_sparse.c", "orc_setup.c", "orc_solve.c"]
HEADERS = ["orc.h", "orc_internal.h"]
LIB = os.path.join(HERE, "liboracle.so")

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ESINGULAR, ORC_ESTALL, ORC_ENOTCONV, ORC_EINTERNAL = 0, 1, 2, 3, 4, 5, 8
FREE, ROOT, UNAGG = 0, 1, 2


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES + HEADERS]
    if not force and os.path.exists(LIB):
        if os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs):
            return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall",
           "-fopenmp", "-o", LIB + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class _CSR(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.POINTER(C.c_int32)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double))]


class _Params(C.Structure):
    _fields_ = [("soc_theta", C.c_double), ("degree", C.c_int), ("n_sweeps", C.c_int), ("method", C.c_int),
                ("prefilter", C.c_double), ("postfilter", C.c_double), ("max_coarse", C.c_int),
                ("max_levels", C.c_int), ("b_sweeps", C.c_int), ("omega", C.c_double), ("seed", C.c_uint64),
                ("symmetric", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int), ("precond", C.c_int),
                ("soc_theta_coarse", C.c_double), ("gamma", C.c_int), ("soc_kind", C.c_int), ("ncand", C.c_int),
                ("block_size", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_res", C.c_double), ("rho", C.c_double), ("status", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_set_threads(1)  # one thread unless a caller asks for more (set_threads)
        i32p, dp = P(C.c_int32), P(C.c_double)
        L.orc_csr_free.argtypes = [P(_CSR)]
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_strength.argtypes = [P(_CSR), C.c_double, P(_CSR)]
        L.orc_strength_classical.argtypes = [P(_CSR), C.c_double, P(_CSR)]
        L.orc_tentative_k.argtypes = [P(_CSR), i32p, i32p, i32p, dp, C.c_int, dp]
        L.orc_project_k.argtypes = [P(_CSR), i32p, dp, C.c_int]
        L.orc_enforce_k.argtypes = [P(_CSR), i32p, dp, dp, C.c_int]
        L.orc_energy_min_cg_k.argtypes = [P(_CSR), P(_CSR), i32p, dp, C.c_int, C.c_int, C.c_int, dp]
        L.orc_smooth_candidates_k.argtypes = [P(_CSR), dp, C.c_int, C.c_int, C.c_double]
        L.orc_row_svd.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.orc_row_svd.restype = C.c_int
        L.orc_amalgamate.argtypes = [P(_CSR), C.c_int, P(_CSR)]
        L.orc_aggregate.argtypes = [P(_CSR), C.c_uint64, i32p, P(i32p), i32p]
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_smooth_candidates.argtypes = [P(_CSR), dp, C.c_int, C.c_double]
        L.orc_pattern.argtypes = [P(_CSR), i32p, i32p, C.c_int32, C.c_int, C.c_double, P(_CSR)]
        L.orc_row_types.argtypes = [C.c_int32, i32p, i32p, C.c_int32, i32p]
        L.orc_tentative.argtypes = [P(_CSR), i32p, i32p, dp, dp]
        L.orc_masked_product.argtypes = [P(_CSR), P(_CSR), P(_CSR)]
        L.orc_project.argtypes = [P(_CSR), i32p, dp]
        L.orc_energy_min_cg.argtypes = [P(_CSR), P(_CSR), i32p, dp, C.c_int, C.c_int, dp]
        L.orc_energy_min_gmres.argtypes = [P(_CSR), P(_CSR), i32p, dp, C.c_int, dp]
        L.orc_postfilter.argtypes = [P(_CSR), i32p, i32p, C.c_double, P(_CSR), P(C.c_int64)]
        L.orc_enforce.argtypes = [P(_CSR), i32p, dp, dp]
        L.orc_transpose.argtypes = [P(_CSR), P(_CSR)]
        L.orc_spgemm.argtypes = [P(_CSR), P(_CSR), P(_CSR)]
        L.orc_lu_factor.argtypes = [C.c_int, dp, i32p]
        L.orc_lu_solve.argtypes = [C.c_int, dp, i32p, dp]
        L.orc_setup.argtypes = [P(_CSR), dp, dp, P(_Params), P(C.c_void_p)]
        L.orc_hier_free.argtypes = [C.c_void_p]
        L.orc_hier_nlevels.argtypes = [C.c_void_p]
        L.orc_hier_csr.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_hier_csr.restype = P(_CSR)
        L.orc_hier_ivec.argtypes = [C.c_void_p, C.c_int, C.c_int, i32p]
        L.orc_hier_ivec.restype = i32p
        L.orc_hier_dvec.argtypes = [C.c_void_p, C.c_int, C.c_int, i32p]
        L.orc_hier_dvec.restype = dp
        L.orc_hier_near_ties.argtypes = [C.c_void_p]
        L.orc_hier_near_ties.restype = C.c_int64
        L.orc_vcycle.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_solve.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_int, C.c_int, C.c_int, P(_Info)]
        _lib = L
    return _lib


# ---------------------------------------------------------------- marshalling
def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))



def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's row loops; results do not depend on the count."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())

class _In:
    """Keeps numpy buffers alive while a _CSR view of them is passed to C."""

    def __init__(self, m, with_val=True):
        m = sp.csr_matrix(m)
        # private copies: several oracle routines update values in place
        self.rowptr = np.array(m.indptr, dtype=np.int32, copy=True)
        self.col = np.array(m.indices, dtype=np.int32, copy=True)
        self.val = np.array(m.data, dtype=np.float64, copy=True) if with_val else None
        self.s = _CSR(m.shape[0], m.shape[1], int(self.rowptr[-1]), _ip(self.rowptr), _ip(self.col),
                      _dp(self.val) if with_val else C.POINTER(C.c_double)())


def _out(c: _CSR, free=True) -> sp.csr_matrix:
    n, ncols, nnz = c.nrows, c.ncols, c.nnz
    rowptr = np.ctypeslib.as_array(c.rowptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(c.col, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    if c.val and nnz:
        val = np.ctypeslib.as_array(c.val, shape=(nnz,)).copy()
    else:
        val = np.zeros(nnz)
    if free:
        lib().orc_csr_free(C.byref(c))
    m = sp.csr_matrix((val, col, rowptr), shape=(n, ncols))
    m.has_sorted_indices = True
    return m


def _check(rc, what):
    if rc != ORC_OK:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# ------------------------------------------------------------------ step API
def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def strength(A, theta: float) -> sp.csr_matrix:
    a = _In(A)
    S = _CSR()
    _check(lib().orc_strength(C.byref(a.s), theta, C.byref(S)), "strength")
    return _out(S)


def strength_classical(A, theta: float) -> sp.csr_matrix:
    a = _In(A)
    S = _CSR()
    _check(lib().orc_strength_classical(C.byref(a.s), theta, C.byref(S)), "strength_classical")
    return _out(S)


def amalgamate(S, m: int) -> sp.csr_matrix:
    s_ = _In(S)
    out = _CSR()
    _check(lib().orc_amalgamate(C.byref(s_.s), m, C.byref(out)), "amalgamate")
    return _out(out)


def aggregate(S, seed: int):
    s = _In(S)
    n = s.s.nrows
    agg = np.zeros(n, np.int32)
    roots = C.POINTER(C.c_int32)()
    nc = C.c_int32()
    _check(lib().orc_aggregate(C.byref(s.s), C.c_uint64(seed), _ip(agg), C.byref(roots), C.byref(nc)), "aggregate")
    r = np.ctypeslib.as_array(roots, shape=(max(nc.value, 1),))[: nc.value].copy()
    roots = C.cast(roots, C.c_void_p)
    lib().orc_free(roots)
    return agg, r


def smooth_candidates(A, B, sweeps: int, omega: float) -> np.ndarray:
    a = _In(A)
    Bv = np.ascontiguousarray(B, dtype=np.float64).reshape(-1).copy()
    lib().orc_smooth_candidates(C.byref(a.s), _dp(Bv), sweeps, omega)
    return Bv


def row_types(n, agg, roots) -> np.ndarray:
    rt = np.zeros(n, np.int32)
    agg = np.ascontiguousarray(agg, np.int32)
    roots = np.ascontiguousarray(roots, np.int32)
    lib().orc_row_types(n, _ip(agg), _ip(roots), len(roots), _ip(rt))
    return rt


def pattern(S, agg, roots, d: int, theta_pre: float) -> sp.csr_matrix:
    s = _In(S)
    agg = np.ascontiguousarray(agg, np.int32)
    roots = np.ascontiguousarray(roots, np.int32)
    N = _CSR()
    _check(lib().orc_pattern(C.byref(s.s), _ip(agg), _ip(roots), len(roots), d, theta_pre, C.byref(N)), "pattern")
    return _out(N)


def tentative(N, agg, roots, B):
    n = _In(N)
    agg = np.ascontiguousarray(agg, np.int32)
    roots = np.ascontiguousarray(roots, np.int32)
    Bv = np.ascontiguousarray(B, np.float64).reshape(-1)
    Bc = np.zeros(N.shape[1])
    _check(lib().orc_tentative(C.byref(n.s), _ip(agg), _ip(roots), _dp(Bv), _dp(Bc)), "tentative")
    T = sp.csr_matrix((n.val.copy(), n.col.copy(), n.rowptr.copy()), shape=N.shape)
    return T, Bc


def masked_product(A, X) -> sp.csr_matrix:
    a, x = _In(A), _In(X)
    w = _In(X)
    lib().orc_masked_product(C.byref(a.s), C.byref(x.s), C.byref(w.s))
    return sp.csr_matrix((w.val, w.col, w.rowptr), shape=X.shape)


def row_svd(M: np.ndarray):
    """(U, V Sigma^+, rank) of a row's |J| x k matrix Bc_J (orc_row_svd)."""
    M = np.ascontiguousarray(M, np.float64)
    n, k = M.shape
    U = np.zeros((n, k))
    VS = np.zeros((k, k))
    rank = lib().orc_row_svd(n, k, _dp(M.reshape(-1)), _dp(U.reshape(-1)), _dp(VS.reshape(-1)))
    return U, VS, int(rank)


def tentative_k(N, agg, roots, rowtype, B):
    """T and Bc (nc x k) for the k columns of B (n x k)."""
    n = _In(N)
    B = np.ascontiguousarray(B, np.float64)
    k = B.shape[1]
    agg = np.ascontiguousarray(agg, np.int32)
    roots = np.ascontiguousarray(roots, np.int32)
    rt = np.ascontiguousarray(rowtype, np.int32)
    Bc = np.zeros((N.shape[1], k))
    _check(lib().orc_tentative_k(C.byref(n.s), _ip(agg), _ip(roots), _ip(rt), _dp(B.reshape(-1)), k, _dp(Bc)),
           "tentative_k")
    return sp.csr_matrix((n.val.copy(), n.col.copy(), n.rowptr.copy()), shape=N.shape), Bc


def project_k(W, rowtype, Bc) -> sp.csr_matrix:
    w = _In(W)
    Bc = np.ascontiguousarray(Bc, np.float64)
    lib().orc_project_k(C.byref(w.s), _ip(np.ascontiguousarray(rowtype, np.int32)), _dp(Bc), Bc.shape[1])
    return sp.csr_matrix((w.val, w.col, w.rowptr), shape=W.shape)


def energy_min_cg_k(A, P0, rowtype, Bc, sweeps: int, precond: int = 1):
    a, p = _In(A), _In(P0)
    Bc = np.ascontiguousarray(Bc, np.float64)
    trace = np.zeros(sweeps + 1)
    _check(lib().orc_energy_min_cg_k(C.byref(a.s), C.byref(p.s), _ip(np.ascontiguousarray(rowtype, np.int32)),
                                     _dp(Bc), Bc.shape[1], sweeps, precond, _dp(trace)), "energy_min_cg_k")
    return sp.csr_matrix((p.val, p.col, p.rowptr), shape=P0.shape), trace


def project(W, rowtype, Bc) -> sp.csr_matrix:
    w = _In(W)
    rt = np.ascontiguousarray(rowtype, np.int32)
    Bc = np.ascontiguousarray(Bc, np.float64)
    lib().orc_project(C.byref(w.s), _ip(rt), _dp(Bc))
    return sp.csr_matrix((w.val, w.col, w.rowptr), shape=W.shape)


def energy_min_cg(A, P0, rowtype, Bc, sweeps: int, precond: int = 1):
    a, p = _In(A), _In(P0)
    rt = np.ascontiguousarray(rowtype, np.int32)
    Bc = np.ascontiguousarray(Bc, np.float64)
    trace = np.zeros(sweeps + 1)
    _check(lib().orc_energy_min_cg(C.byref(a.s), C.byref(p.s), _ip(rt), _dp(Bc), sweeps, precond, _dp(trace)),
           "energy_min_cg")
    return sp.csr_matrix((p.val, p.col, p.rowptr), shape=P0.shape), trace


def energy_min_gmres(A, P0, rowtype, Bc, m: int):
    a, p = _In(A), _In(P0)
    rt = np.ascontiguousarray(rowtype, np.int32)
    Bc = np.ascontiguousarray(Bc, np.float64)
    trace = np.zeros(m + 1)
    _check(lib().orc_energy_min_gmres(C.byref(a.s), C.byref(p.s), _ip(rt), _dp(Bc), m, _dp(trace)),
           "energy_min_gmres")
    return sp.csr_matrix((p.val, p.col, p.rowptr), shape=P0.shape), trace


def postfilter(P, agg, rowtype, theta: float):
    p = _In(P)
    agg = np.ascontiguousarray(agg, np.int32)
    rt = np.ascontiguousarray(rowtype, np.int32)
    out = _CSR()
    ties = C.c_int64(0)
    _check(lib().orc_postfilter(C.byref(p.s), _ip(agg), _ip(rt), theta, C.byref(out), C.byref(ties)),
           "postfilter")
    return _out(out), ties.value


def enforce(P, rowtype, B, Bc) -> sp.csr_matrix:
    p = _In(P)
    rt = np.ascontiguousarray(rowtype, np.int32)
    B = np.ascontiguousarray(B, np.float64).reshape(-1)
    Bc = np.ascontiguousarray(Bc, np.float64)
    lib().orc_enforce(C.byref(p.s), _ip(rt), _dp(B), _dp(Bc))
    return sp.csr_matrix((p.val, p.col, p.rowptr), shape=P.shape)


def transpose(A) -> sp.csr_matrix:
    a = _In(A)
    out = _CSR()
    _check(lib().orc_transpose(C.byref(a.s), C.byref(out)), "transpose")
    return _out(out)


def spgemm(A, B) -> sp.csr_matrix:
    a, b = _In(A), _In(B)
    out = _CSR()
    _check(lib().orc_spgemm(C.byref(a.s), C.byref(b.s), C.byref(out)), "spgemm")
    return _out(out)


def lu_solve_dense(M: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    n = M.shape[0]
    LU = np.ascontiguousarray(M, np.float64).copy()
    piv = np.zeros(n, np.int32)
    _check(lib().orc_lu_factor(n, _dp(LU), _ip(piv)), "lu_factor")
    x = np.ascontiguousarray(rhs, np.float64).copy()
    lib().orc_lu_solve(n, _dp(LU), _ip(piv), _dp(x))
    return x


# ------------------------------------------------------------ full setup/solve
def make_params(**kw) -> _Params:
    d = dict(soc_theta=0.25, degree=2, n_sweeps=4, method=0, prefilter=0.0, postfilter=0.0, max_coarse=64,
             max_levels=25, b_sweeps=4, omega=2.0 / 3.0, seed=12345, symmetric=1, nu_pre=1, nu_post=1, precond=1,
             soc_theta_coarse=-1.0, gamma=1, soc_kind=0, ncand=1, block_size=1)
    for k, v in kw.items():
        if k in d:
            d[k] = v
    return _Params(**d)


@dataclass
class Level:
    A: sp.csr_matrix
    S: sp.csr_matrix | None = None
    N: sp.csr_matrix | None = None
    T: sp.csr_matrix | None = None
    P: sp.csr_matrix | None = None
    R: sp.csr_matrix | None = None
    agg: np.ndarray | None = None
    roots: np.ndarray | None = None
    rowtype: np.ndarray | None = None
    B: np.ndarray | None = None
    Bc: np.ndarray | None = None
    Bhat: np.ndarray | None = None
    Bhatc: np.ndarray | None = None


class Hierarchy:
    """Owns an oracle hierarchy handle; ``levels`` holds numpy/scipy copies."""

    def __init__(self, A, B, Bhat=None, **params):
        self.params = params
        self._p = make_params(**params)
        a = _In(A)
        Bv = np.ascontiguousarray(B, np.float64).reshape(-1)
        Bh = np.ascontiguousarray(Bhat, np.float64).reshape(-1) if Bhat is not None else None
        h = C.c_void_p()
        rc = lib().orc_setup(C.byref(a.s), _dp(Bv), _dp(Bh) if Bh is not None else C.POINTER(C.c_double)(),
                             C.byref(self._p), C.byref(h))
        _check(rc, "setup")
        self._h = h
        self.n = A.shape[0]
        self.levels = []
        L = lib()
        nlev = L.orc_hier_nlevels(h)
        for l in range(nlev):
            def csr(which):
                c = L.orc_hier_csr(h, l, which)
                if not c or not c.contents.rowptr:
                    return None
                return _out(c.contents, free=False)

            def ivec(which):
                ln = C.c_int32()
                p = L.orc_hier_ivec(h, l, which, C.byref(ln))
                return np.ctypeslib.as_array(p, shape=(ln.value,)).copy() if p and ln.value > 0 else None

            kc = max(1, int(params.get("ncand", 1)))

            def dvec(which):
                ln = C.c_int32()
                p = L.orc_hier_dvec(h, l, which, C.byref(ln))
                if not (p and ln.value > 0):
                    return None
                v = np.ctypeslib.as_array(p, shape=(ln.value,)).copy()
                return v if kc == 1 else v.reshape(-1, kc)

            self.levels.append(Level(A=csr(0), S=csr(1), N=csr(2), T=csr(3), P=csr(4), R=csr(5), agg=ivec(0),
                                     roots=ivec(1), rowtype=ivec(2), B=dvec(0), Bc=dvec(1), Bhat=dvec(2),
                                     Bhatc=dvec(3)))
        self.near_ties = int(L.orc_hier_near_ties(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_hier_free(h)
            self._h = None

    def vcycle(self, b: np.ndarray, x: np.ndarray | None = None) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n) if x is None else np.ascontiguousarray(x, np.float64).copy()
        lib().orc_vcycle(self._h, 0, _dp(b), _dp(x))
        return x

    def solve(self, b, tol=1e-8, maxit=500, outer=0, restart=30, x0=None):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n) if x0 is None else np.ascontiguousarray(x0, np.float64).copy()
        info = _Info()
        lib().orc_solve(self._h, _dp(b), _dp(x), tol, maxit, outer, restart, C.byref(info))
        return x, dict(iters=info.iters, rel_res=info.rel_res, rho=info.rho, status=info.status)

    def stats(self):
        nnzA0 = self.levels[0].A.nnz
        oc = sum(L.A.nnz for L in self.levels) / nnzA0
        nu = self.params.get("nu_pre", 1) + self.params.get("nu_post", 1)
        cc = sum((nu + 1) * L.A.nnz + (L.P.nnz if L.P is not None else 0) + (L.R.nnz if L.R is not None else 0)
                 for L in self.levels[:-1]) / nnzA0
        return dict(levels=len(self.levels), n=[L.A.shape[0] for L in self.levels],
                    nnz=[L.A.nnz for L in self.levels], oc=oc, cc=cc)
