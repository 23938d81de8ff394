"""Pins for the CPU oracle: each test checks it against something other than
itself - closed forms, dense brute force written independently here in numpy,
special cases with known answers, and the paper's worked examples.

These run without a GPU (``-m "not gpu"``).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from paper_1610_03154_gb300 import problems as PR
from tests.conftest import read_golden

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


# --------------------------------------------------------------------------- generators
def test_q1_laplacian_50x50_nnz_matches_paper():
    g = read_golden("q1_laplacian_50x50.txt")
    A = PR.q1_aniso(49, 1.0, 0.0, dirichlet=False)
    assert A.n_rows == int(g["n"][0])
    assert A.nnz == int(g["nnz"][0])


@pytest.mark.parametrize("m", [5, 8, 12])
def test_poisson5_spectrum_closed_form(m):
    # eigenvalues of the unscaled 5-point Laplacian: 4 sin^2(j pi h/2) + 4 sin^2(k pi h/2), h = 1/(m+1)
    A = PR.poisson5(m).to_scipy().toarray()
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam1 = 4 * np.sin(j * np.pi * h / 2) ** 2
    expect = np.sort((lam1[:, None] + lam1[None, :]).ravel())
    assert np.allclose(np.linalg.eigvalsh(A), expect, atol=1e-12)


def test_q1_aniso_unrotated_spectrum_is_separable():
    # psi = 0: K = diag(1, eps).  The Q1 stiffness is a sum of Kronecker products
    # of 1-D stiffness and mass matrices; check against that construction.
    ne, eps = 7, 1e-3
    A = PR.q1_aniso(ne, eps, 0.0).to_scipy().toarray()
    m = ne - 1
    K1 = (np.diag(2 * np.ones(m)) - np.diag(np.ones(m - 1), 1) - np.diag(np.ones(m - 1), -1))
    M1 = (np.diag(4 * np.ones(m)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)) / 6.0
    # x fastest: A = M_y (x) K_x + eps K_y (x) M_x  (element size cancels in 2-D)
    expect = np.kron(M1, K1) + eps * np.kron(K1, M1)
    assert np.allclose(A, expect, atol=1e-14)


def test_convdiff_upwind_is_m_matrix_and_nnz():
    m = 16
    A = PR.convdiff_upwind(m).to_scipy()
    assert A.nnz == 5 * m * m - 4 * m
    D = A.diagonal()
    off = A - sp.diags(D)
    assert (D > 0).all() and (off.data <= 0).all()
    # weak diagonal dominance by rows (strict where a boundary neighbour was eliminated)
    assert (D + np.asarray(off.sum(axis=1)).ravel() >= -1e-12).all()
    # half-grid Reynolds number of the 2048^2 workload is in the good regime (Sec. 5.3 remark)
    h = 2.0 / 2049
    assert max(abs(2 * 1.0 * (1 - 0.0)), 2.0) * h / (2 * 1e-3) < 1.25


def test_splitmix64_published_values(oracle):
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0 yields 0xE220A8397B1DCDAF,
    # then 0x6E789E6AA1B965F4: output k is mix(seed + k*golden), k = 1, 2.
    golden = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(golden) == 0x6E789E6AA1B965F4


# --------------------------------------------------------------------------- strength
def test_strength_poisson_all_neighbours_strong(oracle):
    # 5-point Laplacian: |a_ij|/sqrt(a_ii a_jj) = 1/4 exactly = theta (the tie the
    # guard band resolves to 'strong'); after scaling every entry is 1.
    A = PR.poisson5(10).to_scipy()
    S = oracle.strength(A, 0.25)
    assert S.nnz == A.nnz
    assert np.array_equal(S.indices, A.indices) and np.array_equal(S.indptr, A.indptr)
    assert np.all(S.data == 1.0)


def test_strength_grid_aligned_anisotropy(oracle):
    # psi = 0, eps = 1e-3: only the x-neighbours (same grid row) are strong.
    ne = 9
    m = ne - 1
    A = PR.q1_aniso(ne, 1e-3, 0.0).to_scipy()
    S = oracle.strength(A, 0.25)
    for i in range(A.shape[0]):
        cols = S.indices[S.indptr[i]:S.indptr[i + 1]]
        for j in cols:
            if j != i:
                assert j // m == i // m and abs(j - i) == 1
        xi = i % m
        assert len(cols) == 1 + (xi > 0) + (xi < m - 1)


def test_strength_normalisation_invariants(oracle):
    A = PR.q1_aniso(12, 1e-2, math.pi / 6).to_scipy()
    S = oracle.strength(A, 0.25)
    Ad = A.toarray()
    d = np.diag(Ad)
    for i in range(A.shape[0]):
        cols = S.indices[S.indptr[i]:S.indptr[i + 1]]
        vals = S.data[S.indptr[i]:S.indptr[i + 1]]
        assert vals[cols == i][0] == 1.0
        off = vals[cols != i]
        if off.size:
            assert off.max() == 1.0 and off.min() > 0
        # brute force strong set
        v = np.abs(Ad[i]) / np.sqrt(np.abs(d[i] * d))
        v[i] = 0
        strong = set(np.nonzero(v >= 0.25 * (1 - 1e-10))[0])
        assert strong == set(cols[cols != i])


# --------------------------------------------------------------------------- aggregation
def _graph(S):
    G = (abs(S) + abs(S).T).tocsr()
    G.setdiag(0)
    G.eliminate_zeros()
    return (G != 0).astype(int).tocsr()


def _prio(oracle, seed, n):
    return [(oracle.splitmix64(seed ^ i), i) for i in range(n)]


def _mis2_parallel_rounds(G, prio):
    """Independent restatement: rounds in which an undecided node joins if its
    priority beats every undecided node within distance 2."""
    n = G.shape[0]
    G2 = ((G + G @ G) != 0).astype(int).toarray()
    np.fill_diagonal(G2, 0)
    isolated = np.asarray(G.sum(axis=1)).ravel() == 0
    state = np.where(isolated, -2, 0)  # 0 undecided, 1 root, -1 removed, -2 isolated
    while (state == 0).any():
        new = []
        for i in np.nonzero(state == 0)[0]:
            nb = np.nonzero(G2[i])[0]
            if all(prio[i] > prio[j] for j in nb if state[j] == 0):
                new.append(i)
        assert new
        for i in new:
            state[i] = 1
        for i in new:
            for j in np.nonzero(G2[i])[0]:
                if state[j] == 0:
                    state[j] = -1
    return np.nonzero(state == 1)[0]


@pytest.mark.parametrize("case", ["poisson", "aniso", "convdiff"])
def test_aggregation_mis2_bruteforce(oracle, case):
    if case == "poisson":
        A = PR.poisson5(14).to_scipy()
    elif case == "aniso":
        A = PR.q1_aniso(14, 1e-3, math.pi / 8).to_scipy()
    else:
        A = PR.convdiff_upwind(14).to_scipy()
    S = oracle.strength(A, 0.25)
    seed = 777
    agg, roots = oracle.aggregate(S, seed)
    G = _graph(S)
    n = A.shape[0]
    prio = _prio(oracle, seed, n)
    # roots: sorted, equal to the parallel-rounds MIS-2
    assert np.all(np.diff(roots) > 0)
    assert np.array_equal(roots, _mis2_parallel_rounds(G, prio))
    # independence at distance 2 and maximality
    G2 = ((G + G @ G) != 0).toarray()
    np.fill_diagonal(G2, False)
    rs = set(roots.tolist())
    for r in roots:
        assert not any(j in rs for j in np.nonzero(G2[r])[0])
    isolated = np.asarray(G.sum(axis=1)).ravel() == 0
    for i in range(n):
        if not isolated[i] and i not in rs:
            assert any(j in rs for j in np.nonzero(G2[i])[0])
    # assignment: roots own their aggregate; every non-isolated node aggregated;
    # pass 1 picks the neighbouring root of largest priority
    for c, r in enumerate(roots):
        assert agg[r] == c
    assert np.all((agg >= 0) == ~isolated)
    Gd = G.toarray()
    for i in range(n):
        if isolated[i] or i in rs:
            continue
        nbr_roots = [j for j in np.nonzero(Gd[i])[0] if j in rs]
        if nbr_roots:
            best = max(nbr_roots, key=lambda j: prio[j])
            assert agg[i] == agg[best]
        else:
            # pass 2: some neighbour with a root neighbour carries agg[i]
            cands = [j for j in np.nonzero(Gd[i])[0] if any(k in rs for k in np.nonzero(Gd[j])[0])]
            assert agg[i] in {agg[j] for j in cands}


# --------------------------------------------------------------------------- pattern
def test_pattern_is_boolean_power_without_filter(oracle):
    A = PR.q1_aniso(10, 1e-2, math.pi / 8).to_scipy()
    S = oracle.strength(A, 0.25)
    agg, roots = oracle.aggregate(S, 5)
    n, nc = A.shape[0], len(roots)
    Cm = np.zeros((n, nc))
    Cm[agg >= 0, agg[agg >= 0]] = 1.0
    for d in (1, 2, 3):
        N = oracle.pattern(S, agg, roots, d, 0.0)
        Nd = np.linalg.matrix_power(S.toarray(), d) @ Cm
        # root rows become identity rows; everything else is the boolean power
        expect = Nd != 0
        expect[roots, :] = False
        expect[roots, agg[roots]] = True
        assert np.array_equal(N.toarray() != 0, expect)
        Nv = N.toarray()
        free = (agg >= 0)
        free[roots] = False
        assert np.allclose(Nv[free], Nd[free], rtol=1e-14, atol=0)


def test_prefilter_keeps_relative_large_and_own_aggregate(oracle):
    A = PR.q1_aniso(12, 1e-3, math.pi / 8).to_scipy()
    S = oracle.strength(A, 0.25)
    agg, roots = oracle.aggregate(S, 9)
    n, nc = A.shape[0], len(roots)
    Cm = np.zeros((n, nc))
    Cm[agg >= 0, agg[agg >= 0]] = 1.0
    Nd = np.linalg.matrix_power(S.toarray(), 3) @ Cm
    N = oracle.pattern(S, agg, roots, 3, 0.2).toarray()
    rs = set(roots.tolist())
    for i in range(n):
        if agg[i] < 0 or i in rs:
            continue
        keep = Nd[i] >= 0.2 * Nd[i].max() * (1 - 1e-10)
        keep[agg[i]] = True
        keep &= Nd[i] != 0
        assert np.array_equal(N[i] != 0, keep)


def test_tentative_paper_1d_example(oracle):
    # eq. exampleinterp: RN T with B = 1 on the given aggregates is C itself
    g = read_golden("agg1d_example.txt")
    n = int(g["n"][0])
    agg = np.array([int(v) for v in g["agg"]], np.int32)
    Cm = np.array([[float(v) for v in row] for row in g["C"]])
    roots = np.array([1, 3, 6], np.int32)  # any member may be the root when B = 1
    N = sp.csr_matrix(Cm)
    T, Bc = oracle.tentative(N, agg, roots, np.ones(n))
    assert np.array_equal(T.toarray(), Cm)
    assert np.array_equal(Bc, np.ones(3))


def test_tentative_constraints_and_roots(oracle):
    A = PR.poisson5(12).to_scipy()
    S = oracle.strength(A, 0.25)
    agg, roots = oracle.aggregate(S, 3)
    N = oracle.pattern(S, agg, roots, 2, 0.0)
    B = oracle.smooth_candidates(A, np.ones(A.shape[0]), 4, 2 / 3)
    T, Bc = oracle.tentative(N, agg, roots, B)
    assert np.allclose(T @ Bc, B, rtol=1e-13, atol=0)
    Td = T.toarray()
    for c, r in enumerate(roots):
        e = np.zeros(len(roots))
        e[c] = 1.0
        assert np.array_equal(Td[r], e)


def test_candidate_smoothing_is_jacobi_matrix_power(oracle):
    A = PR.q1_aniso(8, 1e-2, 0.3).to_scipy()
    B0 = np.ones(A.shape[0])
    Ad = A.toarray()
    G = np.eye(A.shape[0]) - (2 / 3) * np.diag(1 / np.diag(Ad)) @ Ad
    expect = np.linalg.matrix_power(G, 4) @ B0
    got = oracle.smooth_candidates(A, B0, 4, 2 / 3)
    assert np.allclose(got, expect, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------- energy minimisation
def _setup_level(oracle, A, d, seed=1, theta=0.25, B=None):
    S = oracle.strength(A, theta)
    agg, roots = oracle.aggregate(S, seed)
    N = oracle.pattern(S, agg, roots, d, 0.0)
    rt = oracle.row_types(A.shape[0], agg, roots)
    if B is None:
        B = np.ones(A.shape[0])
    T, Bc = oracle.tentative(N, agg, roots, B)
    return dict(S=S, agg=agg, roots=roots, N=N, rt=rt, T=T, Bc=Bc, B=B)


class _Dense:
    """Vectorised free entries of P (entries of free rows on the pattern)."""

    def __init__(self, A, N, rt, Bc):
        self.A = A.toarray()
        self.N = N
        n, nc = N.shape
        I, J = [], []
        for i in range(n):
            if rt[i] == 0:
                for j in N.indices[N.indptr[i]:N.indptr[i + 1]]:
                    I.append(i)
                    J.append(j)
        self.I, self.J = np.array(I), np.array(J)
        m = len(I)
        self.H = self.A[np.ix_(self.I, self.I)] * (self.J[:, None] == self.J[None, :])
        rows = sorted(set(I))
        rix = {r: k for k, r in enumerate(rows)}
        Cm = np.zeros((len(rows), m))
        for t in range(m):
            Cm[rix[I[t]], t] = Bc[J[t]]
        self.Cm = Cm
        self.Pi = np.eye(m) - Cm.T @ np.linalg.solve(Cm @ Cm.T, Cm)
        self.rt = rt
        self.fixed = np.zeros((n, nc))

    def full(self, x, P0):
        X = P0.toarray().copy()
        X[self.I, self.J] = x
        return X

    def grad(self, X):  # (A X) on the free entries
        return (self.A @ X)[self.I, self.J]


def test_cg_converges_to_ideal_interpolation_lemma(oracle):
    # Lemma th:cg: over the full F x C pattern, minimising the columns of [W; I]
    # in the A-norm gives P_ideal = [-A_ff^{-1} A_fc; I].  A Neumann Laplacian
    # (row sums 0) makes P_ideal 1 = 1, so the constraint P Bc = B (B = 1) is
    # inactive at the optimum.
    A = PR.q1_aniso(6, 1.0, 0.0, dirichlet=False).to_scipy()
    n = A.shape[0]
    # Q1 Laplacian: every normalised off-diagonal is 1/8, so theta = 0.1 keeps them all
    lev = _setup_level(oracle, A, 1, theta=0.1)
    assert np.all(lev["rt"] != 2)
    agg, roots, rt = lev["agg"], lev["roots"], lev["rt"]
    nc = len(roots)
    full = np.zeros((n, nc))
    full[rt == 0, :] = 1.0
    full[roots, agg[roots]] = 1.0
    N = sp.csr_matrix(full)
    T, Bc = oracle.tentative(N, agg, roots, np.ones(n))
    P, trace = oracle.energy_min_cg(A, T, rt, Bc, 400)
    Ad = A.toarray()
    F = np.nonzero(rt == 0)[0]
    Pideal = np.zeros((n, nc))
    Pideal[roots, np.arange(nc)] = 1.0
    Pideal[F] = -np.linalg.solve(Ad[np.ix_(F, F)], Ad[np.ix_(F, roots)])
    assert np.allclose(P.toarray(), Pideal, atol=1e-10)


@pytest.mark.parametrize("precond", [1, 0])
def test_cg_converged_equals_dense_kkt(oracle, precond):
    A = PR.poisson5(7).to_scipy()
    rng = np.random.default_rng(0)
    B = 1.0 + 0.3 * rng.random(A.shape[0])
    lev = _setup_level(oracle, A, 2, B=B)
    D = _Dense(A, lev["N"], lev["rt"], lev["Bc"])
    # minimise sum_j p_j^T A p_j over free entries x subject to Cm x = B_free
    X0 = lev["T"].toarray().copy()
    X0[D.I, D.J] = 0.0
    h = D.grad(X0)
    m = len(D.I)
    rows = sorted(set(D.I.tolist()))
    K = np.block([[2 * D.H, D.Cm.T], [D.Cm, np.zeros((len(rows), len(rows)))]])
    rhs = np.concatenate([-2 * h, B[rows]])
    x = np.linalg.solve(K, rhs)[:m]
    P, trace = oracle.energy_min_cg(A, lev["T"], lev["rt"], lev["Bc"], 600, precond)
    assert np.allclose(P.toarray()[D.I, D.J], x, atol=1e-10)
    assert np.allclose(P @ lev["Bc"], np.where(lev["agg"] >= 0, B, 0.0), atol=1e-13)


def test_cg_fixed_sweeps_equals_dense_pcg_and_energy_decreases(oracle):
    A = PR.q1_aniso(9, 1e-2, math.pi / 8).to_scipy()
    lev = _setup_level(oracle, A, 2)
    D = _Dense(A, lev["N"], lev["rt"], lev["Bc"])
    T = lev["T"]
    sweeps = 5
    P, trace = oracle.energy_min_cg(A, T, lev["rt"], lev["Bc"], sweeps)
    # dense projected PCG on the vectorised free entries, same recurrences
    dinv = 1.0 / np.diag(D.A)[D.I]
    x = T.toarray()[D.I, D.J].copy()
    r = -D.Pi @ D.grad(D.full(x, T))
    d = None
    rho_old = None
    for it in range(sweeps):
        z = dinv * r
        rho = r @ z
        d = z if it == 0 else z + (rho / rho_old) * d
        w = D.Pi @ (D.H @ d)
        alpha = rho / (d @ w)
        x = x + alpha * d
        r = r - alpha * w
        rho_old = rho
    assert np.allclose(P.toarray()[D.I, D.J], x, rtol=1e-12, atol=1e-13)
    assert np.all(np.diff(trace) <= 1e-12 * abs(trace[0]))
    # energy = trace(P^T A P)
    Pd = P.toarray()
    assert np.isclose(trace[-1], np.trace(Pd.T @ D.A @ Pd), rtol=1e-12)


def test_gmres_fixed_steps_is_krylov_least_squares(oracle):
    A = PR.convdiff_upwind(9, 0.05).to_scipy()
    lev = _setup_level(oracle, A, 1)
    D = _Dense(A, lev["N"], lev["rt"], lev["Bc"])
    T = lev["T"]
    for m in (1, 2, 3):
        P, res = oracle.energy_min_gmres(A, T, lev["rt"], lev["Bc"], m)
        Aop = D.Pi @ D.H
        xT = T.toarray()[D.I, D.J]
        r0 = -D.Pi @ D.grad(D.full(xT, T))
        K = np.stack([np.linalg.matrix_power(Aop, k) @ r0 for k in range(m)], axis=1)
        y, *_ = np.linalg.lstsq(Aop @ K, r0, rcond=None)
        x = xT + K @ y
        assert np.allclose(P.toarray()[D.I, D.J], x, rtol=1e-10, atol=1e-12)
        assert np.all(np.diff(res) <= 1e-12 * res[0])
        assert np.isclose(res[-1], np.linalg.norm(r0 - Aop @ K @ y), rtol=1e-10)


def test_postfilter_and_enforce(oracle):
    A = PR.q1_aniso(12, 1e-3, math.pi / 8).to_scipy()
    B = oracle.smooth_candidates(A, np.ones(A.shape[0]), 4, 2 / 3)
    lev = _setup_level(oracle, A, 3, B=B)
    P, _ = oracle.energy_min_cg(A, lev["T"], lev["rt"], lev["Bc"], 4)
    Pf, ties = oracle.postfilter(P, lev["agg"], lev["rt"], 0.1)
    Pd, Pfd = P.toarray(), Pf.toarray()
    for i in range(A.shape[0]):
        if lev["rt"][i] != 0:
            assert np.array_equal(Pd[i] != 0, Pfd[i] != 0) or lev["rt"][i] == 2
            continue
        cols = P.indices[P.indptr[i]:P.indptr[i + 1]]
        v = np.abs(Pd[i, cols])
        keep = cols[(v >= 0.1 * v.max() * (1 - 1e-10)) | (cols == lev["agg"][i])]
        assert np.array_equal(Pf.indices[Pf.indptr[i]:Pf.indptr[i + 1]], keep)
    Pe = oracle.enforce(Pf, lev["rt"], B, lev["Bc"])
    aggd = lev["agg"] >= 0
    assert np.allclose((Pe @ lev["Bc"])[aggd], B[aggd], rtol=1e-13, atol=0)
    # minimal-norm: the update is a multiple of Bc on the row's pattern
    dd = (Pe - Pf).toarray()
    for i in np.nonzero(lev["rt"] == 0)[0][:50]:
        cols = Pf.indices[Pf.indptr[i]:Pf.indptr[i + 1]]
        u, b = dd[i, cols], lev["Bc"][cols]
        assert np.allclose(u, (u @ b) / (b @ b) * b, atol=1e-15)


# --------------------------------------------------------------------------- sparse products, LU
def test_transpose_and_spgemm_against_dense(oracle):
    rng = np.random.default_rng(3)
    A = sp.random(40, 30, density=0.1, random_state=rng, format="csr")
    B = sp.random(30, 50, density=0.1, random_state=rng, format="csr")
    At = oracle.transpose(A)
    assert np.array_equal(At.toarray(), A.toarray().T)
    Cm = oracle.spgemm(A, B)
    assert np.allclose(Cm.toarray(), A.toarray() @ B.toarray(), rtol=1e-14, atol=1e-15)
    sym = ((A != 0).astype(int) @ (B != 0).astype(int)).toarray() != 0
    assert np.array_equal(Cm.toarray() != 0 if Cm.nnz else sym, sym) or True
    # pattern is exactly the symbolic product (explicit zeros kept)
    pat = np.zeros(sym.shape, bool)
    for i in range(Cm.shape[0]):
        pat[i, Cm.indices[Cm.indptr[i]:Cm.indptr[i + 1]]] = True
    assert np.array_equal(pat, sym)


def test_masked_product_and_projection(oracle):
    A = PR.poisson5(9).to_scipy()
    lev = _setup_level(oracle, A, 2)
    X = lev["T"].copy()
    X.data = np.random.default_rng(1).standard_normal(X.nnz)
    W = oracle.masked_product(A, X)
    full = (A @ X).toarray()
    mask = X.toarray() != 0
    pat = np.zeros(X.shape, bool)
    for i in range(X.shape[0]):
        pat[i, X.indices[X.indptr[i]:X.indptr[i + 1]]] = True
    assert np.allclose(W.toarray(), np.where(pat, full, 0.0), rtol=1e-13, atol=1e-14)
    Wp = oracle.project(W, lev["rt"], lev["Bc"])
    assert np.allclose((Wp @ lev["Bc"]), 0.0, atol=1e-13)
    assert np.all(Wp.toarray()[lev["rt"] != 0] == 0.0)
    del mask


def test_galerkin_rap_dense_and_symmetry(oracle):
    pr = PR.poisson_problem(20)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    for l in range(len(h.levels) - 1):
        L, Lc = h.levels[l], h.levels[l + 1]
        Ad, Pd, Rd = L.A.toarray(), L.P.toarray(), L.R.toarray()
        assert np.array_equal(Rd, Pd.T)
        Ac = Rd @ Ad @ Pd
        assert np.allclose(Lc.A.toarray(), Ac, rtol=0, atol=1e-13 * np.abs(Ac).max())
        Acd = Lc.A.toarray()
        assert np.array_equal(Acd != 0, (Acd != 0).T) or np.array_equal(
            np.sort(Lc.A.indices), np.sort(Lc.A.tocsc().indices))
        assert np.allclose(Acd, Acd.T, rtol=0, atol=1e-15 * np.abs(Acd).max())


def test_lu_against_numpy_and_singular(oracle):
    rng = np.random.default_rng(5)
    M = rng.standard_normal((30, 30))
    b = rng.standard_normal(30)
    assert np.allclose(oracle.lu_solve_dense(M, b), np.linalg.solve(M, b), rtol=1e-11)
    M[:, 3] = M[:, 7]
    with pytest.raises(RuntimeError):
        oracle.lu_solve_dense(M, b)


# --------------------------------------------------------------------------- hierarchy, cycle, solve
def test_hierarchy_invariants(oracle):
    pr = PR.aniso_problem(32)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    assert len(h.levels) >= 2
    for l in range(len(h.levels) - 1):
        L = h.levels[l]
        Pd = L.P.toarray()
        for c, r in enumerate(L.roots):
            e = np.zeros(len(L.roots))
            e[c] = 1.0
            assert np.array_equal(Pd[r], e)  # P_C = I
        aggd = L.agg >= 0
        assert np.allclose((L.P @ L.Bc)[aggd], L.B[aggd], rtol=0, atol=1e-13)  # P Bc = B
        # P lives on the (filtered) pattern: subset of N
        Nd = L.N.toarray() != 0
        assert not np.any((Pd != 0) & ~Nd)


def test_two_grid_factor_matches_dense_spectral_radius(oracle):
    pr = PR.poisson_problem(16)
    params = dict(pr.params)
    params["max_coarse"] = 200  # two levels: the coarse level is solved exactly
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **params)
    assert len(h.levels) == 2
    L = h.levels[0]
    Ad, Pd, Rd = L.A.toarray(), L.P.toarray(), L.R.toarray()
    n = Ad.shape[0]
    G = np.eye(n) - (2 / 3) * np.diag(1 / np.diag(Ad)) @ Ad
    E = G @ (np.eye(n) - Pd @ np.linalg.solve(Rd @ Ad @ Pd, Rd @ Ad)) @ G
    rho = max(abs(np.linalg.eigvals(E)))
    x = np.random.default_rng(0).standard_normal(n)
    zero = np.zeros(n)
    ratio = 0.0
    for _ in range(300):
        y = h.vcycle(zero, x)
        ratio = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    assert abs(ratio - rho) < 1e-3


@pytest.mark.parametrize("outer", [0, 1, 2])
def test_solve_matches_direct_solver(oracle, outer):
    pr = PR.poisson_problem(32)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    x, info = h.solve(pr.b, tol=1e-8, outer=outer)
    A = pr.A.to_scipy()
    assert info["status"] == 0
    assert np.linalg.norm(pr.b - A @ x) / np.linalg.norm(pr.b) < 1e-8
    xe = sla.spsolve(A.tocsc(), pr.b)
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) < cond * 1e-8


def test_nonsymmetric_solve_gmres(oracle):
    # R^T is built from A^T on the same pattern and roots: without a
    # post-filter (which drops entries of P and R^T by their own values) R^T
    # has P's pattern
    pr = PR.convdiff_problem(32, params=PR.PARAMS_CONVDIFF_RN1)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, Bhat=pr.Bhat, **pr.params)
    assert len(h.levels) >= 2
    L = h.levels[0]
    Rt = L.R.T.tocsr()
    assert np.array_equal(Rt.indptr, L.P.indptr) and np.array_equal(Rt.indices, L.P.indices)
    A = pr.A.to_scipy()
    for params in (PR.PARAMS_CONVDIFF_RN1, PR.PARAMS_CONVDIFF):
        h = oracle.Hierarchy(A, pr.B, Bhat=pr.Bhat, **params)
        x, info = h.solve(pr.b, tol=1e-8, outer=2, restart=30)
        assert info["status"] == 0
        assert np.linalg.norm(pr.b - A @ x) / np.linalg.norm(pr.b) < 1e-8


def test_one_level_hierarchy_is_exact(oracle):
    pr = PR.poisson_problem(6)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    assert len(h.levels) == 1
    x, info = h.solve(pr.b, tol=1e-12, outer=0)
    xe = np.linalg.solve(pr.A.to_scipy().toarray(), pr.b)
    assert np.allclose(x, xe, rtol=1e-13, atol=1e-14)
    assert info["iters"] <= 1


def test_operator_and_cycle_complexity_formulas(oracle):
    pr = PR.poisson_problem(32)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    st = h.stats()
    nnz = [L.A.nnz for L in h.levels]
    assert st["oc"] == sum(nnz) / nnz[0]  # eq. oc
    cc = sum(3 * L.A.nnz + L.P.nnz + L.R.nnz for L in h.levels[:-1]) / nnz[0]  # eq. cc, V(1,1)
    assert st["cc"] == cc


def test_single_entry_rows_have_empty_constraint_space(oracle):
    # a free row whose pattern is only its own aggregate cannot move: U Bc = 0
    # on one entry forces U = 0, so energy minimisation returns T unchanged
    A = PR.poisson5(9).to_scipy()
    lev = _setup_level(oracle, A, 0)  # d = 0: N = C, one entry per aggregated row
    assert np.all(np.diff(lev["N"].indptr)[lev["agg"] >= 0] == 1)
    P, trace = oracle.energy_min_cg(A, lev["T"], lev["rt"], lev["Bc"], 6)
    assert np.array_equal(P.toarray(), lev["T"].toarray())
    Pg, res = oracle.energy_min_gmres(A, lev["T"], lev["rt"], lev["Bc"], 3)
    assert np.array_equal(Pg.toarray(), lev["T"].toarray())


def test_energy_monotone_on_every_level(oracle):
    pr = PR.aniso_problem(96)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    for L in h.levels[:-1]:
        P, tr = oracle.energy_min_cg(L.A, L.T, L.rowtype, L.Bc, 6)
        assert np.all(np.diff(tr) <= 1e-12 * abs(tr[0])), tr


# --------------------------------------------------------------------------- adjoint reference
def test_adjoint_reference_gradient_matches_central_differences():
    """The hand-derived adjoint gradient of the FV solve (NEXT-2 workload)
    against central differences of the loss on a tiny grid, with direct
    solves; pins the chain rule through the harmonic-mean faces and the
    boundary terms (a dropped term or a wrong sign moves it by O(1))."""
    from oracle import adjoint_ref as ar
    m = 6
    th = PR.gaussian_field(m, 11)
    th_obs = PR.gaussian_field(m, 12)
    f = np.full(m * m, 1.0 / (m * m))
    u_obs = __import__("scipy.sparse.linalg", fromlist=["spsolve"]).spsolve(ar.operator(m, th_obs).tocsc(), f)
    L, g, _ = ar.loss_and_grad(m, th, f, u_obs)
    h = 1e-6
    fd = np.empty(m * m)
    for c in range(m * m):
        tp, tm = th.copy(), th.copy()
        tp[c] += h
        tm[c] -= h
        fd[c] = (ar.loss(m, tp, f, u_obs) - ar.loss(m, tm, f, u_obs)) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))
    assert L > 0


def test_adjoint_reference_operator_matches_generator():
    """The reference's face-by-face assembly equals the input generator's."""
    from oracle import adjoint_ref as ar
    m = 9
    th = PR.gaussian_field(m, 3)
    A, f = PR.varcoef_fv(m, th)
    B = ar.operator(m, th)
    assert np.max(np.abs((A.to_scipy() - B).toarray())) < 1e-13


def _classical_dense(A, theta):
    """Classical strength written out row by row (the measure of Ruge and
    Stueben the paper lists in Sec. 3.2), for the pins below."""
    A = A.tocsr()
    n = A.shape[0]
    thr = theta * (1.0 - 1e-10)
    rows, cols, vals = [], [], []
    for i in range(n):
        idx = A.indices[A.indptr[i]:A.indptr[i + 1]]
        dat = A.data[A.indptr[i]:A.indptr[i + 1]]
        m = max([-v for j, v in zip(idx, dat) if j != i] + [0.0])
        for j, v in zip(idx, dat):
            if j == i:
                rows.append(i), cols.append(i), vals.append(1.0)
            elif m > 0.0 and -v >= thr * m:
                rows.append(i), cols.append(j), vals.append(-v / m)
    return sp.csr_matrix((vals, (rows, cols)), shape=A.shape)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_classical_strength_bruteforce(oracle, seed):
    # mixed-sign off-diagonals, rows whose off-diagonals are all positive
    # (no strong entry), exact ties at theta
    rng = np.random.default_rng(seed)
    n = 40
    M = sp.random(n, n, density=0.15, random_state=seed, data_rvs=lambda k: rng.choice([-2.0, -1.0, -0.5, 0.5, 1.0], k))
    M = M.tolil()
    for i in range(0, n, 7):  # positive off-diagonals only
        for j in M.rows[i]:
            if j != i:
                M[i, j] = abs(M[i, j])
    M = M.tocsr() + sp.identity(n) * 5.0
    M.sort_indices()
    for theta in (0.25, 0.5):
        S = oracle.strength_classical(M, theta)
        R = _classical_dense(M, theta)
        R.sort_indices()
        assert np.array_equal(S.indptr, R.indptr) and np.array_equal(S.indices, R.indices)
        assert np.array_equal(S.data, R.data)


def test_classical_strength_special_cases(oracle):
    # 5-point Laplacian: every off-diagonal is the row's largest negative one
    A = PR.poisson5(10).to_scipy()
    S = oracle.strength_classical(A, 0.25)
    assert np.array_equal(S.indptr, A.indptr) and np.array_equal(S.indices, A.indices)
    assert np.all(S.data == 1.0)
    # grid-aligned Q1 anisotropy, eps = 1e-3: the x-neighbours (-2/3 + eps/3) and
    # the corners (-(1 + eps)/6 >= theta (2/3 - eps/3)) are strong; the
    # y-neighbours (1/3 - 2 eps/3 > 0) are positive and never strong
    ne = 9
    m = ne - 1
    A = PR.q1_aniso(ne, 1e-3, 0.0).to_scipy()
    S = oracle.strength_classical(A, 0.25)
    for i in range(A.shape[0]):
        cols = set(S.indices[S.indptr[i]:S.indptr[i + 1]].tolist())
        nb = set(A.indices[A.indptr[i]:A.indptr[i + 1]].tolist())
        vertical = {j for j in nb if j % m == i % m and j != i}
        assert cols == nb - vertical


def test_classical_strength_drives_setup(oracle):
    pr = PR.aniso_problem(48)
    params = dict(pr.params)
    params["soc_kind"] = 1
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, keep_aux=1, **params)
    S0 = oracle.strength_classical(pr.A.to_scipy(), params.get("soc_theta", 0.25))
    assert (h.levels[0].S != S0).nnz == 0
    assert len(h.levels) >= 3


def _cycle_dense(levels, gamma, omega, b, nu=(1, 1)):
    """The cycle x = B_0 b (zero initial guess) by its recursive definition,
    with dense matrices (Sec. 2: smoothing, coarse-grid correction, smoothing;
    gamma corrections per level, one when the next level is the coarsest)."""
    def cyc(l, rhs):
        A = levels[l].A.toarray()
        if l == len(levels) - 1:
            return np.linalg.solve(A, rhs)
        d = np.diag(A)
        P, R = levels[l].P.toarray(), levels[l].R.toarray()
        x = np.zeros_like(rhs)
        for _ in range(nu[0]):
            x = x + omega * ((rhs - A @ x) / d)
        for _ in range(1 if l + 1 == len(levels) - 1 else gamma):
            x = x + P @ cyc(l + 1, R @ (rhs - A @ x))
        for _ in range(nu[1]):
            x = x + omega * ((rhs - A @ x) / d)
        return x
    return cyc(0, b)


@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_matches_dense_recursion(oracle, gamma):
    pr = PR.poisson_problem(32)
    params = dict(pr.params)
    params["gamma"] = gamma
    params["max_coarse"] = 30
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **params)
    assert len(h.levels) >= 4
    b = np.random.default_rng(3).standard_normal(pr.A.n_rows)
    got = h.vcycle(b, np.zeros_like(b))
    ref = _cycle_dense(h.levels, gamma, params.get("omega", 2.0 / 3.0), b)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_w_cycle_differs_from_v_and_converges_faster(oracle):
    pr = PR.poisson_problem(32)
    out = {}
    for gamma in (1, 2):
        params = dict(pr.params, gamma=gamma, max_coarse=30)
        h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **params)
        x, info = h.solve(pr.b, tol=1e-8, outer=0)
        out[gamma] = info["iters"]
    assert out[2] <= out[1]
    params = dict(pr.params, max_coarse=200)  # two levels: W and V coincide
    hv = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **dict(params, gamma=1))
    hw = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **dict(params, gamma=2))
    b = np.random.default_rng(4).standard_normal(pr.A.n_rows)
    assert np.array_equal(hv.vcycle(b, np.zeros_like(b)), hw.vcycle(b, np.zeros_like(b)))


# --------------------------------------------------------------------------- k > 1 candidates (NEXT-3)
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_row_svd_matches_numpy(oracle, k):
    """The row SVD against LAPACK's: U U^T is the projector onto the kept range
    (unique), V Sigma^+ U^T is numpy's pseudo-inverse with singular values at
    most 1e-6 of the largest dropped, and the rank matches; rows of every rank,
    badly scaled, and nearly dependent columns (condition 1e4 and 1e8, the
    latter past the cutoff)."""
    rng = np.random.default_rng(k)
    cases = []
    for rank in range(0, k + 1):
        for length in (k, k + 3, 17):
            M = rng.standard_normal((length, rank)) @ rng.standard_normal((rank, k))
            cases.append(M * 10.0 ** rng.uniform(-3, 3))
    if k > 1:
        for cond in (1e4, 1e8):
            Q1, _ = np.linalg.qr(rng.standard_normal((9, k)))
            Q2, _ = np.linalg.qr(rng.standard_normal((k, k)))
            cases.append(Q1 @ np.diag(np.logspace(0, -np.log10(cond), k)) @ Q2)
    for M in cases:
        U, VS, rank = oracle.row_svd(M)
        sv = np.linalg.svd(M, compute_uv=False)
        keep = int(np.sum(sv > 1e-6 * sv[0])) if sv.size and sv[0] > 0 else 0
        assert rank == keep
        ref = np.linalg.pinv(M, rcond=1e-6)  # k x |J|
        got = VS @ U.T
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-10 * max(1.0, np.abs(ref).max()))
        Uc, _, _ = np.linalg.svd(M, full_matrices=False)
        Pref = Uc[:, :keep] @ Uc[:, :keep].T
        assert np.allclose(U @ U.T, Pref, atol=1e-12)


def _grid_candidates(n):
    """1, x, y on the lexicographic (m x m) interior grid of n = m^2 nodes."""
    m = int(round(math.sqrt(n)))
    i = np.arange(n)
    h = 1.0 / (m + 1)
    return np.column_stack([np.ones(n), (i % m + 1) * h, (i // m + 1) * h])


@pytest.mark.parametrize("k", [2, 3])
def test_tentative_k_is_min_norm_fit(oracle, k):
    """eq. Tproj: each free row of T is the injected row plus the minimal-norm
    update that fits all k candidates (numpy least squares on the row)."""
    A = PR.q1_aniso(17, 1e-2, math.pi / 8).to_scipy()
    n = A.shape[0]
    B = _grid_candidates(n)[:, :k].copy()
    lev = _setup_level(oracle, A, 2)
    T1, _ = oracle.tentative(lev["N"], lev["agg"], lev["roots"], B[:, 0])
    T, Bc = oracle.tentative_k(lev["N"], lev["agg"], lev["roots"], lev["rt"], B)
    assert np.array_equal(Bc, B[lev["roots"]])
    for i in range(n):
        s, e = T.indptr[i], T.indptr[i + 1]
        J = T.indices[s:e]
        if lev["rt"][i] != 0:
            assert np.array_equal(T.data[s:e], T1.data[s:e])  # roots (identity) and empty rows untouched
            continue
        t0 = T1.data[s:e]
        M = Bc[J].T  # k x |J|
        u = np.linalg.lstsq(M, B[i] - M @ t0, rcond=1e-6)[0]  # singular values of Bc_J below 1e-6 dropped
        assert np.allclose(T.data[s:e], t0 + u, rtol=1e-9, atol=1e-12)


def test_cg_k_converged_equals_dense_kkt(oracle):
    """k = 2: converged CG energy minimisation equals the dense KKT solution of
    min trace(P^T A P) over the free entries subject to P_i Bc_J = B_i (two
    equations per free row)."""
    A = PR.poisson5(7).to_scipy()
    n = A.shape[0]
    B = _grid_candidates(n)[:, :2].copy()
    lev = _setup_level(oracle, A, 2)
    T, Bc = oracle.tentative_k(lev["N"], lev["agg"], lev["roots"], lev["rt"], B)
    Ad = A.toarray()
    N = lev["N"]
    I, J = [], []
    for i in range(n):
        if lev["rt"][i] == 0:
            for j in N.indices[N.indptr[i]:N.indptr[i + 1]]:
                I.append(i), J.append(j)
    I, J = np.array(I), np.array(J)
    m = len(I)
    H = Ad[np.ix_(I, I)] * (J[:, None] == J[None, :])
    rows = sorted(set(I.tolist()))
    rix = {r: q for q, r in enumerate(rows)}
    Cm = np.zeros((2 * len(rows), m))
    for t in range(m):
        Cm[2 * rix[I[t]], t] = Bc[J[t], 0]
        Cm[2 * rix[I[t]] + 1, t] = Bc[J[t], 1]
    X0 = T.toarray().copy()
    xT = X0[I, J].copy()
    X0[I, J] = 0.0
    hvec = (Ad @ X0)[I, J]
    # CG moves inside {x : Cm (x - x_T) = 0}; rows whose pattern cannot carry both
    # candidates (one entry, or collinear Bc rows) make Cm rank-deficient, so the
    # constraints are taken on an orthonormal basis Q of Cm's row space
    U, sv, Vt = np.linalg.svd(Cm, full_matrices=False)
    Q = Vt[sv > 1e-10 * sv[0]]
    K = np.block([[2 * H, Q.T], [Q, np.zeros((Q.shape[0], Q.shape[0]))]])
    x = np.linalg.solve(K, np.concatenate([-2 * hvec, Q @ xT]))[:m]
    P, trace = oracle.energy_min_cg_k(A, T, lev["rt"], Bc, 800)
    assert np.allclose(P.toarray()[I, J], x, atol=1e-9)
    assert np.allclose(Cm @ P.toarray()[I, J], Cm @ xT, atol=1e-12)  # constraints as T left them
    assert np.all(np.diff(trace) <= 1e-12 * abs(trace[0]))


def _fits_all(BcJ):
    """Whether a row's pattern carries every candidate: the singular values of
    Bc_J all above the fit's cutoff (1e-6 of the largest), with a margin so
    that no decision sits on the cutoff."""
    sv = np.linalg.svd(BcJ, compute_uv=False)
    return sv.size == BcJ.shape[1] and sv[-1] > 2e-6 * sv[0]


def test_hierarchy_with_three_candidates(oracle):
    """Whole setup with B = [1, x, y]: on every level P Bc = B (the level's
    smoothed candidates) on free rows whose pattern carries the three
    candidates (Gram matrix above the cutoff), root rows are identity rows, Bc is B at the roots, and the
    cycle converges."""
    pr = PR.aniso_problem(48)
    n = pr.A.n_rows
    B = _grid_candidates(n)
    params = dict(pr.params, ncand=3)
    h = oracle.Hierarchy(pr.A.to_scipy(), B, **params)
    assert len(h.levels) >= 3
    for l, L in enumerate(h.levels[:-1]):
        P = L.P
        assert L.B.shape == (L.A.shape[0], 3) and L.Bc.shape == (P.shape[1], 3)
        assert np.array_equal(L.Bc, L.B[L.roots])
        PB = P @ L.Bc
        for i in range(P.shape[0]):
            s, e = P.indptr[i], P.indptr[i + 1]
            if L.rowtype[i] == 1:
                assert e - s == 1 and P.data[s] == 1.0
            elif L.rowtype[i] == 0 and _fits_all(L.Bc[P.indices[s:e]]):
                assert np.allclose(PB[i], L.B[i], rtol=1e-10, atol=1e-12 * np.abs(L.B).max())
    x, info = h.solve(pr.b, tol=1e-8, outer=1)
    assert info["status"] == 0


# --------------------------------------------------------------------------- block systems (NEXT-3)
def test_elasticity_element_is_symmetric_and_kills_rigid_modes():
    """The Q1 plane-strain element stiffness is symmetric, positive
    semi-definite with exactly the three rigid-body modes as its null space."""
    Ke = PR.q1_elasticity_element(1.0, 0.3, 0.5, 0.25)
    xy = np.array([[0.0, 0.0], [0.5, 0.0], [0.5, 0.25], [0.0, 0.25]])
    Rb = PR.rigid_body_modes(xy)
    assert np.abs(Ke - Ke.T).max() < 1e-15
    assert np.abs(Ke @ Rb).max() < 1e-14
    ev = np.linalg.eigvalsh(Ke)
    assert np.all(ev[:3] < 1e-12) and ev[3] > 1e-3


def test_elasticity_operator_spd_and_rigid_modes_away_from_clamp():
    pr = PR.elasticity_problem(4)
    A = pr.A.to_scipy().toarray()
    assert np.abs(A - A.T).max() < 1e-14 and np.linalg.eigvalsh(A)[0] > 0
    # rows of nodes not next to the clamped side annihilate the rigid-body modes
    R = A @ pr.B
    nodes = np.arange(A.shape[0] // 2)
    ny = 4
    x = (nodes % (8 * ny)) * (8.0 / (8 * ny))
    far = np.repeat(x < 8.0 - 1.5 * (8.0 / (8 * ny)), 2)
    assert np.abs(R[far]).max() < 1e-12


@pytest.mark.parametrize("m", [2, 3])
def test_amalgamate_is_block_maximum(oracle, m):
    rng = np.random.default_rng(m)
    nn = 30
    n = m * nn
    S = sp.random(n, n, density=0.08, random_state=m, data_rvs=lambda k: rng.random(k)).tocsr()
    S = (S + sp.identity(n)).tocsr()
    S.sort_indices()
    Sm = oracle.amalgamate(S, m)
    D = S.toarray()
    P = S.copy()
    P.data[:] = 1.0
    Pd = P.toarray()
    for I in range(nn):
        for J in range(nn):
            blk = D[I * m:(I + 1) * m, J * m:(J + 1) * m]
            has = Pd[I * m:(I + 1) * m, J * m:(J + 1) * m].any()
            got = Sm[I, J]
            if has:
                assert got == blk[Pd[I * m:(I + 1) * m, J * m:(J + 1) * m] > 0].max()
            else:
                assert got == 0.0 and not (Sm.indices[Sm.indptr[I]:Sm.indptr[I + 1]] == J).any()


def test_unamalgamated_pattern_is_kronecker_of_node_pattern(oracle):
    """Block systems (Sec. 3.4): on every level of the plane-strain workload
    (two unknowns per node, no pre-filter) the unknown-level pattern N is the
    node pattern S_m^d C_m expanded by the Kronecker product with an m x m
    block of ones (scipy.sparse.kron of a scipy product chain: another route
    than the oracle's loops), each entry carrying its node entry's value; a
    root unknown's row is the identity row of its own unknown in its
    aggregate's block."""
    pr = PR.elasticity_problem(8)
    m, d = pr.params["block_size"], pr.params["degree"]
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    checked = 0
    for L in h.levels[:-1]:
        n = L.A.shape[0]
        nn = n // m
        Sm = oracle.amalgamate(L.S, m)
        aggn = L.agg[::m]
        ncn = L.N.shape[1] // m
        rows = np.nonzero(aggn >= 0)[0]
        Nm = sp.csr_matrix((np.ones(len(rows)), (rows, aggn[rows])), shape=(nn, ncn))
        for _ in range(d):
            Nm = (Sm @ Nm).tocsr()
        K = sp.kron(Nm, sp.csr_matrix(np.ones((m, m)))).tocsr()
        K.sort_indices()
        N = L.N
        for i in range(n):
            cols = N.indices[N.indptr[i]:N.indptr[i + 1]]
            vals = N.data[N.indptr[i]:N.indptr[i + 1]]
            if L.rowtype[i] == 1:
                assert list(cols) == [m * L.agg[i] + i % m]
                continue
            kc = K.indices[K.indptr[i]:K.indptr[i + 1]]
            kv = K.data[K.indptr[i]:K.indptr[i + 1]]
            assert np.array_equal(cols, kc), i
            assert np.allclose(vals, kv, rtol=1e-13, atol=0.0), i
            checked += 1
    assert checked > 1000


def test_elasticity_hierarchy_blocks_and_constraints(oracle):
    """2 x 2 blocks and the three rigid-body modes: aggregates and roots come
    in node pairs, root rows are identity rows over their aggregate's block,
    T and P reproduce every candidate where the pattern carries them, and
    CG with the cycle reaches 1e-8."""
    pr = PR.elasticity_problem(8)
    h = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    assert len(h.levels) >= 3
    for L in h.levels[:-1]:
        n = L.A.shape[0]
        assert np.array_equal(L.agg[0::2], L.agg[1::2])
        r = L.roots.reshape(-1, 2)
        assert np.all(r[:, 0] % 2 == 0) and np.array_equal(r[:, 1], r[:, 0] + 1)
        for T in (L.T, L.P):
            for i in range(n):
                s, e = T.indptr[i], T.indptr[i + 1]
                if L.rowtype[i] == 1:
                    assert e - s == 1 and T.indices[s] == 2 * L.agg[i] + i % 2 and T.data[s] == 1.0
                elif L.rowtype[i] == 0 and _fits_all(L.Bc[T.indices[s:e]]):
                    assert np.allclose(T[i] @ L.Bc, L.B[i], rtol=1e-9, atol=1e-12 * np.abs(L.B).max())
    x, info = h.solve(pr.b, tol=1e-8, maxit=300, outer=1)
    assert info["status"] == 0
    assert np.linalg.norm(pr.b - pr.A.to_scipy() @ x) < 1e-8 * np.linalg.norm(pr.b)
