"""NEXT-3 for scalar problems: k > 1 candidate vectors (Sec. 3.6, eq. Tproj),
GPU hierarchy and solve against the oracle."""
import math

import numpy as np
import pytest

from paper_1610_03154_gb300 import problems as PR
from tests.test_gpu_parity import (CASES, as_csr, close_strength, dev, gpu_solve, rn,  # noqa: F401
                                   same_pattern, torch_dev)  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu
# Row fits go through the singular value decomposition of each row's Bc_J
# (condition kappa_i), so a fit carries rounding multiplied by kappa_i (a fit
# through the Gram matrix would multiply it by kappa_i^2); singular values at
# most 1e-6 of the largest are dropped, so kappa_i <= 1e6 on what is kept.
# Level 0 (exact inputs): T within 1e-12 on rows with kappa_i <= 1e4
# (measured <= 2.3e-14), P, R and the coarse operator within TOL0 (measured
# <= 1.9e-12); symmetric setups keep TOL0 on every level.
TOL0 = 1e-11
TOL_ROW = 1e-12
# The nonsymmetric setup (GMRES minimisations for P and for R^T from A^T,
# whose least-squares steps add to the fits' conditioning): level 0 measured
# <= 1.8e-11 (80^2 convection-diffusion, d = 3, three candidates, R up to
# 4.5e3), coarse levels, whose inputs already differ, <= 3.2e-8 (level 2,
# d = 1, two candidates); well-conditioned level-0 rows of T <= 4e-15.
TOL_NONSYM0 = 1e-10
TOL_NONSYM = 1e-7
TOL = TOL0
# Block systems (m x m root blocks, rigid-body modes; 1k-4k unknowns):
# measured <= 7e-15 on every level
TOL_BLOCK = 1e-12


def grid_candidates(n, k):
    """1, x, y on the lexicographic (m x m) interior grid of n = m^2 nodes."""
    m = int(round(math.sqrt(n)))
    i = np.arange(n)
    h = 1.0 / (m + 1)
    return np.column_stack([np.ones(n), (i % m + 1) * h, (i // m + 1) * h])[:, :k].copy()


def close(g, o, what, tol=None):
    tol = TOL if tol is None else tol
    d = np.max(np.abs(g - o)) if g.size else 0.0
    assert d <= tol * max(np.max(np.abs(o)) if o.size else 0.0, 1e-300), (what, d)


def level0_rows(h, L, k):
    """T on level 0 by row class of kappa(Bc_J): rows with kappa <= 1e4 within
    TOL_ROW of the oracle; returns the counts of free rows with kappa <= 1e4,
    1e4 < kappa <= 1e6, and with a direction past the cutoff (rank < k)."""
    T = as_csr(h.export_csr(0, 3))
    scale = np.max(np.abs(L.T.data))
    counts = {"well": 0, "fair": 0, "cut": 0}
    for i in np.nonzero(L.rowtype == 0)[0]:
        s, e = L.T.indptr[i], L.T.indptr[i + 1]
        sv = np.linalg.svd(L.Bc[L.T.indices[s:e]], compute_uv=False)
        if sv.size < k or sv[-1] <= 1e-6 * sv[0]:
            counts["cut"] += 1
            continue
        if sv[0] <= 1e4 * sv[-1]:
            counts["well"] += 1
            d = np.max(np.abs(T.data[s:e] - L.T.data[s:e]))
            assert d <= TOL_ROW * scale, ("T[0] row", i, d)
        else:
            counts["fair"] += 1
    return counts


def compare_levels(h, oh, theta, tol, tol0=TOL0):
    """Level by level: S, aggregates, roots, N and the patterns of T, P, R and
    the coarse A bit-exact; level-0 smoothed candidates bit-exact; values and
    every level's B, Bc within tol; P Bc = B on free rows whose pattern can
    carry all k candidates.  With a post-filter (drop threshold theta) a
    decision may flip only on an entry within 1e-6 of its threshold, and the
    comparison stops at that level."""
    st = h.stats()
    assert st["levels"] == len(oh.levels)
    for l, L in enumerate(oh.levels[:-1]):
        tol_l = tol0 if l == 0 else tol
        Bg = h.export_vec(l, 3)
        assert Bg.shape == L.B.shape
        if l == 0:
            assert np.array_equal(Bg, L.B)
        else:
            close(Bg, L.B, f"B[{l}]", tol_l)
        close(h.export_vec(l, 4), L.Bc, f"Bc[{l}]", tol_l)
        assert np.array_equal(h.export_vec(l, 0), L.agg)
        assert np.array_equal(h.export_vec(l, 1), L.roots)
        for which, name, ref in ((1, "S", L.S), (2, "N", L.N), (3, "T", L.T)):
            g = as_csr(h.export_csr(l, which))
            same_pattern(g, ref, f"{name}[{l}]")
            if which == 1 and l > 0:  # a quotient of the coarse operator's entries: its bar, row-scaled
                close_strength(g, ref, L.A, f"S[{l}]", tol)
            else:
                close(g.data, ref.data, f"{name}[{l}]", tol_l)
        Pg = as_csr(h.export_csr(l, 4))
        if not (np.array_equal(Pg.indptr, L.P.indptr) and np.array_equal(Pg.indices, L.P.indices)):
            # values agree to TOL, so a post-filter decision may flip on an entry
            # within TOL of the drop threshold; every difference must be one, and
            # the levels below then differ legitimately
            assert theta > 0.0, f"P[{l}] pattern differs without a post-filter"
            flips = 0
            for i in range(Pg.shape[0]):
                a = set(Pg.indices[Pg.indptr[i]:Pg.indptr[i + 1]].tolist())
                b = set(L.P.indices[L.P.indptr[i]:L.P.indptr[i + 1]].tolist())
                for j, M in [(j, Pg) for j in a - b] + [(j, L.P) for j in b - a]:
                    row = M[i].toarray().ravel()
                    thr = theta * np.abs(row).max()
                    assert abs(abs(row[j]) - thr) <= 1e-6 * thr, (l, i, j, row[j], thr)
                    flips += 1
            assert flips > 0
            break
        close(Pg.data, L.P.data, f"P[{l}]", tol_l)
        Rg = as_csr(h.export_csr(l, 5))
        same_pattern(Rg, L.R, f"R[{l}]")
        close(Rg.data, L.R.data, f"R[{l}]", tol_l)
        Ac = as_csr(h.export_csr(l + 1, 0))
        same_pattern(Ac, oh.levels[l + 1].A, f"A[{l + 1}]")
        close(Ac.data, oh.levels[l + 1].A.data, f"A[{l + 1}]", tol_l)
        P = as_csr(h.export_csr(l, 4))
        Bc = h.export_vec(l, 4)
        rt = h.export_vec(l, 2)
        PB = P @ Bc
        for i in np.nonzero(rt == 0)[0][:2000]:
            cols = P.indices[P.indptr[i]:P.indptr[i + 1]]
            sv = np.linalg.svd(Bc[cols], compute_uv=False)
            if sv.size == Bc.shape[1] and sv[-1] > 2e-6 * sv[0]:  # the pattern carries all k candidates
                assert np.allclose(PB[i], Bg[i], rtol=1e-10, atol=1e-12 * np.abs(Bg).max())


def hier(rn, torch_dev, pr, B, Bhat=None, **over):
    torch, d = torch_dev
    A = pr.A
    params = rn.params_from_config(pr.params, keep_aux=1, **over)
    return rn.Hierarchy(dev(torch_dev, A.rowptr), dev(torch_dev, A.col), dev(torch_dev, A.val),
                        dev(torch_dev, B), None if Bhat is None else dev(torch_dev, Bhat), params=params)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("case", ["poisson64", "aniso96", "convdiff80", "convdiff80rn1"])
def test_k_candidates_hierarchy_parity(rn, torch_dev, oracle, case, k):
    """Patterns (S, aggregates, roots, N, P, R, coarse A) bit-exact; level-0
    smoothed candidates bit-exact; level-0 T within 1e-12 on rows whose Bc_J
    has condition <= 1e4 (the rows past the cutoff counted); T, P, R, coarse A
    and every level's B, Bc within TOL0 on level 0 and within TOL (symmetric)
    or TOL_NONSYM below; P Bc = B on free rows that can carry the k
    candidates.  A post-filter decision may flip only on an entry within the
    bar of its threshold; the comparison stops at that level."""
    pr = CASES[case]()
    tol = TOL if pr.Bhat is None else TOL_NONSYM
    n = pr.A.n_rows
    B = grid_candidates(n, k)
    Bhat = None if pr.Bhat is None else B.copy()
    h = hier(rn, torch_dev, pr, B, Bhat)
    oh = oracle.Hierarchy(pr.A.to_scipy(), B, Bhat=Bhat, **dict(pr.params, ncand=k))
    counts = level0_rows(h, oh.levels[0], k)
    assert counts["well"] > 0
    print(f"{case} k={k}: level-0 free rows by kappa(Bc_J): {counts}")
    compare_levels(h, oh, pr.params.get("postfilter", 0.0), tol, TOL0 if pr.Bhat is None else TOL_NONSYM0)
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_k_candidates_solve(rn, torch_dev, oracle, precision):
    """CG preconditioned by the cycle of a 3-candidate hierarchy reaches 1e-8
    (true FP64 residual) within 2 iterations of the oracle's count."""
    pr = CASES["aniso255"]()
    B = grid_candidates(pr.A.n_rows, 3)
    oh = oracle.Hierarchy(pr.A.to_scipy(), B, **dict(pr.params, ncand=3))
    _, oinfo = oh.solve(pr.b, tol=1e-8, maxit=500, outer=1)
    h = hier(rn, torch_dev, pr, B, precision=precision)
    x, info, res = gpu_solve(rn, torch_dev, h, pr, maxit=500)
    assert res < 1e-8
    assert abs(info["iters"] - oinfo["iters"]) <= 2
    h.close()


def test_one_candidate_as_n_by_1_matches_vector(rn, torch_dev):
    """B given as n x 1 is the single-candidate setup, bit for bit."""
    torch, d = torch_dev
    pr = CASES["aniso96"]()
    out = []
    for B in (pr.B.reshape(-1), pr.B.reshape(-1, 1)):
        h = hier(rn, torch_dev, pr, np.ascontiguousarray(B))
        out.append(as_csr(h.export_csr(0, 4)))
        h.close()
    assert (out[0] != out[1]).nnz == 0


# ---------------------------------------------------------------- block systems
@pytest.mark.parametrize("postfilter", [0.0, 0.05])
@pytest.mark.parametrize("ny", [8, 16])
def test_block_system_hierarchy_parity(rn, torch_dev, oracle, ny, postfilter):
    """2D plane-strain elasticity, 2 unknowns per node, 3 rigid-body modes
    (Sec. 3.2 amalgamation, Sec. 3.6 block root-node form): node aggregates
    unamalgamated to unknowns, patterns bit-exact and values within TOL of
    the oracle on every level, with and without the post-filter (whose
    own-aggregate block of m columns is always kept)."""
    pr = PR.elasticity_problem(ny)
    h = hier(rn, torch_dev, pr, pr.B, postfilter=postfilter)
    oh = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **dict(pr.params, postfilter=postfilter))
    assert len(oh.levels) >= 3
    for L in oh.levels[:-1]:  # unknowns stay node-major: coarse unknowns 2 r, 2 r + 1 per root node
        assert L.roots.size % 2 == 0
        assert np.array_equal(L.roots[1::2], L.roots[0::2] + 1) and np.all(L.roots[0::2] % 2 == 0)
    compare_levels(h, oh, postfilter, TOL_BLOCK, TOL_BLOCK)
    h.close()


def test_block_system_two_candidates(rn, torch_dev, oracle):
    """k = m = 2 (the translations only): T is the block-normalised injection
    alone, with no row fit for further candidates."""
    pr = PR.elasticity_problem(8)
    B = np.ascontiguousarray(pr.B[:, :2])
    h = hier(rn, torch_dev, pr, B)
    oh = oracle.Hierarchy(pr.A.to_scipy(), B, **dict(pr.params, ncand=2))
    compare_levels(h, oh, 0.0, TOL_BLOCK, TOL_BLOCK)
    h.close()


def test_system_without_amalgamation_is_refused(rn, torch_dev, oracle):
    """Aggregating the system unknown by unknown (block_size 1) lets
    aggregates of one displacement component carry rigid-body modes that
    vanish on it: P grows to ~1e16 and the coarsest matrix is numerically
    singular; both sides refuse the setup with the same status."""
    pr = PR.elasticity_problem(8)
    with pytest.raises(rn.RNError) as e:
        hier(rn, torch_dev, pr, pr.B, block_size=1)
    assert e.value.status == rn.RN_ESINGULAR
    with pytest.raises(RuntimeError, match=f"status {rn.RN_ESINGULAR}"):
        oracle.Hierarchy(pr.A.to_scipy(), pr.B, **dict(pr.params, block_size=1))


@pytest.mark.parametrize("precision", [0, 1])
def test_block_system_solve(rn, torch_dev, oracle, precision):
    """CG preconditioned by the block hierarchy's V(1,1) cycle reaches 1e-8
    (true FP64 residual) within 2 iterations of the oracle's count."""
    pr = PR.elasticity_problem(32)
    oh = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    _, oinfo = oh.solve(pr.b, tol=1e-8, maxit=1000, outer=1)
    h = hier(rn, torch_dev, pr, pr.B, precision=precision)
    x, info, res = gpu_solve(rn, torch_dev, h, pr, maxit=1000)
    assert res < 1e-8
    assert abs(info["iters"] - oinfo["iters"]) <= 2
    h.close()
