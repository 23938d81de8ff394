"""GPU: independent problems set up together (rn_setup_merged).

Problem i's hierarchy from the merged pass must be the one rn_setup builds
for it alone: with FP64 sweeps the same level sizes, strength, aggregates,
roots and every pattern bit for bit, and values to 1e-12 of each matrix's
largest entry (the energy CG's sums run over per-problem chunks, a different
order from the single setup's block sums).  With FP32 sweeps the step
lengths carry FP32 rounding of that other order, so the comparison is on
the first level's values (1e-5) and on the solves.  Every hierarchy solves
like the problem's own; bad arguments are refused."""
import numpy as np
import pytest

from paper_1610_03154_gb300 import problems as PR

pytestmark = pytest.mark.gpu

CSR = {0: "A", 1: "S", 2: "N", 3: "T", 4: "P", 5: "R"}


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03154_gb300 import rn

    return torch, torch.device("cuda:0"), rn


def _diagonal_problem(n=100):
    """A diagonal operator above max_coarse: no strong coupling, so no
    aggregate, and its coarsening stalls on the first level (which becomes its
    coarsest, solved by the dense LU)."""
    import scipy.sparse as sp

    A = PR.CSR.from_scipy(sp.diags(np.linspace(1.0, 3.0, n)).tocsr())
    return PR.Problem("diagonal", A, np.ones((n, 1)), np.random.default_rng(12).uniform(-1.0, 1.0, n),
                      dict(PR.PARAMS_ANISO))


def _problems():
    """Uneven rotated-anisotropy problems of different depths, one that is its
    own coarsest level (7 x 7 interior nodes), one a level deeper, and one
    whose coarsening stalls on its first level (the merged level is redone
    without it)."""
    probs = PR.batch_aniso_problems(count=7, seed=11, side_lo=24, side_hi=180)
    probs.insert(1, PR.aniso_problem(8, seed=9))
    probs.insert(4, PR.aniso_problem(14, seed=10))
    probs.insert(6, _diagonal_problem())
    return probs


def _both(env, probs, precision, keep_aux=1):
    torch, dev, rn = env
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    params = rn.params_from_config(PR.PARAMS_ANISO, precision=precision, outer=rn.RN_OUTER_CG, keep_aux=keep_aux)
    data = [(t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.B.reshape(-1))) for p in probs]
    own = [rn.Hierarchy(*d, params=params) for d in data]
    mer = rn.setup_merged(data, params)
    return own, mer, t


def _close(h):
    for x in h:
        x.close()


def test_merged_setup_fp64_equals_individual_setups(env):
    probs = _problems()
    own, mer, _ = _both(env, probs, 0)
    depths = [h.stats()["levels"] for h in own]
    assert min(depths) == 1 and max(depths) >= 4 and len(set(depths)) >= 3
    for i, (a, b) in enumerate(zip(own, mer)):
        sa, sb = a.stats(), b.stats()
        for key in ("levels", "n", "nnz_A", "nnz_P", "nnz_R"):
            assert sa[key] == sb[key], (i, key, sa[key], sb[key])
        L = sa["levels"]
        for lvl in range(L):
            mats = (0,) if lvl == L - 1 else (0, 1, 2, 3, 4, 5)
            for which in mats:
                ra, ca, va, sha = a.export_csr(lvl, which)
                rb, cb, vb, shb = b.export_csr(lvl, which)
                assert sha == shb and np.array_equal(ra, rb) and np.array_equal(ca, cb), (i, lvl, CSR[which])
                if va.size:
                    err = np.max(np.abs(va - vb))
                    assert err <= 1e-12 * max(np.max(np.abs(va)), 1e-300), (i, lvl, CSR[which], err)
            vecs = (3,) if lvl == L - 1 else (0, 1, 2, 3, 4)
            for which in vecs:
                xa, xb = a.export_vec(lvl, which), b.export_vec(lvl, which)
                if which <= 2:
                    assert np.array_equal(xa, xb), (i, lvl, which)
                else:
                    assert np.max(np.abs(xa - xb)) <= 1e-12 * max(np.max(np.abs(xa)), 1e-300), (i, lvl, which)
    _close(own)
    _close(mer)


@pytest.mark.parametrize("precision", [0, 1])
def test_merged_setup_solves_like_individual_setups(env, precision):
    """Every merged-setup hierarchy reaches 1e-8 (true FP64 residual on the
    host) within 2 CG iterations of the problem's own hierarchy; with FP32
    sweeps the first level's P agrees to 1e-5 on the same pattern."""
    torch, dev, rn = env
    probs = _problems()
    own, mer, t = _both(env, probs, precision, keep_aux=0)
    for i, (p, a, b) in enumerate(zip(probs, own, mer)):
        assert a.stats()["n"] == b.stats()["n"], i
        if a.stats()["levels"] > 1:
            ra, ca, va, _ = a.export_csr(0, 4)
            rb, cb, vb, _ = b.export_csr(0, 4)
            assert np.array_equal(ra, rb) and np.array_equal(ca, cb), i
            tol = 1e-12 if precision == 0 else 1e-5
            assert np.max(np.abs(va - vb)) <= tol * np.max(np.abs(va)), i
        bb = t(p.b)
        xa, xb = torch.zeros_like(bb), torch.zeros_like(bb)
        ia = a.solve(bb, xa, rtol=1e-8, maxit=400)
        ib = b.solve(bb, xb, rtol=1e-8, maxit=400)
        assert abs(ia["iters"] - ib["iters"]) <= 2, (i, ia["iters"], ib["iters"])
        As = p.A.to_scipy()
        res = np.linalg.norm(p.b - As @ xb.cpu().numpy()) / np.linalg.norm(p.b)
        assert res < 1e-8, (i, res)
    _close(own)
    _close(mer)


def test_merged_setup_feeds_the_merged_solve(env):
    """Merged setup, then the merged block-diagonal solve: every problem
    within 2 iterations of its own solve on its own hierarchy."""
    torch, dev, rn = env
    probs = _problems()
    own, mer, t = _both(env, probs, 1, keep_aux=0)
    bs = [t(p.b) for p in probs]
    ref = []
    for h, b in zip(own, bs):
        x = torch.zeros_like(b)
        ref.append(h.solve(b, x, rtol=1e-8, maxit=400)["iters"])
    batch = rn.Batch(mer)
    xs = [torch.zeros_like(b) for b in bs]
    infos = batch.solve(bs, xs, rtol=1e-8, maxit=400)
    for i, (p, info, x) in enumerate(zip(probs, infos, xs)):
        assert abs(info["iters"] - ref[i]) <= 2, (i, info["iters"], ref[i])
        res = np.linalg.norm(p.b - p.A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(p.b)
        assert res < 1e-8, (i, res)
    batch.close()
    _close(own)
    _close(mer)


def test_merged_setup_of_one_problem_is_its_setup(env):
    """One problem through the merged path: the hierarchy rn_setup builds."""
    probs = [PR.aniso_problem(96, seed=13)]
    own, mer, _ = _both(env, probs, 0)
    a, b = own[0], mer[0]
    assert a.stats()["n"] == b.stats()["n"] and a.stats()["nnz_A"] == b.stats()["nnz_A"]
    for lvl in range(a.stats()["levels"] - 1):
        for which in (0, 4, 5):
            ra, ca, va, _ = a.export_csr(lvl, which)
            rb, cb, vb, _ = b.export_csr(lvl, which)
            assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
            assert np.max(np.abs(va - vb)) <= 1e-12 * np.max(np.abs(va))
    _close(own)
    _close(mer)


def test_merged_setup_refuses_bad_arguments(env):
    torch, dev, rn = env
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    probs = _problems()[:3]
    data = [(t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.B.reshape(-1))) for p in probs]
    for over in (dict(symmetric=0), dict(method=rn.RN_ENERGY_GMRES)):
        params = rn.params_from_config(PR.PARAMS_ANISO, **over)
        with pytest.raises(rn.RNError) as e:
            rn.setup_merged(data, params)
        assert e.value.status == rn.RN_EINVAL
    # a column past its own problem's size (inside the merged range) is refused, naming the problem
    col = probs[2].A.col.copy()
    col[5] = probs[2].A.n_rows
    bad = list(data)
    bad[2] = (data[2][0], t(col), data[2][2], data[2][3])
    with pytest.raises(rn.RNError) as e:
        rn.setup_merged(bad, rn.params_from_config(PR.PARAMS_ANISO))
    assert e.value.status == rn.RN_EINVAL
    assert "problem 2" in str(e.value)
