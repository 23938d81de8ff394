"""GPU: independent problems merged into one block-diagonal hierarchy
(rn_batch_merge / rn_batch_solve / rn_batch_cycle).  Each problem's cycle
is its own cycle (problems shallower than the merged hierarchy pass through
its lower levels exactly), and the per-problem CG converges like the
problem's own CG solve."""
import numpy as np
import pytest

from paper_1610_03154_gb300 import problems as PR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03154_gb300 import rn

    return torch, torch.device("cuda:0"), rn


def _problems():
    """Uneven rotated-anisotropy problems of different depths, and one that is
    its own coarsest level (7 x 7 interior nodes, below max_coarse = 64)."""
    probs = PR.batch_aniso_problems(count=6, seed=7, side_lo=24, side_hi=160)
    probs.insert(2, PR.aniso_problem(8, seed=9))
    return probs


def _setup(env, probs, precision):
    torch, dev, rn = env
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    params = rn.params_from_config(PR.PARAMS_ANISO, precision=precision, outer=rn.RN_OUTER_CG)
    hs = [rn.Hierarchy(t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.B.reshape(-1)), params=params) for p in probs]
    return hs, t


@pytest.mark.parametrize("precision", [0, 1])
def test_merged_cycle_is_each_problems_cycle(env, precision):
    """One cycle per problem through the merged hierarchy against the
    problem's own cycle: FP64 to 1e-12 (only SpMV row sums may group
    differently, the merged levels' lanes per row following the longest row
    of all problems), FP32 cycles to 1e-5."""
    torch, dev, rn = env
    probs = _problems()
    hs, t = _setup(env, probs, precision)
    depths = [h.stats()["levels"] for h in hs]
    assert min(depths) == 1 and max(depths) >= 4 and len(set(depths)) >= 3
    batch = rn.Batch(hs)
    rng = np.random.default_rng(3)
    bs = [t(rng.uniform(-1.0, 1.0, p.A.n_rows)) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch.cycle(bs, xs)
    tol = 1e-12 if precision == 0 else 1e-5
    for h, b, x in zip(hs, bs, xs):
        ref = torch.zeros_like(b)
        h.vcycle(b, ref)
        r, g = ref.cpu().numpy(), x.cpu().numpy()
        assert np.max(np.abs(g - r)) <= tol * np.max(np.abs(r))
    batch.close()
    for h in hs:
        h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_merged_solve_matches_individual_solves(env, precision):
    """Every problem reaches 1e-8 (true FP64 residual, checked on the host)
    within 2 iterations of its own CG solve; a zero right-hand side stops at
    once with x = 0; the hierarchies may be freed after merging."""
    torch, dev, rn = env
    probs = _problems()
    hs, t = _setup(env, probs, precision)
    bs = [t(p.b) for p in probs]
    bs[4] = torch.zeros_like(bs[4])
    own = []
    for h, b in zip(hs, bs):
        x = torch.zeros_like(b)
        own.append(h.solve(b, x, rtol=1e-8, maxit=1000)["iters"])
    batch = rn.Batch(hs)
    for h in hs:
        h.close()
    xs = [torch.zeros_like(b) for b in bs]
    infos = batch.solve(bs, xs, rtol=1e-8, maxit=1000)
    for k, (p, b, x, info) in enumerate(zip(probs, bs, xs, infos)):
        assert info["status"] == 0
        bh, xh = b.cpu().numpy(), x.cpu().numpy()
        if k == 4:
            assert info["iters"] == 0 and not np.any(xh)
            continue
        res = np.linalg.norm(bh - p.A.to_scipy() @ xh) / np.linalg.norm(bh)
        assert res < 1e-8
        assert abs(info["rel_res"] - res) <= 1e-3 * res + 1e-15
        assert abs(info["iters"] - own[k]) <= 2, (k, info["iters"], own[k])
    # a second solve from the solutions: converged at once
    infos2 = batch.solve(bs, xs, rtol=1e-8, maxit=1000)
    assert all(i["iters"] == 0 for i in infos2)
    batch.close()


def test_merged_solve_iteration_limit(env):
    """maxit reached: RN_ENOTCONV for the batch, per-problem statuses, and
    no problem iterates past the limit."""
    torch, dev, rn = env
    probs = _problems()[:4]
    hs, t = _setup(env, probs, 0)
    batch = rn.Batch(hs)
    bs = [t(p.b) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    with pytest.raises(rn.RNError) as e:
        batch.solve(bs, xs, rtol=1e-8, maxit=3)
    assert e.value.status == rn.RN_ENOTCONV
    xs = [torch.zeros_like(b) for b in bs]
    infos = batch.solve(bs, xs, rtol=1e-8, maxit=3, raise_on_notconv=False)
    for p, info in zip(probs, infos):
        assert info["iters"] <= 3
        assert info["status"] in (0, rn.RN_ENOTCONV)
        if p.A.n_rows > 64:
            assert info["status"] == rn.RN_ENOTCONV
    batch.close()
    for h in hs:
        h.close()


def test_merged_solve_against_the_oracle(env, oracle):
    """Uneven problems merged (FP64 cycle): each reaches 1e-8 within 2
    iterations of the oracle's CG on the same hierarchy recipe."""
    torch, dev, rn = env
    probs = PR.batch_aniso_problems(count=4, seed=11, side_lo=16, side_hi=64)
    probs.append(PR.aniso_problem(8, seed=9))
    hs, t = _setup(env, probs, 0)
    batch = rn.Batch(hs)
    for h in hs:
        h.close()
    bs = [t(p.b) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = batch.solve(bs, xs, rtol=1e-8, maxit=1000)
    batch.close()
    for p, info, x in zip(probs, infos, xs):
        oh = oracle.Hierarchy(p.A.to_scipy(), p.B, **dict(PR.PARAMS_ANISO, outer=1))
        _, oinfo = oh.solve(p.b, tol=1e-8, maxit=1000, outer=1)
        assert info["status"] == 0
        assert abs(info["iters"] - oinfo["iters"]) <= 2, (p.name, info["iters"], oinfo["iters"])
        xh = x.cpu().numpy()
        assert np.linalg.norm(p.b - p.A.to_scipy() @ xh) / np.linalg.norm(p.b) < 1e-8


def test_merged_block_systems(env):
    """Block-system hierarchies (plane-strain elasticity, 2 unknowns per
    node, 3 rigid-body modes) of three sizes merged: each solve within 2
    iterations of the problem's own CG, true residual below 1e-8."""
    torch, dev, rn = env
    probs = [PR.elasticity_problem(ny) for ny in (4, 8, 16)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    params = rn.params_from_config(PR.PARAMS_ELASTICITY, outer=rn.RN_OUTER_CG)
    hs = [rn.Hierarchy(t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.B), params=params) for p in probs]
    bs = [t(p.b) for p in probs]
    own = []
    for h, b in zip(hs, bs):
        x = torch.zeros_like(b)
        own.append(h.solve(b, x, rtol=1e-8, maxit=1000)["iters"])
    batch = rn.Batch(hs)
    xs = [torch.zeros_like(b) for b in bs]
    infos = batch.solve(bs, xs, rtol=1e-8, maxit=1000)
    for p, info, x, n_own in zip(probs, infos, xs, own):
        assert info["status"] == 0
        assert abs(info["iters"] - n_own) <= 2
        xh = x.cpu().numpy()
        assert np.linalg.norm(p.b - p.A.to_scipy() @ xh) / np.linalg.norm(p.b) < 1e-8
    batch.close()
    for h in hs:
        h.close()
