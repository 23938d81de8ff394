"""GPU: many right-hand sides at once (rn_solve_multi) on the 4096-dof
Poisson operator: every column reaches the tolerance, and the iteration
count is the largest of the single-vector stationary solves'."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1610_03154_gb300 import problems as PR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03154_gb300 import rn

    return torch, torch.device("cuda:0"), rn


def _hier(env, pr, **over):
    torch, dev, rn = env
    A = pr.A
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    params = rn.params_from_config(pr.params, **over)
    return rn.Hierarchy(t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)), params=params)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("s", [256, 37, 300])
def test_solve_multi_columns_converge_like_single_solves(env, precision, s):
    torch, dev, rn = env
    pr = PR.poisson_problem(64)
    A = pr.A.to_scipy()
    n = A.shape[0]
    B = np.random.default_rng(4).uniform(-1.0, 1.0, (n, s))
    B[:, 3] = 0.0  # a zero right-hand side stays zero
    h = _hier(env, pr, precision=precision, outer=rn.RN_OUTER_STATIONARY)
    Bd = torch.from_numpy(B.copy()).to(dev)
    Xd = torch.zeros_like(Bd)
    info = h.solve_multi(Bd, Xd, rtol=1e-8, maxit=500)
    X = Xd.cpu().numpy()
    bn = np.linalg.norm(B, axis=0)
    rn_ = np.linalg.norm(B - A @ X, axis=0)
    ok = np.where(bn > 0, rn_ / np.where(bn > 0, bn, 1.0), rn_)
    assert np.all(ok < 1e-8), ok.max()
    assert np.all(X[:, 3] == 0.0)
    # single-vector stationary solves of a few columns: the multi solve runs
    # until its slowest column converges
    its = []
    for c in (0, 1, s - 1):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        its.append(h.solve(torch.from_numpy(B[:, c].copy()).to(dev), x, rtol=1e-8, maxit=500)["iters"])
        assert np.max(np.abs(x.cpu().numpy() - X[:, c])) <= 1e-5 * np.max(np.abs(X[:, c]))
    assert info["iters"] >= max(its) - 1
    h.close()


def test_solve_multi_host_buffers(env):
    torch, dev, rn = env
    pr = PR.poisson_problem(37)
    n = pr.A.n_rows
    B = np.random.default_rng(8).uniform(-1.0, 1.0, (n, 8))
    X = np.zeros_like(B)
    h = _hier(env, pr, outer=rn.RN_OUTER_STATIONARY)
    info = h.solve_multi(B, X, rtol=1e-8)
    res = np.linalg.norm(B - pr.A.to_scipy() @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert info["status"] == 0 and np.all(res < 1e-8)
    h.close()


def test_batched_problems_match_individual_solves(env):
    """Uneven independent problems set up and solved concurrently
    (rn_setup_batched / rn_solve_batched): every hierarchy and solution is
    bit-identical to building and solving that problem alone."""
    torch, dev, rn = env
    probs = PR.batch_aniso_problems(count=6, seed=7, side_lo=24, side_hi=96)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    params = rn.params_from_config(PR.PARAMS_ANISO, precision=rn.RN_MIXED)
    dev_probs = [(t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.B.reshape(-1))) for p in probs]
    hs = rn.setup_batched(dev_probs, params=params, threads=3)
    bs = [t(p.b) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = rn.solve_batched(hs, bs, xs, rtol=1e-8, maxit=1000)
    for p, h, x, info, dp in zip(probs, hs, xs, infos, dev_probs):
        assert info["status"] == 0
        xr = x.cpu().numpy()
        assert np.linalg.norm(p.b - p.A.to_scipy() @ xr) / np.linalg.norm(p.b) < 1e-8
        h1 = rn.Hierarchy(*dp, params=params)
        x1 = torch.zeros_like(x)
        i1 = h1.solve(t(p.b), x1, rtol=1e-8, maxit=1000)
        assert i1["iters"] == info["iters"]
        assert np.array_equal(x1.cpu().numpy(), xr)
        assert np.array_equal(h1.export_csr(0, 4)[2], h.export_csr(0, 4)[2])
        h1.close()
        h.close()
