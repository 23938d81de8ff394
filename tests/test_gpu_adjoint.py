"""GPU: differentiation through the AMG solve (the variable-coefficient
workload): torch.autograd through ``adjoint.solve`` against the FP64 adjoint
reference (direct solves, hand-derived chain rule) and against central
differences of the loss computed with AMG solves."""
import numpy as np
import pytest

from paper_1610_03154_gb300 import problems as PR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03154_gb300 import adjoint, rn

    return torch, torch.device("cuda:0"), adjoint, rn


def _setup(env, m, seed=21, seed_obs=22):
    torch, dev, adjoint, rn = env
    from oracle import adjoint_ref as ar
    import scipy.sparse.linalg as spla

    th = PR.gaussian_field(m, seed)
    th_obs = PR.gaussian_field(m, seed_obs)
    f = np.full(m * m, 1.0 / (m * m))
    u_obs = spla.spsolve(ar.operator(m, th_obs).tocsc(), f)
    op = adjoint.VarCoefFV(m, dev)
    params = rn.params_from_config(PR.PARAMS_VARCOEF)
    return th, f, u_obs, op, params


def _gpu_loss_grad(env, th, f, u_obs, op, params, rtol):
    torch, dev, adjoint, rn = env
    t = torch.tensor(th, dtype=torch.float64, device=dev, requires_grad=True)
    fd = torch.tensor(f, dtype=torch.float64, device=dev)
    uo = torch.tensor(u_obs, dtype=torch.float64, device=dev)
    u = adjoint.solve(op.values(t), fd, op.rowptr, op.col, params=params, rtol=rtol)
    L = 0.5 * torch.sum((u - uo) ** 2)
    L.backward()
    return float(L.detach()), t.grad.cpu().numpy()


@pytest.mark.parametrize("m,rtol", [(16, 1e-13), (48, 1e-12)])
def test_adjoint_gradient_matches_fp64_reference(env, m, rtol):
    """rtol: near the FP64 attainable residual of each grid (the oracle's
    CG stalls at 4e-13 on 48^2)."""
    from oracle import adjoint_ref as ar

    th, f, u_obs, op, params = _setup(env, m)
    L, g = _gpu_loss_grad(env, th, f, u_obs, op, params, rtol=rtol)
    Lr, gr, _ = ar.loss_and_grad(m, th, f, u_obs)
    assert abs(L - Lr) <= 1e-9 * abs(Lr)
    assert np.max(np.abs(g - gr)) <= 1e-7 * np.max(np.abs(gr))


def test_adjoint_gradient_central_differences_512(env):
    """The full-size workload: 512^2 cells.  The gradient from AMG solves
    (true relative residual 1e-10, near FP64's attainable accuracy on this
    grid) against central differences (h = 1e-6) of the loss on 32 random
    cells, each loss from a sparse direct solve on the host."""
    torch, dev, adjoint, rn = env
    import scipy.sparse.linalg as spla
    from oracle import adjoint_ref as ar

    m = 512
    th, f, u_obs, op, params = _setup(env, m)
    L, g = _gpu_loss_grad(env, th, f, u_obs, op, params, rtol=1e-10)
    rng = np.random.default_rng(5)
    cells = rng.choice(m * m, 32, replace=False)
    h = 1e-6
    thetas = []
    for c in cells:
        for sgn in (1.0, -1.0):
            t = th.copy()
            t[c] += sgn * h
            thetas.append(t)
    # 64 direct solves on the host's cores (spawned workers: CUDA is live here)
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        losses = list(ex.map(_host_loss, [(m, t, f, u_obs) for t in thetas]))
    fd = np.array([(losses[2 * k] - losses[2 * k + 1]) / (2 * h) for k in range(len(cells))])
    scale = np.max(np.abs(g))
    assert np.max(np.abs(g[cells] - fd)) <= 1e-4 * scale, (g[cells], fd)


def _host_loss(args):
    from oracle import adjoint_ref as ar

    m, t, f, u_obs = args
    return ar.loss(m, t, f, u_obs)


def test_adjoint_nonsymmetric_matches_dense(env):
    """A nonsymmetric operator (upwind convection-diffusion): the adjoint
    solve runs on a hierarchy built for A^T; gradients with respect to the
    values and the right-hand side against dense FP64 formulas."""
    torch, dev, adjoint, rn = env
    pr = PR.convdiff_problem(24)
    A = pr.A
    Ad = A.to_scipy().toarray()
    n = A.n_rows
    rng = np.random.default_rng(9)
    w = rng.standard_normal(n)
    b = pr.b
    rp = torch.tensor(A.rowptr, device=dev)
    ci = torch.tensor(A.col, device=dev)
    vals = torch.tensor(A.val, dtype=torch.float64, device=dev, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, device=dev, requires_grad=True)
    params = rn.params_from_config(pr.params, outer=rn.RN_OUTER_FGMRES)
    x = adjoint.solve(vals, bt, rp, ci, params=params, rtol=1e-13, symmetric=False)
    L = torch.sum(torch.tensor(w, device=dev) * x)
    L.backward()
    xr = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad.T, w)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    gv = -lam[rows] * xr[A.col]
    assert np.max(np.abs(x.detach().cpu().numpy() - xr)) <= 1e-10 * np.max(np.abs(xr))
    assert np.max(np.abs(bt.grad.cpu().numpy() - lam)) <= 1e-9 * np.max(np.abs(lam))
    assert np.max(np.abs(vals.grad.cpu().numpy() - gv)) <= 1e-9 * np.max(np.abs(gv))
