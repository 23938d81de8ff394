"""rn_energy_min_noalloc: the CG energy minimisation for callers that must not
allocate device memory (for example a host framework whose caching allocator
already holds the GPU's memory).  It must give the same result as
rn_energy_min on the same inputs, on repeated calls (its static scratch keeps
the previous call's contents), make no allocation (the library's allocation
counter and torch's allocator both unchanged across the call), and reject
inputs above its stated limits.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1610_03154_gb300 import problems as PR

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the floating-point bar of the parity tests


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03154_gb300 import rn

    return torch, torch.device("cuda:0"), rn


def _level(oracle, pr):
    oh = oracle.Hierarchy(pr.A.to_scipy(), pr.B, **pr.params)
    return oh.levels[0]


def test_noalloc_matches_allocating_entry_point_on_two_calls(env, oracle):
    torch, dev, rn = env
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cases = [(PR.aniso_problem(96), 6), (PR.poisson_problem(64), 4)]
    for pr, sweeps in cases:
        L = _level(oracle, pr)
        A, N, T = L.A, L.N, L.T
        args = (d(A.indptr.astype(np.int32)), d(A.indices.astype(np.int32)), d(A.data),
                d(N.indptr.astype(np.int32)), d(N.indices.astype(np.int32)), N.shape[1], d(L.rowtype), d(L.Bc))
        P_ref = d(T.data.astype(np.float64))
        a0 = rn.rn_allocation_count()
        rn.energy_min(*args, P_ref, sweeps, method=rn.RN_ENERGY_CG)
        assert rn.rn_allocation_count() > a0  # the counter sees the allocating entry point's scratch
        ref = P_ref.cpu().numpy()
        for _ in range(2):  # the second call starts from the first call's leftover scratch
            P = d(T.data.astype(np.float64))
            torch.cuda.synchronize()
            a1 = rn.rn_allocation_count()
            t1 = torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0)
            rn.energy_min_noalloc(*args, P, sweeps)
            assert rn.rn_allocation_count() == a1, "rn_energy_min_noalloc allocated memory"
            assert torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0) == t1
            got = P.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    torch, dev, rn = env
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    A = PR.poisson5(520)  # 270,400 rows > 262,144
    n = A.n_rows
    P = d(np.ones(n))
    with pytest.raises(rn.RNError) as e:
        rn.energy_min_noalloc(d(A.rowptr), d(A.col), d(A.val), d(np.arange(n + 1, dtype=np.int32)),
                              d(np.zeros(n, np.int32)), 1, d(np.zeros(n, np.int32)), d(np.ones(1)), P, 2)
    assert e.value.status == rn.RN_EINVAL
    assert "limit" in str(e.value)
