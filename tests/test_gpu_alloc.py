"""Device memory through the caller's hooks (rn_params alloc / dealloc /
alloc_ctx): torch's caching allocator, and a hook that runs out."""
import ctypes as C

import numpy as np
import pytest

from paper_1610_03154_gb300 import problems as PR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch, torch.device("cuda", 0)


@pytest.fixture(scope="module")
def rn(torch_dev):
    from paper_1610_03154_gb300 import build

    build.build()
    from paper_1610_03154_gb300 import rn as mod

    return mod


def _arrays(torch, d, pr):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
    A = pr.A
    return t(A.rowptr), t(A.col), t(A.val), t(pr.B.reshape(-1)), t(pr.b)


@pytest.mark.parametrize("precision", [0, 1])
def test_torch_allocator_same_bits_and_returns_memory(rn, torch_dev, precision):
    """A hierarchy on torch's caching allocator solves to the same bits as one
    on the library's pool, holds its buffers in torch's pool while it lives
    and gives all of them back at rn_free."""
    torch, d = torch_dev
    pr = PR.aniso_problem(96)
    rp, ci, va, B, b = _arrays(torch, d, pr)
    xs = []
    for hooked in (False, True):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated(d)
        p = rn.params_from_config(pr.params, precision=precision)
        if hooked:
            rn.use_torch_allocator(p)
        h = rn.Hierarchy(rp, ci, va, B, params=p)
        held = torch.cuda.memory_allocated(d) - base
        info = h.solve(b, x, rtol=1e-8, maxit=200)
        h.close()
        torch.cuda.synchronize()
        if hooked:
            assert held > 8 * pr.A.nnz  # at least A's values and indices live in torch's pool
        else:
            assert held == 0
        assert torch.cuda.memory_allocated(d) == base
        xs.append((info["iters"], x.cpu().numpy()))
    assert xs[0][0] == xs[1][0]
    assert np.array_equal(xs[0][1].view(np.uint64), xs[1][1].view(np.uint64))


def test_allocator_running_out_fails_cleanly(rn, torch_dev):
    """A hook that returns NULL fails the setup with RN_ENOMEM, and every
    buffer handed out before it is handed back."""
    torch, d = torch_dev
    pr = PR.poisson_problem(64)
    rp, ci, va, B, b = _arrays(torch, d, pr)
    live = {}
    calls = {"n": 0}

    @rn.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        calls["n"] += 1
        if calls["n"] > 40:
            return None
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), d.index, stream or 0)
        live[ptr] = nbytes
        return ptr

    @rn.DEALLOC_FN
    def dealloc(ptr, nbytes, stream, ctx):
        assert live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)

    p = rn.params_from_config(pr.params)
    p.alloc, p.dealloc = alloc, dealloc
    p.stream = C.c_void_p(torch.cuda.current_stream(d).cuda_stream)
    with pytest.raises(rn.RNError) as e:
        rn.Hierarchy(rp, ci, va, B, params=p)
    assert e.value.status == rn.RN_ENOMEM
    assert calls["n"] == 41 and not live
