"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/rn.h, fills defaults, and rejects bad arguments before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rn():
    from paper_1610_03154_gb300 import build

    build.build()
    from paper_1610_03154_gb300 import rn as mod

    return mod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rn_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rn_setup", "rn_solve", "rn_free", "rn_default_params", "rn_hierarchy_stats",
                     "rn_export_csr", "rn_export_vec", "rn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(rn):
    missing = [n for n in declared_functions() if not hasattr(rn.lib, n)]
    assert not missing, missing


def test_default_params(rn):
    p = rn.default_params()
    assert p.soc_theta == 0.25 and p.degree == 2 and p.n_sweeps == 4
    assert abs(p.omega - 2.0 / 3.0) < 1e-16
    assert p.symmetric == 1 and p.nu_pre == 1 and p.nu_post == 1
    assert rn.rn_default_params(None) == rn.RN_EINVAL


def test_setup_rejects_bad_arguments_without_gpu(rn):
    p = rn.default_params()
    h = C.c_void_p(123)
    assert rn.rn_setup(None, None, None, 1, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
    assert h.value is None
    A = rn.rn_csr(0, 0, 0, None, None, None)
    assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, 1, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
    A = rn.rn_csr(4, 4, 4, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8))
    for k in (0, 5):  # 1 <= k <= RN_MAX_CANDIDATES = 4
        assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, k, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
        assert b"k must be" in rn.rn_last_error()
    for bs, k in ((4, 4), (0, 1), (3, 4), (2, 1)):  # block_size in [1, 3], dividing n = 4, at most k
        p = rn.default_params(block_size=bs)
        assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, k, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
        assert b"block_size" in rn.rn_last_error()
    p = rn.default_params()
    p.degree = -1
    assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, 1, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
    p = rn.default_params(symmetric=0)
    assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, 1, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
    assert rn.rn_solve(None, None, None, 0, 1e-8, 10, None) == rn.RN_EINVAL
    rn.rn_free(None)


def test_allocator_hooks_must_come_in_pairs(rn):
    """alloc without dealloc (or the reverse) is rejected before any allocation."""
    A = rn.rn_csr(4, 4, 4, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8))
    h = C.c_void_p()
    p = rn.default_params()
    assert not p.alloc and not p.dealloc and p.alloc_ctx is None
    p.alloc = rn.TORCH_ALLOC
    assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, 1, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
    assert b"alloc and dealloc" in rn.rn_last_error()
    p = rn.default_params()
    p.dealloc = rn.TORCH_DEALLOC
    assert rn.rn_setup(C.byref(A), C.c_void_p(8), None, 1, 0, C.byref(p), C.byref(h)) == rn.RN_EINVAL
    assert h.value is None


def test_status_strings(rn):
    for i, name in enumerate(rn.STATUS_NAMES):
        assert rn.rn_status_string(i).decode() == name


def test_profile_api_without_launches(rn):
    rn.profile_reset()
    assert rn.profile_read() == {}


def test_batch_rejects_bad_arguments_without_gpu(rn):
    b = C.c_void_p(123)
    assert rn.rn_batch_merge(0, None, None, C.byref(b)) == rn.RN_EINVAL
    assert b.value is None
    H = (C.c_void_p * 2)(None, None)
    assert rn.rn_batch_merge(2, H, None, C.byref(b)) == rn.RN_EINVAL
    assert b"NULL" in rn.rn_last_error()
    assert rn.rn_batch_solve(None, None, None, 1e-8, 10, None) == rn.RN_EINVAL
    assert rn.rn_batch_cycle(None, None, None) == rn.RN_EINVAL
    rn.rn_batch_free(None)
