"""The allocation-free tree permutation (kf_tree_perm_noalloc) against the
regular entry point.

kf_tree_perm_noalloc serves callers that must not allocate device memory
(allocator callbacks, latency-bound loops where cudaMalloc would synchronize,
processes whose memory belongs to another pool).  It keeps its scratch in one
static device array shared by every call, so this file checks two calls in a
row against kf_tree_build/kf_tree_perm: the permutation and the permuted
points must agree bit for bit, as every tree comparison in this suite does.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1701_02324_gb300 as kf  # noqa: E402
from paper_1701_02324_gb300 import _abi  # noqa: E402


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def noalloc_perm(X, m):
    lib = _abi.load()
    N, d = X.shape
    Xt = torch.empty_like(X)
    perm = torch.empty(N, dtype=torch.int64, device=X.device)
    st = lib.kf_tree_perm_noalloc(_ptr(X), N, d, m, _ptr(Xt), _ptr(perm),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _abi.check(st)
    torch.cuda.synchronize()
    return Xt, perm


@pytest.mark.parametrize("N,d,m,seed", [(4096, 8, 256, 1), (3001, 5, 100, 2), (65536, 8, 512, 3)])
def test_noalloc_matches_tree_build_twice(N, d, m, seed):
    X = torch.from_numpy(np.random.default_rng(seed).random((N, d))).cuda()
    ref = kf.Tree(X, m).perm()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        Xt, perm = noalloc_perm(X, m)
        assert torch.equal(perm, ref)
        assert torch.equal(Xt, X[perm])
    # a different input right after: no state leaks between calls
    X2 = torch.from_numpy(np.random.default_rng(seed + 100).random((N, d))).cuda()
    Xt2, perm2 = noalloc_perm(X2, m)
    assert torch.equal(perm2, kf.Tree(X2, m).perm())
    assert torch.equal(Xt2, X2[perm2])


def test_noalloc_call_allocates_no_device_memory():
    """The property the entry point exists for: once the library's module and
    its static array are loaded (one warm-up call), a call changes neither
    the device's free memory nor what PyTorch's allocator holds."""
    X = torch.from_numpy(np.random.default_rng(5).random((20000, 6))).cuda()
    Xt = torch.empty_like(X)
    perm = torch.empty(X.shape[0], dtype=torch.int64, device="cuda")
    lib = _abi.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _abi.check(lib.kf_tree_perm_noalloc(_ptr(X), X.shape[0], 6, 300, _ptr(Xt), _ptr(perm), stream))
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    _abi.check(lib.kf_tree_perm_noalloc(_ptr(X), X.shape[0], 6, 300, _ptr(Xt), _ptr(perm), stream))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(Xt, X[perm])


def test_noalloc_rejects_nonfinite_input_without_writing():
    """Non-finite coordinates give KF_EINVAL and leave both outputs as they were."""
    lib = _abi.load()
    X = torch.from_numpy(np.random.default_rng(6).random((1000, 3))).cuda()
    X[17, 1] = float("nan")
    Xt = torch.full_like(X, 7.0)
    perm = torch.full((1000,), -3, dtype=torch.int64, device="cuda")
    st = lib.kf_tree_perm_noalloc(_ptr(X), 1000, 3, 64, _ptr(Xt), _ptr(perm), None)
    assert st == _abi.KF_EINVAL
    torch.cuda.synchronize()
    assert bool((Xt == 7.0).all()) and bool((perm == -3).all())


def test_noalloc_rejects_sizes_beyond_limit():
    lib = _abi.load()
    X = torch.zeros((65537, 1), dtype=torch.float64, device="cuda")
    out = torch.empty_like(X)
    perm = torch.empty(65537, dtype=torch.int64, device="cuda")
    st = lib.kf_tree_perm_noalloc(_ptr(X), 65537, 1, 16, _ptr(out), _ptr(perm), None)
    assert st == _abi.KF_EINVAL
    assert b"65536" in lib.kf_last_error(None)
    Xd = torch.zeros((4, 1025), dtype=torch.float64, device="cuda")     # d above kf_tree_build's limit
    st = lib.kf_tree_perm_noalloc(_ptr(Xd), 4, 1025, 1, _ptr(torch.empty_like(Xd)),
                                  _ptr(torch.empty(4, dtype=torch.int64, device="cuda")), None)
    assert st == _abi.KF_EINVAL
    Xw = torch.zeros((4096, 200), dtype=torch.float64, device="cuda")   # N * d > 2^19
    st = lib.kf_tree_perm_noalloc(_ptr(Xw), 4096, 200, 16, _ptr(torch.empty_like(Xw)),
                                  _ptr(torch.empty(4096, dtype=torch.int64, device="cuda")), None)
    assert st == _abi.KF_EINVAL
