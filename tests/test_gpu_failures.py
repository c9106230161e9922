"""Failure statuses through the C ABI (needs a GB300), made on the host: an
allocator callback that returns NULL (KF_ENOMEM, nothing leaked or left
half-built) and a refinement that cannot reach its target (KF_ENOTCONV); the
context stays usable after each.  No GPU fault is provoked."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1701_02324_gb300 as kf  # noqa: E402
from paper_1701_02324_gb300 import _abi  # noqa: E402

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FAIL = [False]
_LIVE = {}


@_ALLOC_FN
def _switchable_alloc(nbytes, stream, user):
    """Torch's caching allocator, or NULL while _FAIL[0] is set."""
    if _FAIL[0]:
        return None
    p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    _LIVE[int(p)] = int(nbytes)
    return p


@_FREE_FN
def _tracked_free(ptr, nbytes, stream, user):
    if ptr:
        _LIVE.pop(int(ptr), None)
        torch.cuda.caching_allocator_delete(int(ptr))


def test_allocator_failure_is_reported():
    lib = _abi.load()
    alloc = _abi.kf_alloc(ctypes.cast(_switchable_alloc, ctypes.c_void_p).value,
                          ctypes.cast(_tracked_free, ctypes.c_void_p).value, None)
    ctx = ctypes.c_void_p()
    assert lib.kf_create(ctypes.byref(ctx), ctypes.byref(alloc)) == _abi.KF_OK
    X = torch.rand((4096, 8), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        # the tree's own buffers cannot be had: KF_ENOMEM, no tree, nothing left allocated
        _FAIL[0] = True
        tree = ctypes.c_void_p()
        st = lib.kf_tree_build(ctx, X.data_ptr(), kf.KF_F64, 4096, 8, 256, stream, ctypes.byref(tree))
        assert st == _abi.KF_ENOMEM and not tree.value
        assert not _LIVE
        # a tree, then a factorization whose buffers cannot be had
        _FAIL[0] = False
        st = lib.kf_tree_build(ctx, X.data_ptr(), kf.KF_F64, 4096, 8, 256, stream, ctypes.byref(tree))
        assert st == _abi.KF_OK and tree.value
        held = dict(_LIVE)
        _FAIL[0] = True
        fac = ctypes.c_void_p()
        o = kf._opts()
        st = lib.kf_factorize(tree, 0.5, 1.0, 1e-6, 64, ctypes.byref(o), stream, ctypes.byref(fac))
        assert st == _abi.KF_ENOMEM and not fac.value
        assert _LIVE == held                      # the partial factor was released
        # the context still works once memory is there again
        _FAIL[0] = False
        st = lib.kf_factorize(tree, 0.5, 1.0, 1e-6, 64, ctypes.byref(o), stream, ctypes.byref(fac))
        assert st == _abi.KF_OK and fac.value
        b = torch.randn(4096, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        assert lib.kf_solve(fac, b.data_ptr(), x.data_ptr(), 1, 4096, kf.KF_F64, 0, stream, None) == _abi.KF_OK
        torch.cuda.synchronize()
        assert torch.isfinite(x).all()
        assert lib.kf_factor_free(fac) == _abi.KF_OK
        assert lib.kf_tree_free(tree) == _abi.KF_OK
    finally:
        _FAIL[0] = False
        lib.kf_destroy(ctx)


def test_refinement_not_reaching_its_target_is_reported():
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.random((4096, 8))).cuda()
    b = torch.from_numpy(rng.standard_normal(4096)).cuda()
    tree = kf.Tree(X, 256)
    F = kf.Factor(tree, 0.5, 1.0, 1e-6, 64, precision=kf.KF_PREC_MIXED, refine_tol=1e-30, refine_max_iter=2,
                  gmres_restart=-1)
    with pytest.raises(kf.KFError) as e:
        F.solve(b)
    assert e.value.status == _abi.KF_ENOTCONV
    G = kf.Factor(tree, 0.5, 1.0, 1e-6, 64, precision=kf.KF_PREC_MIXED, refine_tol=1e-10)
    x, info = G.solve(b, info=True)
    assert info["eps_r"] <= 1e-10


def test_device_wait_that_runs_out_is_reported():
    """KF_ETIMEOUT from a bounded device wait: with the probe on, every CTA of
    the mixed path's tcgen05 products waits on an mbarrier that nothing
    arrives at, gives up after a few polls, flags the time-out and returns
    without its product.  The factor's status word reports KF_ETIMEOUT; with
    the probe off the next factorization on the same context solves to the
    usual accuracy."""
    lib = _abi.load()
    rng = np.random.default_rng(4)
    X = torch.from_numpy(rng.random((4096, 8))).cuda()
    b = torch.from_numpy(rng.standard_normal(4096)).cuda()
    tree = kf.Tree(X, 256)
    assert lib.kf_test_tc_wait_probe(-1) == _abi.KF_EINVAL
    assert lib.kf_test_tc_wait_probe(64) == _abi.KF_OK
    try:
        F = kf.Factor(tree, 0.5, 1.0, 1e-6, 64, precision=kf.KF_PREC_MIXED, sync_errors=False, refine_max_iter=-1)
        assert F.device_status() == _abi.KF_ETIMEOUT
        del F
    finally:
        assert lib.kf_test_tc_wait_probe(0) == _abi.KF_OK
    G = kf.Factor(tree, 0.5, 1.0, 1e-6, 64, precision=kf.KF_PREC_MIXED, refine_tol=1e-10)
    assert G.device_status() == _abi.KF_OK
    x, info = G.solve(b, info=True)
    assert info["eps_r"] <= 1e-10
    H = kf.Factor(tree, 0.5, 1.0, 1e-6, 64, precision=kf.KF_PREC_FP64)
    xh = H.solve(b)
    assert float(torch.linalg.norm(x - xh) / torch.linalg.norm(xh)) <= 1e-8
