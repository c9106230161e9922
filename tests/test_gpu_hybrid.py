"""The hybrid level-restricted solver (Sec. II-C, Algorithms 6-8) on the GPU
against the oracle's (kfo_hybrid, pinned in test_oracle_pins.py), through the
C ABI (needs a GB300).

Frontier at level L: the subtrees of the 2^L nodes of level L are skeletonized
and factorized like the direct solver's, nothing above them is compressed, and
the reduced system I + VW of the frontier skeletons is factored.  Bars: the
frontier subtrees' skeletons equal the oracle's (the same sampled-QR pivots);
the FP64 path's solution and operator within 1e-10 relative of the oracle's;
the mixed path (FP32 frontier subtrees, FP64 reduced system) refined by GMRES
against its FP64-accurate operator within 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1701_02324_gb300 as kf  # noqa: E402
from paper_1701_02324_gb300 import _abi  # noqa: E402

FP64, MIXED = kf.KF_PREC_FP64, kf.KF_PREC_MIXED


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def frontier_nodes(o, L):
    """Every node of the frontier subtrees: levels L..D."""
    return [a for a in range(1 << L, 1 << (o.D + 1))]


@pytest.mark.parametrize("N,d,m,h,lam,tau,smax,L,seed", [
    (4096, 8, 256, 0.5, 1.0, 1e-6, 64, 1, 31),
    (4096, 8, 256, 0.5, 1.0, 1e-6, 64, 2, 31),
    (4096, 8, 256, 0.5, 1.0, 1e-6, 64, 3, 31),
    (3001, 5, 100, 0.35, 0.6, 1e-7, 32, 2, 32),   # ragged tree, depth 5
    (3001, 5, 100, 0.35, 0.6, 1e-7, 32, 5, 32),   # frontier at the leaves
])
def test_hybrid_fp64_matches_oracle(N, d, m, h, lam, tau, smax, L, seed):
    rng = np.random.default_rng(seed)
    X, B = rng.random((N, d)), rng.standard_normal((N, 2))
    o = oracle.Oracle(X, m)
    assert o.hybrid(L, h, tau, smax, lam) == oracle.KFO_OK
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    assert np.array_equal(tree.perm().cpu().numpy(), o.perm())
    F = kf.Factor(tree, h, lam, tau, smax, precision=FP64, hybrid_level=L)
    r = F.ranks()
    nodes = frontier_nodes(o, L)
    assert all(int(r[a]) == o.rank(a) for a in nodes)
    assert all(np.array_equal(F.skeleton(a), o.skel(a)) for a in nodes)
    assert all(int(r[a]) == 0 for a in range(2, 1 << L))       # nothing above the frontier is compressed
    Bt = torch.from_numpy(B).cuda()
    xo = np.stack([o.hybrid_solve(B[:, j]) for j in range(2)], axis=1)
    assert rel(F.solve(Bt[:, 0]).cpu().numpy(), xo[:, 0]) <= 1e-10
    assert rel(F.solve(Bt).cpu().numpy(), xo) <= 1e-10               # two right-hand sides at once
    yo = o.hybrid_matvec(B[:, 1])
    assert rel(F.matvec(Bt[:, 1]).cpu().numpy(), yo) <= 1e-12
    # the solve inverts the operator: residual against the GPU's own operator
    x = F.solve(Bt[:, 0])
    assert rel(F.matvec(x).cpu().numpy(), B[:, 0]) <= 1e-10


@pytest.mark.parametrize("L", [1, 2, 3])
def test_hybrid_mixed_refined_matches_oracle(L):
    """Mixed path: FP32 frontier subtrees and FP64 reduced system, refined by
    GMRES against the FP64-accurate operator to eps_r <= 1e-11."""
    rng = np.random.default_rng(40 + L)
    N, m, h, lam, tau, smax = 4096, 256, 0.5, 1.0, 1e-6, 64
    X, b = rng.random((N, 8)), rng.standard_normal(N)
    o = oracle.Oracle(X, m)
    assert o.hybrid(L, h, tau, smax, lam) == oracle.KFO_OK
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    F = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, hybrid_level=L, refine_tol=1e-11)
    x, info = F.solve(torch.from_numpy(b).cuda(), info=True)
    assert info["eps_r"] <= 1e-11
    assert rel(x.cpu().numpy(), o.hybrid_solve(b)) <= 1e-8
    # the unrefined mixed sweep is within the FP32 factors' accuracy
    G = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, hybrid_level=L, refine_max_iter=-1, fp64_operator=False)
    assert rel(G.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.hybrid_solve(b)) <= 1e-4


def test_hybrid_unsupported_requests_are_reported():
    rng = np.random.default_rng(50)
    X, b = rng.random((2048, 4)), rng.standard_normal(2048)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 128)        # depth 4
    with pytest.raises(kf.KFError) as e:
        kf.Factor(tree, 0.5, 1.0, 1e-6, 32, hybrid_level=5)  # deeper than the tree
    assert e.value.status == _abi.KF_EINVAL
    with pytest.raises(kf.KFError) as e:
        kf.Factor(tree, 0.5, 1.0, 1e-6, 256, hybrid_level=3)  # 2^3 * 256 rows > 1024
    assert e.value.status == _abi.KF_EUNSUPPORTED
    F = kf.Factor(tree, 0.5, 1.0, 1e-6, 32, hybrid_level=2)
    bt = torch.from_numpy(b).cuda()
    with pytest.raises(kf.KFError) as e:
        F.solve(bt, transpose=True)
    assert e.value.status == _abi.KF_EUNSUPPORTED
    with pytest.raises(kf.KFError) as e:
        F.grad(bt, bt)
    assert e.value.status == _abi.KF_EUNSUPPORTED
    x = F.solve(bt)                                         # the context is still usable
    assert rel(F.matvec(x).cpu().numpy(), b) <= 1e-10
