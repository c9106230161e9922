"""Memory-lean factors (row f2; Sec. III, storage), needs a GB300.

kf_opts.w_recompute keeps P^ for the leaves only, with T = Z^-1 P_c of every
node, and applies P^ of any level in the sweep as P^_leaf times the telescoped
T's (Eq. e:invtelescope) pushed down the tree (gathered up for the transpose
sweep); with v_storage = KF_V_RECOMPUTE the factorization also keeps only
three levels of V blocks.  The lean factorization solves like the standard
one (same skeletons, same reduced systems; only the order of the products
changes): FP64 within 1e-12 of the standard path and 1e-10 of the oracle,
forward and transpose, one and several right-hand sides; the mixed sweep
within FP32 accuracy of the standard sweep and refined within 1e-9 of the
oracle.  The factor holds (D - 3) N s_max fewer values of P^ (and of V),
plus the T's.
"""
import gc

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


def factor_bytes(make):
    """Device bytes a factorization keeps (drawn through torch's caching
    allocator), and the factor."""
    gc.collect()
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    F = make()
    torch.cuda.synchronize()
    return torch.cuda.memory_allocated() - m0, F


@pytest.fixture(scope="module", params=[(4096, 8, 256, 64, 0.5), (3001, 5, 100, 32, 0.35)],
                ids=["N4096_depth4", "N3001_ragged_depth5"])
def problem(request):
    N, d, m, smax, h = request.param
    rng = np.random.default_rng(N + 11)
    X = rng.random((N, d))
    lam, tau = 0.8, 1e-6
    o = oracle.Oracle(X, m)
    o.skeletonize(h, tau, smax)
    o.factorize(lam)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    return dict(N=N, smax=smax, h=h, lam=lam, tau=tau, o=o, tree=tree, rng=rng)


@pytest.mark.parametrize("k", [1, 3, 16])
def test_lean_fp64_solves_match_standard_and_oracle(problem, k):
    p = problem
    F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=FP64)
    G = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=FP64, w_recompute=True)
    B = p["rng"].standard_normal((p["N"], k))
    Bt = torch.from_numpy(B if k > 1 else B[:, 0].copy()).cuda()
    for tr in (False, True):
        xs = F.solve(Bt, transpose=tr).cpu().numpy()
        xl = G.solve(Bt, transpose=tr).cpu().numpy()
        assert rel(xl, xs) <= 1e-12, tr
        xo = p["o"].solve(B if k > 1 else B[:, 0], transpose=tr)
        assert rel(xl, xo) <= 1e-10, tr


@pytest.mark.parametrize("k", [1, 16])
def test_lean_mixed_sweep_and_refined_solve(problem, k):
    p = problem
    F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, refine_max_iter=-1)
    G = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, refine_max_iter=-1,
                  w_recompute=True)
    B = p["rng"].standard_normal((p["N"], k))
    Bt = torch.from_numpy(B if k > 1 else B[:, 0].copy()).cuda()
    for tr in (False, True):
        assert rel(G.solve(Bt, transpose=tr).cpu().numpy(), F.solve(Bt, transpose=tr).cpu().numpy()) <= 1e-5, tr
    R = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, refine_tol=1e-12,
                  w_recompute=True)
    xo = p["o"].solve(B if k > 1 else B[:, 0])
    assert rel(R.solve(Bt).cpu().numpy(), xo) <= 1e-9


def test_lean_keeps_leaf_phat_only_and_less_memory(problem):
    p = problem
    tree = p["tree"]
    bs, F = factor_bytes(lambda: kf.Factor(tree, p["h"], p["lam"], p["tau"], p["smax"], precision=FP64))
    bl, G = factor_bytes(lambda: kf.Factor(tree, p["h"], p["lam"], p["tau"], p["smax"], precision=FP64,
                                           w_recompute=True))
    D, N, s = tree.D, p["N"], p["smax"]
    saved = (D - min(D, 3)) * N * s * 8 - (1 << D) * 2 * s * s * 8  # P^ levels dropped, T's kept
    assert bs - bl >= 0.9 * saved
    for a in range(1 << D, 1 << (D + 1)):                        # the leaves' P^ is kept, equal
        lo, hi = p["o"].node_range(a)
        assert np.array_equal(G.Phat(a, hi - lo), F.Phat(a, hi - lo))
    lo, hi = p["o"].node_range(2)
    with pytest.raises(kf.KFError) as e:
        G.Phat(2, hi - lo)
    assert e.value.status == _abi.KF_EUNSUPPORTED


def test_lean_rejected_with_hybrid(problem):
    p = problem
    with pytest.raises(kf.KFError) as e:
        kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], hybrid_level=1, w_recompute=True)
    assert e.value.status == _abi.KF_EUNSUPPORTED


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_lean_v_and_w(problem, prec):
    """Both memory-lean schemes of Sec. III: V evaluated in the sweeps
    (KF_V_RECOMPUTE; the factorization keeps three levels of V blocks in turn)
    and W recomputed.  The solve matches the oracle (FP64: 1e-10; mixed refined:
    1e-9) and the factor holds (D - 3) N s_max fewer values of V and of P^."""
    p = problem
    tree = p["tree"]
    kw = dict(precision=prec) if prec == FP64 else dict(precision=prec, refine_tol=1e-12)
    bs, F = factor_bytes(lambda: kf.Factor(tree, p["h"], p["lam"], p["tau"], p["smax"], **kw))
    del F
    bl, G = factor_bytes(lambda: kf.Factor(tree, p["h"], p["lam"], p["tau"], p["smax"], v_storage=kf.KF_V_RECOMPUTE,
                                           w_recompute=True, **kw))
    D, N, s = tree.D, p["N"], p["smax"]
    ts = 8 if prec == FP64 else 4
    saved = ((D - min(D + 1, 3)) + (D - min(D, 3))) * N * s * ts - (1 << D) * 2 * s * s * ts
    assert bs - bl >= 0.9 * saved
    b = p["rng"].standard_normal(p["N"])
    bt = torch.from_numpy(b).cuda()
    tol = 1e-10 if prec == FP64 else 1e-9
    assert rel(G.solve(bt).cpu().numpy(), p["o"].solve(b)) <= tol
    assert rel(G.solve(bt, transpose=True).cpu().numpy(), p["o"].solve(b, transpose=True)) <= tol
