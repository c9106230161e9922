"""Several right-hand sides at once (needs a GB300): the solve sweep (Alg. 3)
and the hierarchical operator with k >= 2 columns run kernels of their own
(the leaf solves and reduced-system solves with the block of columns in
shared memory, tiled row updates, 16-column sums, tiled pushes), which read
each factor entry once per 8 or 16 columns.  Every column of a block solve
is compared with the same column solved alone (k = 1 kernels) and, on the
FP64 path, with the oracle; the transposed sweep and the FP64-accurate
operator likewise, the latter also with its V pass on the tensor cores
(tc_operator: exact BF16 digit products).  Shapes: ragged leaves, block widths that leave a partial
chunk (5, 19), and the levels with and without the explicit Z^-1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1701_02324_gb300 as kf  # noqa: E402

FP64, MIXED = kf.KF_PREC_FP64, kf.KF_PREC_MIXED


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def problem():
    rng = np.random.default_rng(0x5EED)
    N, d, m, smax, h, lam, tau = 3001, 6, 300, 48, 0.45, 0.7, 1e-6
    X = rng.random((N, d))
    o = oracle.Oracle(X, m)
    o.skeletonize(h, tau, smax)
    o.factorize(lam)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    return dict(N=N, smax=smax, h=h, lam=lam, tau=tau, o=o, tree=tree, rng=rng)


@pytest.mark.parametrize("zinv", [0, -1])  # default explicit Z^-1 on the upper levels / LU solves everywhere
@pytest.mark.parametrize("k", [2, 5, 16, 19])
def test_block_solve_equals_column_solves_fp64(problem, k, zinv):
    p = problem
    F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=FP64, zinv_max_nodes=zinv)
    B = p["rng"].standard_normal((p["N"], k))
    Bt = torch.from_numpy(B).cuda()
    Xb = F.solve(Bt).cpu().numpy()
    Xt = F.solve(Bt, transpose=True).cpu().numpy()
    for c in range(k):
        xc = F.solve(Bt[:, c].contiguous()).cpu().numpy()
        assert rel(Xb[:, c], xc) <= 1e-13, c
        xtc = F.solve(Bt[:, c].contiguous(), transpose=True).cpu().numpy()
        assert rel(Xt[:, c], xtc) <= 1e-13, c
    assert rel(Xb, p["o"].solve(B)) <= 1e-10
    assert rel(Xt, p["o"].solve(B, transpose=True)) <= 1e-10


@pytest.mark.parametrize("k", [3, 8, 16, 40])
def test_block_solve_equals_column_solves_mixed(problem, k):
    """FP32 sweep: the block's sums run in another order than the single
    column's, so columns agree to FP32 rounding amplified by the conditioning
    (1e-5 here); refined by GMRES the block meets the oracle at 1e-9."""
    p = problem
    F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, refine_max_iter=-1)
    B = p["rng"].standard_normal((p["N"], k))
    Bt = torch.from_numpy(B).cuda()
    Xb = F.solve(Bt).cpu().numpy()
    for c in range(k):
        xc = F.solve(Bt[:, c].contiguous()).cpu().numpy()
        assert rel(Xb[:, c], xc) <= 1e-5, c
    G = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, refine_tol=1e-12)
    assert rel(G.solve(Bt).cpu().numpy(), p["o"].solve(B)) <= 1e-9
    # the transpose solve refined against the transposed FP64-accurate operator (k-column passes)
    assert rel(G.solve(Bt, transpose=True).cpu().numpy(), p["o"].solve(B, transpose=True)) <= 1e-9


@pytest.mark.parametrize("k", [2, 7, 16, 33])
def test_block_operator_equals_column_operator(problem, k):
    """lambda x + K~ x for a block of columns: the FP64 path and the mixed
    path's FP64-accurate (double-float) operator against single columns and
    the oracle's matvec."""
    p = problem
    B = p["rng"].standard_normal((p["N"], k))
    Bt = torch.from_numpy(B).cuda()
    ref = p["o"].matvec(B)
    for prec, kw in ((FP64, {}), (MIXED, {"fp64_operator": True})):
        F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=prec, **kw)
        Yb = F.matvec(Bt).cpu().numpy()
        for c in range(k):
            yc = F.matvec(Bt[:, c].contiguous()).cpu().numpy()
            assert rel(Yb[:, c], yc) <= 1e-13, (prec, c)
        assert rel(Yb, ref) <= (1e-12 if prec == FP64 else 1e-12), prec


@pytest.mark.parametrize("k", [16, 33, 64])
def test_tensor_core_v_pass_equals_double_float(problem, k):
    """The FP64-accurate operator with its V pass as exact BF16 digit products
    on the tensor cores (16 or more columns) against the double-float
    CUDA-core pass (tc_operator off), single columns and the oracle's matvec;
    node starts here are not multiples of 8 and nodes span several 1024-row
    chunks and ragged 128-row windows."""
    p = problem
    B = p["rng"].standard_normal((p["N"], k)) * np.exp(p["rng"].uniform(-3, 3, k))  # columns of unequal scale
    Bt = torch.from_numpy(B).cuda()
    ref = p["o"].matvec(B)
    F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, fp64_operator=True,
                  tc_operator=True)
    G = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, fp64_operator=True)
    Yt = F.matvec(Bt).cpu().numpy()
    Yd = G.matvec(Bt).cpu().numpy()
    for c in range(k):
        assert rel(Yt[:, c], Yd[:, c]) <= 1e-13, c
    assert rel(Yt, ref) <= 1e-12
    # refined block solve on those factors: the residuals come from the tensor-core pass
    H = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, fp64_operator=True,
                  tc_operator=True, refine_tol=1e-12)
    assert rel(H.solve(Bt).cpu().numpy(), p["o"].solve(B)) <= 1e-9


def test_tensor_core_v_pass_two_skeleton_tiles():
    """Ranks above 128 (two 128-column skeleton tiles per node) and a column
    count that leaves a partial group of 32: the tensor-core V pass against
    the double-float pass."""
    rng = np.random.default_rng(0x0253)
    N, d, m, smax = 20000, 5, 512, 160
    X = torch.from_numpy(rng.random((N, d))).cuda()
    tree = kf.Tree(X, m)
    F = kf.Factor(tree, 0.25, 1.0, 1e-9, smax, precision=MIXED, fp64_operator=True, tc_operator=True)
    G = kf.Factor(tree, 0.25, 1.0, 1e-9, smax, precision=MIXED, fp64_operator=True)
    assert int(F.ranks().max()) > 128
    B = torch.from_numpy(rng.standard_normal((N, 40))).cuda()
    Yt, Yd = F.matvec(B).cpu().numpy(), G.matvec(B).cpu().numpy()
    for c in range(40):
        assert rel(Yt[:, c], Yd[:, c]) <= 1e-13, c



def test_tensor_core_operator_is_bitwise_deterministic(problem):
    """The tensor-core operator passes sum exact integers per window and
    reduce the chunks in a fixed order: two products give the same bits."""
    p = problem
    B = torch.from_numpy(p["rng"].standard_normal((p["N"], 33))).cuda()
    F = kf.Factor(p["tree"], p["h"], p["lam"], p["tau"], p["smax"], precision=MIXED, fp64_operator=True,
                  tc_operator=True)
    Y1, Y2 = F.matvec(B), F.matvec(B)
    assert torch.equal(Y1, Y2)
    X1, X2 = F.solve(B), F.solve(B)  # refined against that operator
    assert torch.equal(X1, X2)
