"""Near-field sampling of S' on the GPU against the oracle (pinned in
test_oracle_near.py), through the C ABI (needs a GB300).

Integer results are compared bit for bit: every point's neighbour list
(randomized projection trees, FP32 leaf distances with sequential fused
multiply-adds, ties to the smaller position), every node's list, and the
skeletons the IDs pick from the resulting S'.  The factorization and solve
downstream are then held to the FP64 bar of 1e-10, the mixed path refined to
1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1701_02324_gb300 as kf  # noqa: E402
from paper_1701_02324_gb300 import _abi, inputs  # noqa: E402

FP64, MIXED = kf.KF_PREC_FP64, kf.KF_PREC_MIXED
SEED = 0x1701


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("N,d,m,kappa,trees,leaf,smax,h", [
    (4096, 8, 256, 16, 4, 512, 64, 0.5),     # several projection-tree leaves, list width 16
    (3001, 5, 100, 7, 3, 200, 32, 0.35),     # ragged trees, kappa below the width 8
    (2500, 70, 128, 12, 2, 300, 48, 2.5),    # d > 64: coordinates read from shared memory
    (2048, 6, 128, 32, 2, 256, 32, 0.4),     # list width 32
])
def test_near_field_lists_and_factorization_match_oracle(N, d, m, kappa, trees, leaf, smax, h):
    rng = np.random.default_rng(N + d)
    X, b = rng.random((N, d)), rng.standard_normal(N)
    tau, lam = 1e-6, 0.8
    o = oracle.Oracle(X, m)
    nbr_o = o.knn(kappa, trees, leaf, SEED)
    o.set_near(nbr_o, smax)                     # near_cap = n_samp / 2 = s_max
    o.skeletonize(h, tau, smax, n_samp=2 * smax, seed=SEED)
    o.factorize(lam)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    F = kf.Factor(tree, h, lam, tau, smax, precision=FP64, knn_kappa=kappa, knn_trees=trees, knn_leaf=leaf)
    assert np.array_equal(F.knn(), nbr_o)
    for a in range(2, o.nnodes + 1):
        pos, cnt = F.near(a)
        po, co = o.node_near(a)
        assert np.array_equal(pos, po) and np.array_equal(cnt, co), a
    r = F.ranks()
    nodes = range(2, o.nnodes + 1)
    assert all(int(r[a]) == o.rank(a) for a in nodes)
    same = sum(np.array_equal(F.skeleton(a), o.skel(a)) for a in nodes)
    assert same == len(nodes)
    xo = o.solve(b)
    bt = torch.from_numpy(b).cuda()
    assert rel(F.solve(bt).cpu().numpy(), xo) <= 1e-10
    G = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, knn_kappa=kappa, knn_trees=trees, knn_leaf=leaf,
                  refine_tol=1e-11)
    assert rel(G.solve(bt).cpu().numpy(), xo) <= 1e-8


def test_near_field_options_are_checked():
    X = np.random.default_rng(1).random((2048, 4))
    tree = kf.Tree(torch.from_numpy(X).cuda(), 256)
    for kw in ({"knn_kappa": 33}, {"knn_kappa": 8, "knn_leaf": 1}, {"knn_kappa": 8, "knn_trees": 65}):
        with pytest.raises(kf.KFError) as e:
            kf.Factor(tree, 0.5, 1.0, 1e-6, 32, **kw)
        assert e.value.status == _abi.KF_EINVAL
    tree2 = kf.Tree(torch.from_numpy(np.random.default_rng(2).random((4096, 4))).cuda(), 1024)
    with pytest.raises(kf.KFError) as e:                        # leaf of 1024 points x 17 > 16384
        kf.Factor(tree2, 0.5, 1.0, 1e-6, 32, knn_kappa=17)
    assert e.value.status == _abi.KF_EUNSUPPORTED
    F = kf.Factor(tree, 0.5, 1.0, 1e-6, 32)
    with pytest.raises(kf.KFError):
        F.knn()                                                 # off by default


def test_near_field_scale_recipe_lowers_the_operator_error():
    """The 6-D manifold recipe at N = 2^15 with the scale workload's
    parameters: near-field rows give IDs whose operator is closer to K than
    uniform rows' (the oracle measured 0.46 -> 0.33 at this size), and the
    sampled points' neighbour lists equal the oracle's."""
    p = inputs.scale(1 << 15)
    X = torch.from_numpy(p.X).cuda()
    tree = kf.Tree(X, p.m)
    v = torch.from_numpy(np.random.default_rng(9).standard_normal(p.N)).cuda()
    # the exact operator lambda v + K v, in FP64 on the GPU by torch (test reference only)
    ref = p.lam * v
    for i in range(0, p.N, 4096):
        d2 = torch.cdist(X[i:i + 4096], X) ** 2
        ref[i:i + 4096] += torch.exp(-0.5 * d2 / p.h**2) @ v
    errs = []
    for kappa in (0, 16):
        F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64, fp64_operator=True, knn_kappa=kappa)
        errs.append(rel(F.matvec(v).cpu().numpy(), ref.cpu().numpy()))
        if kappa:
            o = oracle.Oracle(p.X, p.m)
            nbr_o = o.knn(16, 4, 512, SEED)
            assert np.array_equal(F.knn(), nbr_o)
        del F
    assert errs[1] < 0.85 * errs[0], errs
