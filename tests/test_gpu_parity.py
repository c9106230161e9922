"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Bars (stated per test): tree permutation bit-exact; skeleton lists exact
where the pivoted QR takes the same pivots (reduction order may flip a near
tie, so agreement is counted and the factorization is also checked with the
oracle's skeletons imported); FP64 path within 1e-10 relative of the oracle;
mixed path within 1e-5 relative after refinement.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1701_02324_gb300 as kf  # noqa: E402
from paper_1701_02324_gb300 import inputs  # noqa: E402

FP64, MIXED = kf.KF_PREC_FP64, kf.KF_PREC_MIXED


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def ids_from_oracle(o, smax):
    nn = o.nnodes
    leaf_max = max(o.node_range(a)[1] - o.node_range(a)[0] for a in range(1 << o.D, 1 << (o.D + 1)))
    cmax = max(leaf_max, 2 * smax)
    ranks = np.zeros(nn + 1, np.int32)
    skel = np.zeros((nn + 1) * smax, np.int64)
    P = np.zeros((nn + 1) * smax * cmax)
    for a in range(2, nn + 1):
        s = o.rank(a)
        ranks[a] = s
        skel[a * smax: a * smax + s] = o.skel(a)
        Pa = o.P(a)
        P[a * smax * cmax: a * smax * cmax + Pa.size] = Pa.ravel()
    return ranks, skel, P


def problem(N, d, seed=0):
    rng = np.random.default_rng(seed)
    return rng.random((N, d)), rng.standard_normal(N)


@pytest.fixture(scope="module")
def c1():
    p = inputs.plain_fp64()
    o = oracle.Oracle(p.X, p.m)
    o.skeletonize(p.h, p.tau, p.s_max)
    o.factorize(p.lam)
    tree = kf.Tree(torch.from_numpy(p.X).cuda(), p.m)
    return p, o, tree


# ---------------------------------------------------------------- tree
@pytest.mark.parametrize("N,d,m", [(4096, 8, 256), (5000, 4, 300), (777, 1, 50), (3, 2, 1), (100, 3, 1000),
                                   (65536, 8, 512), (70001, 28, 1024)])
def test_tree_permutation_bit_exact(N, d, m):
    X, _ = problem(N, d, seed=N)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    o = oracle.Oracle(X, m)
    assert tree.D == o.D
    assert np.array_equal(tree.perm().cpu().numpy(), o.perm())


def test_tree_from_float32_host_input():
    X, _ = problem(3000, 5, seed=1)
    X32 = X.astype(np.float32)
    tree = kf.Tree(torch.from_numpy(X32), 100)           # host tensor, FP32
    o = oracle.Oracle(X32.astype(np.float64), 100)
    assert np.array_equal(tree.perm().cpu().numpy(), o.perm())


# ---------------------------------------------------------------- skeletons
def test_skeletons_match_oracle(c1):
    p, o, tree = c1
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64)
    r = F.ranks()
    nodes = range(2, o.nnodes + 1)
    same_rank = sum(int(r[a]) == o.rank(a) for a in nodes)
    same = sum(np.array_equal(F.skeleton(a), o.skel(a)) for a in nodes)
    assert same_rank == len(nodes)
    assert same == len(nodes)
    for a in nodes:
        np.testing.assert_allclose(F.P(a, o.ncols(a)), o.P(a), rtol=0, atol=1e-9 * max(1, np.abs(o.P(a)).max()))


# ---------------------------------------------------------------- factorization and solve
def test_fp64_solve_end_to_end(c1):
    p, o, tree = c1
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64)
    b = p.B[:, 0]
    x, info = F.solve(torch.from_numpy(b).cuda(), info=True)
    assert rel(x.cpu().numpy(), o.solve(b)) <= 1e-10
    assert info["eps_r"] <= 1e-10


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-5)])
def test_factorization_with_oracle_ids(c1, prec, tol):
    p, o, tree = c1
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=prec)
    for a in range(2, o.nnodes + 1):
        lo, hi = o.node_range(a)
        Po = o.Phat(a)
        ptol = 1e-10 if prec == FP64 else 1e-4
        assert np.abs(F.Phat(a, hi - lo) - Po).max() <= ptol * max(1.0, np.abs(Po).max())
    b = p.B[:, 0]
    x = F.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert rel(x, o.solve(b)) <= tol


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-5)])
def test_cluster_and_single_cta_kernels_agree(c1, prec, tol):
    """The upper levels run the pivoted QR and the reduced-system LU on CTA
    clusters; one CTA per node everywhere must give the same skeletons and,
    with the oracle's skeletons imported, the same solution."""
    p, o, tree = c1
    Fa = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64)
    Fb = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64, cluster_kernels=False)
    assert np.array_equal(Fa.ranks(), Fb.ranks())
    for a in range(2, o.nnodes + 1):
        assert np.array_equal(Fa.skeleton(a), Fb.skeleton(a))
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    b = p.B[:, 0]
    xo = o.solve(b)
    for cl in (True, False):
        F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=prec, cluster_kernels=cl)
        assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), xo) <= tol


@pytest.mark.parametrize("h,N,m", [(0.5, 4096, 256), (2.0, 4096, 256), (0.5, 5000, 300)])
def test_fp64_operator_matches_oracle_matvec(h, N, m):
    """The FP64-accurate operator of the mixed path (V blocks and leaf blocks
    in double-float arithmetic with a table-driven exponential, FP32 for the
    entries below 2^-24) against the oracle's FP64 matvec, same skeletons.
    h = 0.5 on [0,1]^8 puts the exponent arguments over [-16, 0]; N = 5000
    gives ragged leaves (312 and 313 points: a partial 64 x 64 tile)."""
    X, _ = problem(N, 8, seed=11)
    o = oracle.Oracle(X, m)
    o.skeletonize(h, 1e-6, 64)
    o.factorize(1.0)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    ranks, skel, P = ids_from_oracle(o, 64)
    F = kf.factorize_with_ids(tree, h, 1.0, 64, ranks, skel, P, precision=MIXED, fp64_operator=True)
    x = np.random.default_rng(12).standard_normal(N)
    y = F.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, o.matvec(x)) <= 1e-13


def test_cluster_kernels_medium_tree():
    """N = 65,536 with 512-point leaves (D = 7) puts 64, 32 and 16 nodes on the
    upper levels, i.e. LU clusters of 2, 4 and 8 CTAs and the cluster QR on
    levels of 64 nodes and fewer.  The skeletons and the FP64 solution must not
    depend on whether those kernels or one CTA per node run."""
    X, b = problem(65536, 8, seed=21)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 512)
    Fa = kf.Factor(tree, 0.4, 0.5, 1e-5, 64, precision=FP64)
    Fb = kf.Factor(tree, 0.4, 0.5, 1e-5, 64, precision=FP64, cluster_kernels=False)
    ra, rb = Fa.ranks(), Fb.ranks()
    assert np.array_equal(ra, rb)
    for a in range(2, 256):
        assert np.array_equal(Fa.skeleton(a), Fb.skeleton(a))
    bt = torch.from_numpy(b).cuda()
    xa, xb = Fa.solve(bt).cpu().numpy(), Fb.solve(bt).cpu().numpy()
    assert rel(xa, xb) <= 1e-10


def test_tc_tile_width_128(c1):
    """The tcgen05 products with 128-column tiles (the autotuner's other tile
    width) against the oracle, with the oracle's skeletons imported."""
    p, o, tree = c1
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=MIXED, tc_tile_n=128)
    b = p.B[:, 0]
    assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-5
    with pytest.raises(kf.KFError):
        kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED, tc_tile_n=64)


def test_autotune_picks_a_candidate_that_solves(c1):
    """kf_autotune times the kernel variants (cluster kernels, tcgen05 or CUDA-
    core products, tile width) and returns the fastest; the chosen options give
    the same skeletons and a solution within the mixed tolerance."""
    p, o, tree = c1
    chosen, ms = kf.autotune(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED)
    assert len(ms) == 6 and all(t > 0 for t in ms)
    assert chosen["tc_tile_n"] in (0, 128, 256)
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED, **chosen)
    F0 = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED)
    assert np.array_equal(F.ranks(), F0.ranks())
    b = p.B[:, 0]
    assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-5
    chosen64, ms64 = kf.autotune(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64)
    assert len(ms64) == 2


def test_matvec_transpose_and_grad_parity(c1):
    p, o, tree = c1
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=FP64)
    b = p.B[:, 0]
    bt = torch.from_numpy(b).cuda()
    assert rel(F.matvec(bt).cpu().numpy(), o.matvec(b)) <= 1e-12
    assert rel(F.solve(bt, transpose=True).cpu().numpy(), o.solve(b, transpose=True)) <= 1e-10
    xo = o.solve(b)
    y = np.random.default_rng(5).standard_normal(p.N)
    g = 2 * (xo - y)
    db, dl, dh = F.grad(torch.from_numpy(xo).cuda(), torch.from_numpy(g).cuda())
    dbo, dlo, dho = o.grad(xo, g)
    assert rel(db.cpu().numpy(), dbo) <= 1e-10
    assert abs(dl - dlo) <= 1e-10 * abs(dlo)
    assert abs(dh - dho) <= 1e-9 * abs(dho)


@pytest.mark.parametrize("prec,extra", [(MIXED, {"refine_tol": 1e-13}),
                                         (FP64, {"refine_tol": 1e-13, "refine_max_iter": 20, "fp64_operator": True})])
def test_refined_transpose_solve_and_gradient(c1, prec, extra):
    """Transpose solves and the adjoint of kf_grad are refined like forward
    solves: GMRES on the transpose system against the transposed operator
    (double-float V and leaf blocks on the mixed path, FP64 on the FP64 path),
    preconditioned by the transpose sweep; both reach the oracle's transpose
    solve and gradient of the same K~.  dL/dh sums terms about 4,600 times
    larger than itself here, so it gets 1e-7."""
    p, o, tree = c1
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=prec, **extra)
    b = p.B[:, 0]
    xt, info = F.solve(torch.from_numpy(b).cuda(), transpose=True, info=True)
    assert info["eps_r"] <= extra["refine_tol"]
    assert rel(xt.cpu().numpy(), o.solve(b, transpose=True)) <= 1e-10
    xo = o.solve(b)
    y = np.random.default_rng(5).standard_normal(p.N)
    g = 2 * (xo - y)
    db, dl, dh = F.grad(torch.from_numpy(xo).cuda(), torch.from_numpy(g).cuda())
    dbo, dlo, dho = o.grad(xo, g)
    assert rel(db.cpu().numpy(), dbo) <= 1e-10
    assert abs(dl - dlo) <= 1e-10 * abs(dlo)
    assert abs(dh - dho) <= 1e-7 * abs(dho)


def test_transposed_operator_ragged_leaves():
    """The transposed FP64-accurate operator on ragged leaves (N = 5000, 312
    and 313 points): the refined transpose solve against the oracle's."""
    X, b = problem(5000, 8, seed=11)
    o = oracle.Oracle(X, 300)
    o.skeletonize(0.5, 1e-6, 64)
    o.factorize(1.0)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 300)
    ranks, skel, P = ids_from_oracle(o, 64)
    F = kf.factorize_with_ids(tree, 0.5, 1.0, 64, ranks, skel, P, precision=MIXED, refine_tol=1e-13)
    xt = F.solve(torch.from_numpy(b).cuda(), transpose=True).cpu().numpy()
    assert rel(xt, o.solve(b, transpose=True)) <= 1e-10


@pytest.mark.parametrize("zn", [-1, 1, 4, 64])
def test_reduced_system_inverse_levels(c1, zn):
    """The sweeps solve the reduced systems of the levels with at most
    zinv_max_nodes nodes by their explicit inverse (formed after each level's
    LU) and the others by the LU: every split gives the oracle's forward and
    transpose solutions (direct sweeps; FP32 factors on the mixed path)."""
    p, o, tree = c1
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    b = p.B[:, 0]
    bt = torch.from_numpy(b).cuda()
    xo, xto = o.solve(b), o.solve(b, transpose=True)
    for prec, tol in ((FP64, 1e-10), (MIXED, 1e-4)):
        F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=prec, refine_max_iter=-1,
                                  zinv_max_nodes=zn)
        assert rel(F.solve(bt).cpu().numpy(), xo) <= tol
        assert rel(F.solve(bt, transpose=True).cpu().numpy(), xto) <= tol


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-4)])
def test_v_recompute_matches_oracle(c1, prec, tol):
    """KF_V_RECOMPUTE: the solve sweeps and the operator evaluate the V blocks
    K(x_i, sib~) on the fly (matrix-free, Sec. II-D) instead of reading the
    stored ones: forward and transpose solutions (direct sweeps; FP32 factors
    on the mixed path) and, on the FP64 path, the operator equal the oracle's."""
    p, o, tree = c1
    ranks, skel, P = ids_from_oracle(o, p.s_max)
    F = kf.factorize_with_ids(tree, p.h, p.lam, p.s_max, ranks, skel, P, precision=prec, refine_max_iter=-1,
                              v_storage=kf.KF_V_RECOMPUTE, fp64_operator=False)
    b = p.B[:, 0]
    bt = torch.from_numpy(b).cuda()
    assert rel(F.solve(bt).cpu().numpy(), o.solve(b)) <= tol
    assert rel(F.solve(bt, transpose=True).cpu().numpy(), o.solve(b, transpose=True)) <= tol
    if prec == FP64:
        assert rel(F.matvec(bt).cpu().numpy(), o.matvec(b)) <= 1e-12


def test_multiple_rhs_and_float32(c1):
    p, o, tree = c1
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64)
    B = np.random.default_rng(2).standard_normal((p.N, 5))
    X = F.solve(torch.from_numpy(B).cuda()).cpu().numpy()
    Xo = o.solve(B)
    assert rel(X, Xo) <= 1e-10
    X32 = F.solve(torch.from_numpy(B.astype(np.float32))).numpy()   # host FP32 in and out
    assert rel(X32, Xo) <= 1e-6


def test_mixed_path_refined(c1):
    """Mixed path (FP32 factors, tcgen05 products) refined by GMRES against the
    FP64 operator: reaches the oracle's solution of the same K~."""
    p, o, tree = c1
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED, refine_tol=1e-12)
    b = p.B[:, 0]
    x, info = F.solve(torch.from_numpy(b).cuda(), info=True)
    same = all(np.array_equal(F.skeleton(a), o.skel(a)) for a in range(2, o.nnodes + 1))
    assert same
    assert rel(x.cpu().numpy(), o.solve(b)) <= 1e-10
    assert info["eps_r"] <= 1e-12
    # without refinement the FP32 factorization alone is within the mixed bar
    F0 = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED, refine_max_iter=-1, tensor_cores=False)
    assert rel(F0.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-5


def test_mixed_richardson_and_fp64_refinement(c1):
    p, o, tree = c1
    b = p.B[:, 0]
    xo = o.solve(b)
    F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=MIXED, gmres_restart=-1, refine_tol=1e-12)
    assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), xo) <= 1e-10
    # the FP64-accurate operator holds its entries as double-float pairs
    # (about 2^-46 relative), so the refined residual floor is a few 1e-14
    F64 = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64, refine_max_iter=5, refine_tol=5e-14,
                    fp64_operator=True)
    x64, info = F64.solve(torch.from_numpy(b).cuda(), info=True)
    assert rel(x64.cpu().numpy(), xo) <= 1e-12 and info["eps_r"] <= 5e-14


# ---------------------------------------------------------------- edge cases
def test_single_leaf_is_dense_solve():
    X, b = problem(300, 2, seed=4)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 400)
    assert tree.D == 0
    F = kf.Factor(tree, 0.5, 1.0, 1e-6, 16)
    o = oracle.Oracle(X, 400)
    o.skeletonize(0.5, 1e-6, 16)
    o.factorize(1.0)
    assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-12


def test_ragged_sizes():
    X, b = problem(5000, 4, seed=6)
    o = oracle.Oracle(X, 300)
    o.skeletonize(0.4, 1e-5, 48)
    o.factorize(0.5)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 300)
    ranks, skel, P = ids_from_oracle(o, 48)
    F = kf.factorize_with_ids(tree, 0.4, 0.5, 48, ranks, skel, P)
    assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-10


def test_maximum_rank_s_max_512():
    """The largest rank the library takes (s_max = 512, |S'| = 1024): N = 2048
    points in [0,1]^8 with h = 0.3 keep every rank at its cap (full-rank leaves
    of 512 points, z = 1024 reduced systems above), which drives the QR with 32
    rows per lane, 1024 x 1024 reduced systems, their explicit inverse at the
    root and 512-column tcgen05 products.  Skeletons equal the oracle's; FP64
    direct solve and mixed solve refined to 1e-12 within 1e-10 of the oracle,
    forward and transpose."""
    X = np.random.default_rng(31).random((2048, 8))
    b = np.random.default_rng(32).standard_normal(2048)
    h, lam, tau, smax = 0.3, 0.5, 1e-12, 512
    o = oracle.Oracle(X, 512)
    o.skeletonize(h, tau, smax)
    o.factorize(lam)
    xo, xto = o.solve(b), o.solve(b, transpose=True)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 512)
    bt = torch.from_numpy(b).cuda()
    for prec, kw in ((FP64, {}), (MIXED, {"refine_tol": 1e-12})):
        F = kf.Factor(tree, h, lam, tau, smax, precision=prec, **kw)
        r = F.ranks()
        assert all(int(r[a]) == o.rank(a) == 512 for a in range(2, o.nnodes + 1))
        assert all(np.array_equal(F.skeleton(a), o.skel(a)) for a in range(2, o.nnodes + 1))
        assert rel(F.solve(bt).cpu().numpy(), xo) <= 1e-10
        assert rel(F.solve(bt, transpose=True).cpu().numpy(), xto) <= 1e-10


def test_empty_inputs_rejected_and_duplicate_points():
    """Empty inputs are rejected with KF_EINVAL (no points, no coordinates,
    m = 0, no right-hand side); heavily duplicated points (9 distinct
    positions among 1500: ties in every distance and projection, broken by the
    original index) still give the oracle's tree bit for bit."""
    dev = "cuda"
    for X, m in ((torch.zeros((0, 3), dtype=torch.float64, device=dev), 8),
                 (torch.zeros((10, 0), dtype=torch.float64, device=dev), 8),
                 (torch.rand((10, 3), dtype=torch.float64, device=dev), 0)):
        with pytest.raises(kf.KFError) as e:
            kf.Tree(X, m)
        assert e.value.status == kf._abi.KF_EINVAL
    X = np.random.default_rng(41).integers(0, 3, size=(1500, 2)).astype(np.float64)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 64)
    o = oracle.Oracle(X, 64)
    assert np.array_equal(tree.perm().cpu().numpy(), o.perm())
    F = kf.Factor(tree, 0.7, 1.0, 1e-8, 16)
    b = torch.zeros(1500, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    lib = kf._abi.load()
    assert lib.kf_solve(F.h, b.data_ptr(), x.data_ptr(), 0, 1500, kf.KF_F64, 0, None, None) == kf._abi.KF_EINVAL


def test_small_h_limit_is_diagonal():
    X, b = problem(2048, 3, seed=7)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 128)
    F = kf.Factor(tree, 1e-4, 0.5, 1e-6, 32)
    assert int(F.ranks().max()) == 0
    np.testing.assert_allclose(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), b / 1.5, rtol=1e-15, atol=0)


def test_large_h_limit_is_rank_one():
    X, b = problem(2048, 3, seed=8)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 128)
    lam = 2.0
    F = kf.Factor(tree, 1e10, lam, 1e-8, 32)
    r = F.ranks()
    assert (r[2:] == 1).all()
    xref = (b - b.sum() / (lam + 2048)) / lam
    assert rel(F.solve(torch.from_numpy(b).cuda()).cpu().numpy(), xref) <= 1e-12


def test_illconditioned_reported():
    X, _ = problem(512, 3, seed=9)
    X[1] = X[0]
    tree = kf.Tree(torch.from_numpy(X).cuda(), 64)
    F = kf.Factor(tree, 0.5, 0.0, 1e-6, 16)
    assert F.status == kf._abi.KF_EILLCOND


def test_invalid_arguments_rejected():
    X, _ = problem(100, 2, seed=10)
    Xbad = X.copy()
    Xbad[3, 1] = np.nan
    with pytest.raises(kf.KFError) as e:
        kf.Tree(torch.from_numpy(Xbad).cuda(), 10)
    assert e.value.status == kf._abi.KF_EINVAL
    tree = kf.Tree(torch.from_numpy(X).cuda(), 10)
    for h, lam, smax in [(0.0, 1.0, 8), (-1.0, 1.0, 8), (0.5, -1.0, 8), (0.5, 1.0, 0), (0.5, 1.0, 4096)]:
        with pytest.raises(kf.KFError) as e:
            kf.Factor(tree, h, lam, 1e-6, smax)
        assert e.value.status == kf._abi.KF_EINVAL


# ---------------------------------------------------------------- many problems, one graph launch
def test_batched_matches_single_and_oracle():
    """Row a12: uneven problems factorized and solved with one CUDA-graph launch
    each; every problem equals its own single factorization and the oracle."""
    ctx = kf.Context(use_torch_allocator=False)
    rng = np.random.default_rng(11)
    Ns = [2048, 3001, 4096, 2500, 6000, 2222]
    hs = [0.3 + 0.1 * i for i in range(len(Ns))]
    Xs = [rng.random((n, 8)) for n in Ns]
    Bs = [rng.standard_normal((n, 3)) for n in Ns]
    trees = [kf.Tree(torch.from_numpy(X).cuda(), 256, ctx=ctx) for X in Xs]
    o = oracle.Oracle(Xs[1], 256)
    o.skeletonize(hs[1], 1e-5, 64)
    o.factorize(0.5)
    # FP64 direct sweeps; mixed sweeps without refinement (refine_max_iter = -1)
    # and with the batch refined as a whole (the mixed path's default)
    for prec, rmi, tol_single, tol_oracle in ((FP64, 0, 1e-10, 1e-10), (MIXED, -1, 1e-5, 1e-4),
                                              (MIXED, 0, 1e-8, 1e-8)):
        facs = kf.factorize_batched(trees, hs, [0.5] * len(Ns), [1e-5] * len(Ns), 64, precision=prec,
                                    refine_max_iter=rmi)
        xs = kf.solve_batched(facs, [torch.from_numpy(B).cuda() for B in Bs])
        for i in (0, 4):
            single = kf.Factor(trees[i], hs[i], 0.5, 1e-5, 64, precision=prec, refine_max_iter=rmi)
            xi = single.solve(torch.from_numpy(Bs[i]).cuda()).cpu().numpy()
            assert rel(xs[i].cpu().numpy(), xi) <= tol_single
        assert rel(xs[1].cpu().numpy(), o.solve(Bs[1])) <= tol_oracle


def test_autograd_kernel_solve_matches_oracle_gradient():
    """Row a11: torch.autograd through x = (lambda I + K~(h))^-1 b gives dL/db,
    dL/dlambda and dL/dh equal to the oracle's adjoint (skeletons fixed)."""
    X, b = problem(2048, 3, seed=21)
    y = np.random.default_rng(22).standard_normal(2048)
    h, lam = 0.3, 0.8
    tree = kf.Tree(torch.from_numpy(X).cuda(), 128)
    F = kf.Factor(tree, h, lam, 1e-7, 48, precision=FP64)
    o = oracle.Oracle(X, 128)
    o.skeletonize(h, 1e-7, 48)
    o.factorize(lam)
    assert all(np.array_equal(F.skeleton(a), o.skel(a)) for a in range(2, o.nnodes + 1))
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    lt = torch.tensor(lam, device="cuda", dtype=torch.float64, requires_grad=True)
    ht = torch.tensor(h, device="cuda", dtype=torch.float64, requires_grad=True)
    x = kf.KernelSolve.apply(bt, lt, ht, F)
    loss = ((x - torch.from_numpy(y).cuda()) ** 2).sum()
    loss.backward()
    xo = o.solve(b)
    dbo, dlo, dho = o.grad(xo, 2 * (xo - y))
    assert rel(bt.grad.cpu().numpy(), dbo) <= 1e-10
    assert abs(lt.grad.item() - dlo) <= 1e-9 * abs(dlo)
    assert abs(ht.grad.item() - dho) <= 1e-8 * abs(dho)


def test_autograd_kernel_solve_rejects_other_lambda_or_h():
    """KernelSolve solves with the factorization's own lambda and h, so a
    lambda or h that differs from them is an error rather than a stale solve
    whose backward would report gradients at the values passed in."""
    X, b = problem(1024, 3, seed=23)
    tree = kf.Tree(torch.from_numpy(X).cuda(), 128)
    F = kf.Factor(tree, 0.4, 0.9, 1e-7, 32, precision=FP64)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    f64 = dict(device="cuda", dtype=torch.float64)
    x = kf.KernelSolve.apply(bt, torch.tensor(0.9, **f64), torch.tensor(0.4, **f64), F)
    assert x.shape == bt.shape
    for lam, h in ((0.91, 0.4), (0.9, 0.41)):
        with pytest.raises(ValueError):
            kf.KernelSolve.apply(bt, torch.tensor(lam, **f64), torch.tensor(h, **f64), F)


# ---------------------------------------------------------------- profiler
def test_profile_totals_and_timeline(c1):
    """kf_profile_read totals and kf_profile_timeline records of one
    factorization: every launch recorded once, in order of issue per stream,
    with its phase; the per-phase sums of the timeline equal the totals."""
    import ctypes
    from paper_1701_02324_gb300 import _abi
    p, _, tree = c1
    lib = _abi.load()
    nph = len(_abi.PHASES)
    ms = np.zeros(nph)
    ln = np.zeros(nph, dtype=np.int64)
    torch.cuda.synchronize()
    assert lib.kf_profile_enable(1) == 0
    try:
        lib.kf_profile_read(ms.ctypes.data, ln.ctypes.data, nph)  # clears earlier records
        F = kf.Factor(tree, p.h, p.lam, p.tau, p.s_max, precision=FP64)
        F.solve(torch.from_numpy(p.B[:, 0]).cuda())
        torch.cuda.synchronize()
        cap = 4096
        t0, t1 = np.zeros(cap), np.zeros(cap)
        ph, st = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
        n = ctypes.c_int64(0)
        assert lib.kf_profile_timeline(t0.ctypes.data, t1.ctypes.data, ph.ctypes.data, st.ctypes.data, cap,
                                       ctypes.byref(n)) == 0
        k = n.value
        assert 0 < k <= cap
        t0, t1, ph, st = t0[:k], t1[:k], ph[:k], st[:k]
        assert t0[0] == 0.0 and np.all(t1 >= t0) and np.all(t0 >= 0.0)
        assert np.all((ph >= 0) & (ph < nph)) and st.min() == 0
        for s in np.unique(st):  # launches of one stream run in issue order
            a, b = t0[st == s], t1[st == s]
            assert np.all(a[1:] >= b[:-1] - 1e-3)
        assert lib.kf_profile_read(ms.ctypes.data, ln.ctypes.data, nph) == 0
        assert int(ln.sum()) == k
        for q in range(nph):
            assert ln[q] == int(np.sum(ph == q))
            # event timestamps resolve about 0.5 us: allow 2 us per launch
            assert abs(ms[q] - float(np.sum((t1 - t0)[ph == q]))) <= 2e-3 * ln[q] + 1e-3 * ms[q]
        bad = ctypes.c_int64(0)
        assert lib.kf_profile_timeline(None, None, None, None, 0, ctypes.byref(bad)) == _abi.KF_EINVAL
    finally:
        lib.kf_profile_enable(0)


@pytest.mark.parametrize("N,d,m,smax", [(3001, 5, 300, 48), (4096, 8, 1024, 64), (2200, 3, 140, 32)])
def test_leaf_factorization_on_tensor_cores(N, d, m, smax):
    """Row a4 on the mixed path: the leaves' Cholesky factors by 128-column
    panels (diagonal block and its inverse on CUDA cores, panel rows and
    trailing updates as tcgen05 3xTF32 products) and P^ = A^-1 P by panel
    products with those inverses, against the oracle's FP64 P^ of every leaf
    (LU of lambda I + K_aa) at FP32 accuracy scaled by cond(A): ragged leaves of
    1, 2 and 8 panels.  The pivot ratios agree with the CUDA-core kernels'."""
    rng = np.random.default_rng(N)
    X = rng.random((N, d))
    h, lam, tau = 0.4, 0.5, 1e-6
    o = oracle.Oracle(X, m)
    o.skeletonize(h, tau, smax)
    o.factorize(lam)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    Ft = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, refine_max_iter=-1)
    Fc = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, refine_max_iter=-1, tensor_cores=False)
    Xt = X[o.perm()]
    for a in range(1 << o.D, 1 << (o.D + 1)):
        lo, hi = o.node_range(a)
        Y = Xt[lo:hi]
        A = lam * np.eye(hi - lo) + np.exp(-0.5 * ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1) / h**2)
        cond = np.linalg.cond(A)
        ref = o.Phat(a)
        if ref.size == 0:
            continue
        assert rel(Ft.Phat(a, hi - lo), ref) <= 2e-7 * cond, a
        assert rel(Fc.Phat(a, hi - lo), ref) <= 2e-7 * cond, a
    pt, pc = Ft.pivot_ratios(), Fc.pivot_ratios()
    leaves = slice(1 << o.D, 1 << (o.D + 1))
    assert np.allclose(pt[leaves], pc[leaves], rtol=1e-3)
    b = rng.standard_normal(N)
    G = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, refine_tol=1e-11)
    assert rel(G.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-8


@pytest.mark.parametrize("N,d,m,smax,h", [(4096, 8, 256, 64, 0.5), (3001, 5, 100, 32, 0.35)])
def test_fused_z_blocks_match_stored_v(N, d, m, smax, h):
    """Row a5 on the mixed path, kf_opts.zoff_fused = 1: the reduced systems'
    off-diagonal blocks K_{l~ r} P^_r with the kernel entries evaluated inside
    the tcgen05 product against the default product that reads the stored V
    blocks: P^ of every internal node within 1e-4 (the fused entries carry
    ~1e-6 relative error: FP32 squared distances of the FP32 coordinates); the
    fused factors refined by GMRES solve within 1e-8 of the oracle."""
    rng = np.random.default_rng(N + 5)
    X, b = rng.random((N, d)), rng.standard_normal(N)
    lam, tau = 0.7, 1e-6
    o = oracle.Oracle(X, m)
    o.skeletonize(h, tau, smax)
    o.factorize(lam)
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    Ff = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, refine_max_iter=-1, zoff_fused=True)
    Fv = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, refine_max_iter=-1)
    for a in range(2, 1 << o.D):
        lo, hi = o.node_range(a)
        pf, pv = Ff.Phat(a, hi - lo), Fv.Phat(a, hi - lo)
        if pv.size == 0:
            continue
        assert rel(pf, pv) <= 1e-4, a
    G = kf.Factor(tree, h, lam, tau, smax, precision=MIXED, refine_tol=1e-11, zoff_fused=True)
    assert rel(G.solve(torch.from_numpy(b).cuda()).cpu().numpy(), o.solve(b)) <= 1e-8


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_results_are_bitwise_deterministic(prec):
    """Two factorizations of the same problem and two runs of every solve give
    the same bits: the split-K partial sums of the Z blocks, the segmented
    column sums of the sweep and the operator, and the refinement's norms and
    dot products are all added in a fixed order (no floating-point atomics).
    N = 2^15 so that the upper levels split their Z-block products over K."""
    rng = np.random.default_rng(77)
    N, d, m, smax, h, lam = 1 << 15, 6, 256, 64, 0.5, 0.7
    X = rng.random((N, d))
    B = torch.from_numpy(rng.standard_normal((N, 4))).cuda()
    tree = kf.Tree(torch.from_numpy(X).cuda(), m)
    kw = dict(precision=prec, fp64_operator=True, refine_tol=1e-11, refine_max_iter=60, gmres_restart=20)
    F1 = kf.Factor(tree, h, lam, 1e-6, smax, **kw)
    F2 = kf.Factor(tree, h, lam, 1e-6, smax, **kw)
    r = F1.ranks()
    for a in (2, 3, 5, 9, 17, 40):
        if r[a] == 0:
            continue
        rows = _node_rows(tree, a)
        assert np.array_equal(F1.Phat(a, rows), F2.Phat(a, rows)), a
    x1, i1 = F1.solve(B, info=True)
    x2, i2 = F2.solve(B, info=True)
    assert torch.equal(x1, x2) and i1 == i2
    assert torch.equal(F1.solve(B), F1.solve(B))
    assert torch.equal(F1.matvec(B), F2.matvec(B))
    assert torch.equal(F1.solve(B, transpose=True), F2.solve(B, transpose=True))


def _node_rows(tree, a):
    """Number of points of node a (the tree's median split: sizes follow from N)."""
    lvl = int(np.floor(np.log2(a)))
    sizes = [tree.N]
    for _ in range(lvl):
        sizes = [s for n in sizes for s in (n // 2, n - n // 2)]
    return sizes[a - (1 << lvl)]
