"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test ties one oracle function to something other than itself: a library
routine (scipy Cholesky, LAPACK pivoted QR), a closed form (the h -> 0 and
h -> infinity limits of Eq. e:gaussian, Sherman-Morrison), an algebraic
identity (Eq. e:smw, the push-through form of Eq. e:invtelescope), the paper's
statement that the N log N and N log^2 N factorizations agree up to roundoff
(Sec. V, Table 2 discussion), a known-answer vector (splitmix64), or finite
differences (gradients).  A plausible slip in the oracle (dropped term, wrong
sign or index, transposed operand) fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import Oracle, splitmix64, KFO_EILLCOND, KFO_OK

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def gauss_K(X, Y, h):
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    return np.exp(-0.5 * d2 / h**2)


def make(N=512, d=3, m=64, seed=0):
    rng = np.random.default_rng(seed)
    return rng.random((N, d)), rng


# ---------------------------------------------------------------- sampler
def test_splitmix64_known_answer(golden_dir):
    vals = [int(l) for l in open(os.path.join(golden_dir, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    G = 0x9E3779B97F4A7C15
    got = [splitmix64((1234567 + k * G) & (2**64 - 1)) for k in range(5)]
    assert got == vals


def test_sample_properties():
    X, _ = make(N=1000, m=100)
    o = Oracle(X, 100)
    for a in range(2, o.nnodes + 1):
        lo, hi = o.node_range(a)
        S = o.sample(a, 64, 0x1701)
        assert len(S) == min(1000 - (hi - lo), 64)
        assert np.all(np.diff(S) > 0)                      # sorted, distinct
        assert not np.any((S >= lo) & (S < hi))            # outside the node
        assert S.min() >= 0 and S.max() < 1000
    # whole complement when the cap exceeds it
    S = o.sample(2, 10**6, 1)
    lo, hi = o.node_range(2)
    assert np.array_equal(S, np.r_[0:lo, hi:1000])


def test_sample_matches_definition():
    """Brute force restatement of the counter-based draw for one node."""
    X, _ = make(N=300, m=40)
    o = Oracle(X, 40)
    a = 5
    lo, hi = o.node_range(a)
    M = 300 - (hi - lo)
    got, j = [], 0
    while len(got) < 20:
        u = splitmix64(0x1701 ^ (a << 32) ^ j)
        c = u % M
        if c not in got:
            got.append(c)
        j += 1
    ref = sorted(c if c < lo else c + (hi - lo) for c in got)
    assert np.array_equal(o.sample(a, 20, 0x1701), ref)


# ---------------------------------------------------------------- tree
def test_tree_split_rule_bruteforce():
    X, _ = make(N=777, d=4, m=50, seed=3)
    o = Oracle(X, 50)
    assert o.D == int(np.ceil(np.log2(777 / 50)))
    perm = o.perm()
    assert np.array_equal(np.sort(perm), np.arange(777))
    # independent restatement of the split for every internal node
    order = np.arange(777)
    nodes = {1: order}
    for a in range(1, 1 << o.D):
        idx = nodes[a]
        lo, hi = o.node_range(a)
        assert hi - lo == len(idx)
        pts = X[idx]
        ia = np.argmin(idx)
        da = ((pts - pts[ia]) ** 2).sum(1)
        ip = min(np.flatnonzero(da == da.max()), key=lambda i: idx[i])
        dp = ((pts - pts[ip]) ** 2).sum(1)
        iq = min(np.flatnonzero(dp == dp.max()), key=lambda i: idx[i])
        proj = (pts - pts[ip]) @ (pts[iq] - pts[ip])
        srt = np.lexsort((idx, proj))
        nl = len(idx) // 2
        nodes[2 * a], nodes[2 * a + 1] = idx[srt[:nl]], idx[srt[nl:]]
    for a in range(1 << o.D, 1 << (o.D + 1)):
        lo, hi = o.node_range(a)
        assert np.array_equal(perm[lo:hi], nodes[a])


def test_tree_sizes_floor_ceil():
    X, _ = make(N=1001, m=60)
    o = Oracle(X, 60)
    for a in range(1, 1 << o.D):
        lo, hi = o.node_range(a)
        llo, lhi = o.node_range(2 * a)
        rlo, rhi = o.node_range(2 * a + 1)
        assert (llo, rhi, lhi) == (lo, hi, rlo)
        assert lhi - llo == (hi - lo) // 2


# ---------------------------------------------------------------- ID
def test_id_against_lapack_pivoted_qr():
    """The leaf ID equals LAPACK's column-pivoted QR (GEQP3) on K_{S' alpha}:
    same pivots, rank from the |R_kk| < tau |R_00| rule, P = [I, R11^-1 R12]."""
    X, _ = make(N=512, d=3, m=64, seed=5)
    o = Oracle(X, 64)
    h, tau, smax = 0.3, 1e-5, 40
    o.skeletonize(h, tau, smax, n_samp=80)
    Xt = X[o.perm()]
    for a in (8, 13):
        lo, hi = o.node_range(a)
        S = o.sample(a, 80, 0x1701)
        A = gauss_K(Xt[S], Xt[lo:hi], h)
        Q, R, piv = sla.qr(A, pivoting=True, mode="economic")
        dg = np.abs(np.diag(R))
        cut = np.flatnonzero(dg < tau * dg[0])
        s = min(cut[0] if len(cut) else len(dg), smax)
        assert o.rank(a) == s
        assert np.array_equal(o.skel(a), lo + piv[:s])
        T = sla.solve_triangular(R[:s, :s], R[:s, s:])
        Pref = np.zeros((s, hi - lo))
        Pref[:, piv[:s]] = np.eye(s)
        Pref[:, piv[s:]] = T
        np.testing.assert_allclose(o.P(a), Pref, atol=1e-9 * max(1, np.abs(Pref).max()))


def test_id_interpolates_sample_rows():
    X, _ = make(N=512, d=3, m=64, seed=6)
    o = Oracle(X, 64)
    h, tau = 0.4, 1e-6
    o.skeletonize(h, tau, 48, n_samp=96)
    Xt = X[o.perm()]
    for a in range(2, o.nnodes + 1):
        S = o.sample(a, 96, 0x1701)
        if o.is_leaf(a):
            lo, hi = o.node_range(a)
            cols = np.arange(lo, hi)
        else:
            cols = np.r_[o.skel(2 * a), o.skel(2 * a + 1)]
        A = gauss_K(Xt[S], Xt[cols], h)
        sk = o.skel(a)
        P = o.P(a)
        s, c = P.shape
        # skeleton columns are reproduced exactly (identity block of P)
        pos = [int(np.flatnonzero(cols == k)[0]) for k in sk]
        np.testing.assert_array_equal(P[:, pos], np.eye(s))
        # residual bound of a rank-revealing QR, loose constant
        Ak = gauss_K(Xt[S], Xt[sk], h)
        err = np.linalg.norm(A - Ak @ P, 2)
        if s < min(48, c, len(S)):
            assert err <= np.sqrt(s * (c - s) + 1) * 10 * tau * np.linalg.norm(A, 2)


# ---------------------------------------------------------------- factorization / solve
def test_full_rank_equals_dense_cholesky():
    """tau = 0, s_max >= N/2 and S' = the whole complement: every ID keeps all
    columns, K~ = K, and the solve equals scipy's dense Cholesky solve."""
    X, rng = make(N=1024, d=4, m=128, seed=7)
    o = Oracle(X, 128)
    o.skeletonize(0.35, 0.0, 1024, n_samp=1024)
    assert o.factorize(1.0) == KFO_OK
    b = rng.standard_normal(1024)
    x = o.solve(b)
    A = gauss_K(X, X, 0.35) + np.eye(1024)
    xd = sla.cho_solve(sla.cho_factor(A), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10


def test_operator_is_second_uv_form_and_smw_identity():
    """lambda I + K~ assembled from the oracle's matvec equals D + U V with
    U = diag(P_{l l~}, P_{r r~}), V = [[0, K_{l~ r}], [K_{r~ l}, 0]] (second form
    of Eq. e:uv, built here in numpy); W = D^-1 U; Z = I + V W; and
    (I - W Z^-1 V) D^-1 inverts it (Eq. e:smw)."""
    X, rng = make(N=64, d=2, m=8, seed=8)
    lam, h = 0.5, 0.3
    o = Oracle(X, 8)
    o.skeletonize(h, 1e-3, 6, n_samp=12)
    assert o.factorize(lam) == KFO_OK
    Xt = X[o.perm()]
    A = o.dense_Ktilde()                         # original order
    p = o.perm()
    At = A[np.ix_(p, p)]                         # tree order
    for a in range(1, o.nnodes + 1):
        if o.is_leaf(a):
            lo, hi = o.node_range(a)
            np.testing.assert_allclose(At[lo:hi, lo:hi], gauss_K(Xt[lo:hi], Xt[lo:hi], h) + lam * np.eye(hi - lo),
                                       atol=1e-13)
            continue
        lo, hi = o.node_range(a)
        l, r = 2 * a, 2 * a + 1
        (llo, lhi), (rlo, rhi) = o.node_range(l), o.node_range(r)
        nl, nr = lhi - llo, rhi - rlo
        D = np.zeros((hi - lo, hi - lo))
        D[:nl, :nl] = At[llo:lhi, llo:lhi]
        D[nl:, nl:] = At[rlo:rhi, rlo:rhi]
        sl, sr = o.rank(l), o.rank(r)
        U = np.zeros((hi - lo, sl + sr))
        U[:nl, :sl] = o.P_full(l)
        U[nl:, sl:] = o.P_full(r)
        V = np.zeros((sl + sr, hi - lo))
        V[:sl, nl:] = gauss_K(Xt[o.skel(l)], Xt[rlo:rhi], h)
        V[sl:, :nl] = gauss_K(Xt[o.skel(r)], Xt[llo:lhi], h)
        np.testing.assert_allclose(At[lo:hi, lo:hi], D + U @ V, atol=1e-12)
        W = np.zeros_like(U)
        W[:nl, :sl] = o.Phat(l)
        W[nl:, sl:] = o.Phat(r)
        np.testing.assert_allclose(W, np.linalg.solve(D, U), atol=1e-10)
        Z = o.Z(a)
        np.testing.assert_allclose(Z, np.eye(sl + sr) + V @ W, atol=1e-12)
        inv = (np.eye(hi - lo) - W @ np.linalg.solve(Z, V)) @ np.linalg.inv(D)
        np.testing.assert_allclose(inv @ (D + U @ V), np.eye(hi - lo), atol=1e-10)


def test_solve_inverts_dense_ktilde_and_residual():
    X, rng = make(N=1024, d=3, m=64, seed=9)
    o = Oracle(X, 64)
    o.skeletonize(0.2, 1e-5, 32)
    assert o.factorize(1.0) == KFO_OK
    b = rng.standard_normal(1024)
    x = o.solve(b)
    A = o.dense_Ktilde()
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-12
    # epsilon_r of Eq. (e:errors); the paper's direct solver reports 1e-10..1e-13
    assert o.residual(b, x) <= 1e-12
    xt = o.solve(b, transpose=True)
    xtd = np.linalg.solve(A.T, b)
    assert np.linalg.norm(xt - xtd) / np.linalg.norm(xtd) <= 1e-12


def test_telescoping_equals_log2_predecessor():
    """Sec. V: the N log N and N log^2 N algorithms build the same
    factorization up to roundoff."""
    X, rng = make(N=2048, d=3, m=64, seed=10)
    o1, o2 = Oracle(X, 64), Oracle(X, 64)
    for o in (o1, o2):
        o.skeletonize(0.25, 1e-6, 40)
    o1.factorize(0.7, variant=0)
    o2.factorize(0.7, variant=1)
    for a in range(2, o1.nnodes + 1):
        A1, A2 = o1.Phat(a), o2.Phat(a)
        assert np.abs(A1 - A2).max() <= 1e-11 * max(1.0, np.abs(A2).max())
    b = rng.standard_normal(2048)
    x1, x2 = o1.solve(b), o2.solve(b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) <= 1e-12


def test_push_through_identity():
    """u - W Z^-1 V u with u = W P_c equals W Z^-1 P_c, since V W = Z - I."""
    X, _ = make(N=1024, d=3, m=64, seed=11)
    o = Oracle(X, 64)
    o.skeletonize(0.25, 1e-6, 40)
    o.factorize(1.0)
    for a in range(2, 1 << o.D):
        lit, push = o.Phat_forms(a)
        assert np.abs(lit - push).max() <= 1e-12 * max(1.0, np.abs(push).max())
        np.testing.assert_allclose(o.Phat(a), lit, atol=0, rtol=0)


def test_limit_small_h_is_diagonal():
    """h -> 0: K -> I (Eq. e:gaussian); every off-diagonal entry underflows,
    every rank is 0, and x = b / (1 + lambda) exactly."""
    X, rng = make(N=512, d=3, m=64, seed=12)
    o = Oracle(X, 64)
    o.skeletonize(1e-4, 1e-6, 32)
    assert all(o.rank(a) == 0 for a in range(2, o.nnodes + 1))
    o.factorize(0.5)
    b = rng.standard_normal(512)
    np.testing.assert_array_equal(o.solve(b), b / 1.5)


def test_limit_large_h_is_rank_one():
    """h -> infinity: K -> 1 1^T (Eq. e:gaussian); every node has rank 1 and
    Sherman-Morrison gives x = (b - 1 (1^T b) / (lambda + N)) / lambda."""
    X, rng = make(N=512, d=3, m=64, seed=13)
    o = Oracle(X, 64)
    o.skeletonize(1e10, 1e-8, 32)
    assert all(o.rank(a) == 1 for a in range(2, o.nnodes + 1))
    lam = 2.0
    o.factorize(lam)
    b = rng.standard_normal(512)
    xref = (b - b.sum() / (lam + 512)) / lam
    x = o.solve(b)
    assert np.linalg.norm(x - xref) / np.linalg.norm(xref) <= 1e-12


def test_accuracy_improves_with_tau():
    X, rng = make(N=2048, d=4, m=128, seed=14)
    b = rng.standard_normal(2048)
    A = gauss_K(X, X, 0.4) + np.eye(2048)
    xd = sla.cho_solve(sla.cho_factor(A), b)
    errs = []
    for tau in (1e-2, 1e-4, 1e-6, 1e-8):
        o = Oracle(X, 128)
        o.skeletonize(0.4, tau, 2048, n_samp=2048)   # S' = S: the ID error is tau-controlled
        o.factorize(1.0)
        errs.append(np.linalg.norm(o.solve(b) - xd) / np.linalg.norm(xd))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-5


def test_illconditioned_is_detected():
    """Sec. III "Stability": a singular leaf block (duplicated points with
    lambda = 0) is reported, not silently solved."""
    X, _ = make(N=256, d=3, m=64, seed=15)
    X[1] = X[0]
    o = Oracle(X, 64)
    o.skeletonize(0.5, 1e-6, 16)
    assert o.factorize(0.0) == KFO_EILLCOND


# ---------------------------------------------------------------- gradients
def _ids(o):
    out = {}
    for a in range(2, o.nnodes + 1):
        out[a] = (o.skel(a), o.P(a))
    return out


def _with_ids(X, m, h, ids, lam):
    o = Oracle(X, m)
    o.skeletonize(h, 0.0, 1)      # sets h; IDs replaced below, children first
    for a in sorted(ids, reverse=True):
        o.set_id(a, *ids[a])
    o.factorize(lam)
    return o


def test_gradient_finite_differences():
    """dL/db, dL/dlambda and dL/dh (skeletons and P held fixed) of
    L = ||x - y||^2 with x = (lambda I + K~(h))^-1 b, against central
    differences of the oracle pipeline."""
    X, rng = make(N=512, d=3, m=64, seed=16)
    h, lam = 0.3, 0.8
    o = Oracle(X, 64)
    o.skeletonize(h, 1e-7, 40)
    ids = _ids(o)
    o.factorize(lam)
    b = rng.standard_normal(512)
    y = rng.standard_normal(512)

    def loss(oo, bb):
        x = oo.solve(bb)
        return float(((x - y) ** 2).sum())

    x = o.solve(b)
    db, dlam, dh = o.grad(x, 2 * (x - y))
    e = 1e-5
    # lambda: skeletons do not depend on lambda
    o_p = _with_ids(X, 64, h, ids, lam + e)
    o_m = _with_ids(X, 64, h, ids, lam - e)
    fd = (loss(o_p, b) - loss(o_m, b)) / (2 * e)
    assert abs(fd - dlam) <= 1e-6 * max(1, abs(fd))
    # h with fixed skeletons and P
    o_p = _with_ids(X, 64, h + e, ids, lam)
    o_m = _with_ids(X, 64, h - e, ids, lam)
    fd = (loss(o_p, b) - loss(o_m, b)) / (2 * e)
    assert abs(fd - dh) <= 1e-6 * max(1, abs(fd))
    # b: a few coordinates
    for i in (0, 100, 511):
        bp, bm = b.copy(), b.copy()
        bp[i] += e
        bm[i] -= e
        fd = (loss(o, bp) - loss(o, bm)) / (2 * e)
        assert abs(fd - db[i]) <= 1e-6 * max(1, abs(fd))


def test_gradient_close_to_dense_reference():
    """Against the dense FP64 gradient of L through (lambda I + K)^-1 b: equal
    up to the compression error (loose, tau-sized)."""
    X, rng = make(N=1024, d=3, m=64, seed=17)
    h, lam = 0.3, 1.0
    o = Oracle(X, 64)
    o.skeletonize(h, 1e-9, 1024, n_samp=1024)   # S' = S, so the error is tau-sized
    o.factorize(lam)
    b = rng.standard_normal(1024)
    y = rng.standard_normal(1024)
    x = o.solve(b)
    db, dlam, dh = o.grad(x, 2 * (x - y))
    K = gauss_K(X, X, h)
    A = K + lam * np.eye(1024)
    xd = np.linalg.solve(A, b)
    ad = np.linalg.solve(A.T, 2 * (xd - y))
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    dK = K * d2 / h**3
    assert np.linalg.norm(db - ad) / np.linalg.norm(ad) < 1e-5
    assert abs(dlam - (-ad @ xd)) / abs(ad @ xd) < 1e-5
    assert abs(dh - (-ad @ dK @ xd)) / abs(ad @ dK @ xd) < 1e-4


def test_subtrees_equal_the_whole_run():
    """kfo_subtrees (Algorithms 1 and 2 on chosen subtrees only, used to check
    sampled nodes of trees too large for a whole oracle run) gives every node
    of those subtrees bit for bit what the whole run gives it: each node's ID
    reads only its own columns and its sampled rows, each P^ only its
    descendants.  The whole run is pinned by the tests above.  Also a subtree
    root at the tree root, and overlapping roots rejected."""
    X, _ = make(N=3000, d=4, m=100, seed=14)
    whole, part = Oracle(X, 100), Oracle(X, 100)
    whole.skeletonize(0.4, 1e-6, 24)
    assert whole.factorize(0.6) == KFO_OK
    roots = [8, 11, 13]                               # disjoint level-3 subtrees
    assert part.subtrees(roots, 0.4, 1e-6, 24, 0.6) == KFO_OK
    for a in roots:
        for lv in range(whole.D - 3 + 1):
            for b in range(a << lv, (a + 1) << lv):
                assert part.rank(b) == whole.rank(b)
                assert np.array_equal(part.skel(b), whole.skel(b))
                assert np.array_equal(part.P(b), whole.P(b))
                assert np.array_equal(part.Phat(b), whole.Phat(b))
                if not whole.is_leaf(b):
                    assert np.array_equal(part.Z(b), whole.Z(b))
    full = Oracle(X, 100)
    full.subtrees([1], 0.4, 1e-6, 24, 0.6)
    for b in range(2, whole.nnodes + 1):
        assert np.array_equal(full.Phat(b), whole.Phat(b))
    b = np.random.default_rng(3).standard_normal(3000)
    np.testing.assert_array_equal(full.solve(b), whole.solve(b))
    with pytest.raises(ValueError):
        part.subtrees([4, 9], 0.4, 1e-6, 24, 0.6)     # 9 lies under 4


# ---------------------------------------------------------------- hybrid level-restricted solver
def test_hybrid_at_level_1_equals_the_direct_solver():
    """With the frontier at level 1 the hybrid operator D + UV (Sec. II-C) is
    the direct solver's operator (Eq. e:blocksmw at the root, same IDs below),
    and its reduced system I + VW is the root's Z: same operator, same solution."""
    X, rng = make(N=2048, d=3, m=64, seed=15)
    direct, hyb = Oracle(X, 64), Oracle(X, 64)
    direct.skeletonize(0.25, 1e-6, 40)
    direct.factorize(0.7)
    assert hyb.hybrid(1, 0.25, 1e-6, 40, 0.7) == KFO_OK
    b = rng.standard_normal(2048)
    np.testing.assert_allclose(hyb.hybrid_matvec(b), direct.matvec(b), rtol=0, atol=1e-13 * np.abs(b).sum())
    x, xd = hyb.hybrid_solve(b), direct.solve(b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-12


@pytest.mark.parametrize("N,m,L", [(1024, 128, 1), (1024, 128, 2), (1024, 128, 3), (1000, 100, 2), (1000, 100, 4)])
def test_hybrid_full_rank_equals_dense_cholesky(N, m, L):
    """tau = 0, s_max >= N/2 and S' = the whole complement: every ID keeps all
    columns, the hybrid operator is lambda I + K exactly at any frontier level
    (also on ragged trees: N = 1000, leaves of 62 and 63 points), and its solve
    equals scipy's dense Cholesky solve."""
    X, rng = make(N=N, d=4, m=m, seed=7)
    o = Oracle(X, m)
    assert o.hybrid(L, 0.35, 0.0, 1024, 1.0, n_samp=1024) == KFO_OK
    b = rng.standard_normal(N)
    A = gauss_K(X, X, 0.35) + np.eye(N)
    xd = sla.cho_solve(sla.cho_factor(A), b)
    assert np.linalg.norm(o.hybrid_solve(b) - xd) / np.linalg.norm(xd) <= 1e-10


def test_hybrid_operator_blocks_and_solve():
    """Frontier at the leaves (L = D): D = blockdiag(lambda I + K_aa) exact,
    the block between leaves a != b is P_{a a~} K_{a~ b} (second form of
    Eq. e:uv).  The operator assembled column by column from the oracle equals
    that block matrix built here from the kernel definition and the oracle's
    skeletons and P; the hybrid solve (Algorithm 6) equals numpy's dense solve
    of it, and it is a different (less compressed) operator than the direct
    solver's."""
    X, rng = make(N=512, d=3, m=64, seed=16)
    o = Oracle(X, 64)
    h, lam = 0.3, 0.5
    assert o.hybrid(o.D, h, 1e-4, 24, lam) == KFO_OK
    perm = o.perm()
    Xt = X[perm]
    nA = 1 << o.D
    A = np.zeros((512, 512))
    for a in range(nA, 2 * nA):
        la, ha = o.node_range(a)
        A[la:ha, la:ha] = gauss_K(Xt[la:ha], Xt[la:ha], h) + lam * np.eye(ha - la)
        Pa, sk = o.P_full(a), o.skel(a)
        for b in range(nA, 2 * nA):
            if b == a:
                continue
            lb, hb = o.node_range(b)
            A[la:ha, lb:hb] = Pa @ gauss_K(Xt[sk], Xt[lb:hb], h)
    inv = np.argsort(perm)                      # tree position of each original index
    Ao = A[np.ix_(inv, inv)]                    # the same operator in original order
    I = np.eye(512)
    Ah = np.stack([o.hybrid_matvec(I[:, j]) for j in range(512)], axis=1)
    assert np.abs(Ah - Ao).max() <= 1e-13 * np.abs(Ao).max()
    b = rng.standard_normal(512)
    x = o.hybrid_solve(b)
    xd = np.linalg.solve(Ao, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-12
    direct = Oracle(X, 64)
    direct.skeletonize(h, 1e-4, 24)
    direct.factorize(lam)
    assert np.linalg.norm(direct.matvec(b) - Ao @ b) > 1e-8 * np.linalg.norm(Ao @ b)
