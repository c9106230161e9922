"""The seeded synthetic inputs have the shapes, parameters and structure the
workloads are defined with (CPU).

Each recipe stands in for one of the paper's datasets (its Sec. IV table of
datasets); these checks tie the generated arrays to the recipe's statement:
sizes, parameter values, value ranges, standardization, the rank of the
linear manifold, the binary features' frequency, the batch's size range, and
reproducibility from the seed.
"""
import numpy as np
import pytest

from paper_1701_02324_gb300 import inputs


def test_plain_fp64_recipe():
    p = inputs.plain_fp64()
    assert p.X.shape == (4096, 8) and p.B.shape == (4096, 1)
    assert (p.h, p.lam, p.m, p.s_max, p.tau, p.n_samp) == (0.5, 1.0, 256, 64, 1e-6, 128)
    assert p.X.min() >= 0.0 and p.X.max() < 1.0                   # uniform in [0, 1)^8
    assert abs(p.X.mean() - 0.5) < 0.01 and abs(p.X.var() - 1 / 12) < 0.002
    assert abs(p.B.mean()) < 0.05 and abs(p.B.std() - 1.0) < 0.05  # b ~ N(0, 1)
    q = inputs.plain_fp64()
    assert np.array_equal(p.X, q.X) and np.array_equal(p.B, q.B)   # seeded


def test_mixed_recipe_is_a_mixture_of_16_tight_clusters():
    p = inputs.mixed()
    assert p.X.shape == (65536, 8) and p.B.shape == (65536, 16)
    assert (p.h, p.lam, p.m, p.s_max, p.tau) == (0.3, 0.1, 512, 128, 1e-5)
    # sigma = 0.1 clusters around 16 centres in [0,1]^8: a point's nearest
    # other point among a sample is much closer than the spread of the data
    rng = np.random.default_rng(0)
    S = p.X[rng.choice(p.N, 2000, replace=False)]
    d2 = ((S[:, None, :] - S[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    near = np.sqrt(d2.min(axis=1))
    assert np.median(near) < 0.25 * np.sqrt(((S - S.mean(0)) ** 2).sum(1)).mean()
    # and closer than the typical distance of two points of one cluster,
    # sigma * sqrt(2 * 8) = 0.4 for 8-D N(0, 0.1^2 I) clusters
    assert np.median(near) < 0.1 * np.sqrt(2 * 8)


def test_scale_recipe_is_a_standardized_6d_manifold():
    p = inputs.scale()
    assert p.X.shape == (1 << 20, 28) and p.B.shape == (1 << 20, 1)
    assert (p.h, p.lam, p.m, p.s_max, p.tau, p.n_samp) == (1.0, 1.0, 1024, 256, 1e-4, 512)
    np.testing.assert_allclose(p.X.mean(0), 0.0, atol=1e-12)
    np.testing.assert_allclose(p.X.std(0), 1.0, rtol=1e-12)
    sv = np.linalg.svd(p.X[::64], compute_uv=False)
    # six latent directions carry the data; the N(0, 0.01^2) noise is two orders below
    assert sv[5] > 20 * sv[6]
    assert sv[6] / sv[0] < 0.02


def test_batched_recipe():
    probs = inputs.batched()
    assert len(probs) == 256
    Ns = np.array([q.N for q in probs])
    assert Ns.min() >= 2048 and Ns.max() <= 32768
    # log-uniform: the median of N near sqrt(2048 * 32768) = 8192
    assert 6000 < np.median(Ns) < 11000
    for q in probs:
        assert q.X.shape == (q.N, 8) and q.B.shape == (q.N, 64)
        assert 0.2 <= q.h <= 1.0
        assert (q.lam, q.m, q.s_max, q.tau) == (0.5, 256, 64, 1e-5)
        assert q.X.min() >= 0.0 and q.X.max() < 1.0
    hs = np.array([q.h for q in probs])
    assert hs.min() < 0.3 and hs.max() > 0.9                       # spans U[0.2, 1.0]
    again = inputs.batched(3, 64)
    for a, q in zip(again, probs[:3]):                             # seeded per problem
        assert np.array_equal(a.X, q.X) and a.h == q.h


def test_differentiation_recipe_has_10_continuous_and_44_binary_features():
    p = inputs.differentiation()
    assert p.X.shape == (1 << 18, 54) and p.B.shape == (1 << 18, 1)
    assert (p.h, p.lam, p.m, p.s_max, p.tau) == (2.0, 1.0, 512, 256, 1e-5)
    assert p.extra["y"].shape == (1 << 18,)
    np.testing.assert_allclose(p.X.mean(0), 0.0, atol=1e-10)
    np.testing.assert_allclose(p.X.std(0), 1.0, rtol=1e-10)
    for j in range(10):
        assert len(np.unique(p.X[:1000, j])) == 1000                  # continuous
    for j in range(10, 54):
        vals = np.unique(p.X[:, j])
        assert len(vals) == 2                                          # a standardized Bernoulli
        frac = float(np.mean(p.X[:, j] == vals[1]))
        assert abs(frac - 0.1) < 0.01                                  # p = 0.1


@pytest.mark.parametrize("fn", [inputs.plain_fp64, inputs.mixed])
def test_inputs_hold_no_method_arithmetic(fn):
    """The module only draws numbers: float64 arrays, C-contiguous, finite."""
    p = fn()
    for a in (p.X, p.B):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and np.isfinite(a).all()
