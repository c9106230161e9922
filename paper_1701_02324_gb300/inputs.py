"""Seeded synthetic inputs with the shapes of the paper's workloads.

This module holds no arithmetic of the method: it only draws points,
right-hand sides and problem parameters with numpy, so that the CUDA path and
the CPU oracle can be fed the same data.  The datasets of the paper (Table
"datasets": COVTYPE, SUSY, HIGGS, MNIST, MRI, NORMAL) are not available; the
recipes below stand in for their shapes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SAMPLER_SEED = 0x1701


@dataclass
class Problem:
    name: str
    X: np.ndarray           # N x d, float64, original order
    B: np.ndarray           # N x nrhs, float64
    h: float
    lam: float
    m: int
    s_max: int
    tau: float
    n_samp: int = 0
    seed: int = SAMPLER_SEED
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        if self.n_samp == 0:
            self.n_samp = 2 * self.s_max

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def _standardize(X: np.ndarray) -> np.ndarray:
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd == 0] = 1.0
    return (X - mu) / sd


def uniform_cube(N: int, d: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random((N, d))


def gaussian_mixture(N: int, d: int, k: int, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    centres = rng.random((k, d))
    lab = rng.integers(0, k, size=N)
    return centres[lab] + sigma * rng.standard_normal((N, d))


def linear_manifold(N: int, d: int, k: int, noise: float, seed: int) -> np.ndarray:
    """k-dim Gaussian latents mapped by a random k x d orthonormal map, plus
    N(0, noise^2) noise, then standardized (the paper's NORMAL set: a 6-D normal
    embedded in a higher dimension with noise)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((d, k))
    Q, _ = np.linalg.qr(G)            # d x k, orthonormal columns
    z = rng.standard_normal((N, k))
    X = z @ Q.T + noise * rng.standard_normal((N, d))
    return _standardize(X)


def covtype_like(N: int, n_cont: int, n_bin: int, p: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    Xc = rng.standard_normal((N, n_cont))
    Xb = (rng.random((N, n_bin)) < p).astype(np.float64)
    return _standardize(np.concatenate([Xc, Xb], axis=1))


def rhs(N: int, nrhs: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((N, nrhs))


# ---- the five workloads (small/plain, mixed, scale, batched, differentiation)

def plain_fp64(N: int = 4096) -> Problem:
    """N=4096, d=8, uniform in [0,1]^8; h=0.5, lambda=1, m=256, s_max=64, tau=1e-6."""
    seed = 1701001
    return Problem("plain_fp64_N4096_d8", uniform_cube(N, 8, seed), rhs(N, 1, seed + 17),
                   h=0.5, lam=1.0, m=256, s_max=64, tau=1e-6)


def mixed(N: int = 65536) -> Problem:
    """N=65,536, d=8, 16 isotropic Gaussians (sigma 0.1, centres uniform in
    [0,1]^8); h=0.3, lambda=0.1; m=512, s_max=128, tau=1e-5; 16 RHS."""
    seed = 1701002
    return Problem("mixed_N65536_d8", gaussian_mixture(N, 8, 16, 0.1, seed), rhs(N, 16, seed + 17),
                   h=0.3, lam=0.1, m=512, s_max=128, tau=1e-5)


def scale(N: int = 1 << 20) -> Problem:
    """N=2^20, d=28, 6-D linear manifold + N(0, 0.01^2) noise, standardized;
    h=1, lambda=1; m=1024, s_max=256, tau=1e-4; 1 RHS."""
    seed = 1701003
    return Problem("scale_N1048576_d28", linear_manifold(N, 28, 6, 0.01, seed), rhs(N, 1, seed + 17),
                   h=1.0, lam=1.0, m=1024, s_max=256, tau=1e-4)


def batched(n_problems: int = 256, nrhs: int = 64) -> list[Problem]:
    """256 problems, N log-uniform in [2048, 32768], d=8 uniform in [0,1]^8,
    h ~ U[0.2, 1.0], lambda=0.5, m=256, s_max=64, tau=1e-5, 64 RHS each."""
    out = []
    for i in range(n_problems):
        seed = 1701004 * 1000 + i
        rng = np.random.default_rng(seed)
        N = int(math.floor(math.exp(rng.uniform(math.log(2048), math.log(32768)))))
        h = float(rng.uniform(0.2, 1.0))
        out.append(Problem(f"batched_{i}", uniform_cube(N, 8, seed + 1), rhs(N, nrhs, seed + 2),
                           h=h, lam=0.5, m=256, s_max=64, tau=1e-5))
    return out


def differentiation(N: int = 1 << 18) -> Problem:
    """N=2^18, d=54: 10 N(0,1) + 44 Bernoulli(0.1) features, standardized;
    h=2, lambda=1, m=512, s_max=256, tau=1e-5; targets y ~ N(0,1)."""
    seed = 1701005
    p = Problem("differentiation_N262144_d54", covtype_like(N, 10, 44, 0.1, seed), rhs(N, 1, seed + 17),
                h=2.0, lam=1.0, m=512, s_max=256, tau=1e-5)
    p.extra["y"] = rhs(N, 1, seed + 29)[:, 0]
    return p
