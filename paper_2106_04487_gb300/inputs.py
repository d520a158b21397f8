"""Seeded synthetic workloads (points, weights, target subsamples).

This module holds only random-number recipes -- none of the method's
arithmetic -- so the GPU path, the CPU oracle, the tests and the benchmark can
all draw identical inputs from it.  Points are drawn in float64 with numpy's
PCG64 and rounded once to float32; both sides consume the same float32 arrays.

The workloads stand in for no public dataset: they are the synthetic point
distributions of the benchmark configurations (uniform cube, Gaussian mixture,
unit ball, clustered + uniform mix).
"""
from __future__ import annotations

import numpy as np

SEED_POINTS, SEED_WEIGHTS, SEED_SUBSAMPLE, SEED_BATCH = 0, 1, 2, 3


def uniform_cube(n: int, d: int = 3, seed: int = SEED_POINTS) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random((n, d)).astype(np.float32)


def gaussian_mixture(n: int, d: int = 3, components: int = 10, std: float = 0.05,
                     seed: int = SEED_POINTS) -> np.ndarray:
    """Equal-weight isotropic Gaussian mixture, centres U[0,1]^d, unclipped."""
    rng = np.random.default_rng(seed)
    centres = rng.random((components, d))
    lab = rng.integers(0, components, size=n)
    x = centres[lab] + std * rng.standard_normal((n, d))
    return x.astype(np.float32)


def unit_ball(n: int, d: int = 3, seed: int = SEED_POINTS) -> np.ndarray:
    """Uniform in the unit ball: Gaussian direction times U^(1/d) radius."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    rad = rng.random(n) ** (1.0 / d)
    return (g * rad[:, None]).astype(np.float32)


def unit_sphere(n: int, d: int = 3, seed: int = SEED_POINTS) -> np.ndarray:
    """Uniform on the unit hypersphere S^(d-1) (normalised Gaussian vectors): the point set of
    the paper's runtime-versus-N experiment (Sec. 5.1)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def uniform_plus_clusters(n: int, d: int = 3, clusters: int = 100, std: float = 0.005,
                          seed: int = SEED_POINTS) -> np.ndarray:
    """Half uniform in the unit cube, half in tight isotropic clusters."""
    rng = np.random.default_rng(seed)
    nu = n // 2
    a = rng.random((nu, d))
    centres = rng.random((clusters, d))
    lab = rng.integers(0, clusters, size=n - nu)
    b = centres[lab] + std * rng.standard_normal((n - nu, d))
    return np.concatenate([a, b]).astype(np.float32)


def normal_weights(n: int, nrhs: int = 1, seed: int = SEED_WEIGHTS) -> np.ndarray:
    """w ~ N(0,1), layout [nrhs][N], float32."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, n)).astype(np.float32)


def uniform_weights(n: int, nrhs: int = 1, seed: int = SEED_WEIGHTS) -> np.ndarray:
    """w ~ U[-1,1], layout [nrhs][N], float32."""
    rng = np.random.default_rng(seed)
    return (2.0 * rng.random((nrhs, n)) - 1.0).astype(np.float32)


def subsample(n: int, k: int, seed: int = SEED_SUBSAMPLE) -> np.ndarray:
    """k distinct target indices out of n, sorted."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def batch_sizes(count: int = 256, lo: int = 2000, hi: int = 200000, seed: int = SEED_BATCH) -> np.ndarray:
    """Problem sizes log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


# The five benchmark configurations (sizes, kernels, orders).  'kernel' entries are
# (name, lengthscale, alpha, scale); the product and the oracle map names to their own enums.
CONFIGS = {
    "gauss20k": dict(points=lambda: uniform_cube(20000, 3), N=20000, d=3,
                     kernel=("gaussian", 0.1, 1.0, 1.0), p=4, leaf_size=512, theta=0.5, nrhs=1),
    "matern1m": dict(points=lambda: gaussian_mixture(1_000_000, 3, 10, 0.05), N=1_000_000, d=3,
                     kernel=("matern32", 0.2, 1.0, 1.0), p=6, leaf_size=512, theta=0.5, nrhs=1),
    "cauchy1m": dict(points=lambda: gaussian_mixture(1_000_000, 3, 10, 0.05), N=1_000_000, d=3,
                     kernel=("cauchy", 0.05, 1.0, 1.0), p=6, leaf_size=512, theta=0.5, nrhs=1),
}
