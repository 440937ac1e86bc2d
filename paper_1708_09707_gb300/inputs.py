"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module holds no H-matrix arithmetic: only a counter-based random number
generator (SplitMix64, Steele/Lea/Flood 2014) and the recipes that turn its
draws into point clouds and vectors shaped like the paper's workloads
(Sec. 6.2 uses quasi-random points in [0,1]^d; the synthetic sets here stand in
for them).

SplitMix64, output k of a stream with seed s (k = 1, 2, ...):
    z = s + k * 0x9E3779B97F4A7C15            (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)
A uniform double in [0,1) is (out >> 11) * 2^-53.  A standard normal pair is
Box-Muller on two consecutive uniforms.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based stream: draw k depends only on (seed, k)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.seed + k * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u = self.uniform(2 * m).reshape(m, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
        t = 2.0 * math.pi * u[:, 1]
        out = np.empty((m, 2))
        out[:, 0] = r * np.cos(t)
        out[:, 1] = r * np.sin(t)
        return out.reshape(-1)[:n].copy()


# ----------------------------------------------------------------------------
# Point clouds (row-major (N, d) float64)
# ----------------------------------------------------------------------------

def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """N points i.i.d. uniform in the unit cube [0,1]^d."""
    return SplitMix64(seed).uniform(n * d).reshape(n, d)


def mixture_points(n: int, d: int, seed: int,
                   sigmas=(0.05, 0.1, 0.2)) -> np.ndarray:
    """Equal-weight Gaussian mixture, clipped to [0,1]^d.

    Component means are drawn uniform in [0.2, 0.8]^d from the same stream;
    each point picks its component from one uniform draw.  Clipping puts many
    points exactly on the cube's faces, so the set holds exact duplicate
    coordinates (ties in the Morton order and in pivot searches).
    """
    g = SplitMix64(seed)
    k = len(sigmas)
    means = 0.2 + 0.6 * g.uniform(k * d).reshape(k, d)
    comp = np.minimum((g.uniform(n) * k).astype(np.int64), k - 1)
    z = g.normal(n * d).reshape(n, d)
    pts = means[comp] + np.asarray(sigmas, dtype=np.float64)[comp, None] * z
    return np.clip(pts, 0.0, 1.0)


_PRIMES = (2, 3, 5)


def radical_inverse(idx: np.ndarray, base: int) -> np.ndarray:
    """van der Corput radical inverse: the base-b digits of idx mirrored
    about the radix point (digit k of idx becomes the coefficient of
    b^-(k+1))."""
    i = np.asarray(idx, dtype=np.int64).copy()
    assert i.size == 0 or i.max() < (1 << 40)
    # mirrored digits as an integer over base^digits, one rounding at the end
    num = np.zeros(i.shape, dtype=np.int64)
    den = np.ones(i.shape, dtype=np.int64)
    while np.any(i > 0):
        live = i > 0
        num = np.where(live, num * base + i % base, num)
        den = np.where(live, den * base, den)
        i //= base
    return num / den


def halton_points(n: int, d: int, start: int = 1) -> np.ndarray:
    """The first n points of the d-dimensional Halton sequence (Sec. 6.2's
    point sets): coordinate k of point i is the radical inverse of start + i
    in the k-th prime base (2, 3, 5); no scrambling, index 0 skipped."""
    idx = np.arange(start, start + n, dtype=np.int64)
    return np.stack([radical_inverse(idx, _PRIMES[k]) for k in range(d)], axis=1)


def ragged_batch_sizes(count: int, seed: int, lo: float = 1e4,
                       hi: float = 2.0 ** 18):
    """Sizes log-uniform in [lo, hi] and dimensions d in {2,3} with p = 1/2."""
    g = SplitMix64(seed)
    u = g.uniform(count)
    sizes = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    dims = np.where(g.uniform(count) < 0.5, 2, 3)
    return sizes.astype(np.int64), dims.astype(np.int64)


def normal_vector(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """x ~ N(0, 1); shape (n,) or (nrhs, n) (each right-hand side contiguous)."""
    v = SplitMix64(seed).normal(n * nrhs)
    return v if nrhs == 1 else v.reshape(nrhs, n)


def he_uniform(fan_in: int, fan_out: int, seed: int) -> np.ndarray:
    """He-uniform initial weights W (fan_out, fan_in), limit sqrt(6/fan_in)."""
    lim = math.sqrt(6.0 / fan_in)
    w = SplitMix64(seed).uniform(fan_in * fan_out) * (2.0 * lim) - lim
    return w.reshape(fan_out, fan_in)


# Seeds used throughout: points of workload c use 1000 + c, the x of trial t
# uses 2000 + t, the CG right-hand side uses 3000.
POINT_SEED = 1000
X_SEED = 2000
CG_SEED = 3000

# The workloads the tests and the bench use (sizes, kernel, parameters).
WORKLOADS = {
    "gauss2d_n4096": dict(n=4096, d=2, points="uniform", kernel=0,
                          ell=0.1, leaf=32, eta=1.0, adm="max",
                          eps=1e-8, seed=POINT_SEED + 1),
    "matern3d_n1m": dict(n=1 << 20, d=3, points="uniform", kernel=1,
                         ell=0.2, leaf=64, eta=1.0, adm="min",
                         eps=1e-6, seed=POINT_SEED + 2),
    "mix2d_n1m": dict(n=1 << 20, d=2, points="mixture", kernel=0,
                      ell=0.1, leaf=64, eta=1.0, adm="min",
                      eps=1e-6, seed=POINT_SEED + 3),
    "ragged64": dict(count=64, kernel=0, ell=0.15, leaf=64, eta=1.0,
                     adm="min", eps=1e-6, seed=POINT_SEED + 4),
    "matern3d_n4m_cg": dict(n=1 << 22, d=3, points="uniform", kernel=1,
                            ell=0.1, leaf=64, eta=1.0, adm="min",
                            eps=1e-6, sigma2=1e-2, seed=POINT_SEED + 5),
    # the paper's own setting (Sec. 6.7): Halton points in [0,1]^2, the
    # unscaled Gaussian exp(-r^2), C_leaf = 2048, eta = 1.5 and ACA of fixed
    # rank k = 16 without a stopping criterion (eps <= 0)
    "halton2d_n512k_k16": dict(n=1 << 19, d=2, points="halton", kernel=0,
                               ell=1.0, leaf=2048, eta=1.5, adm="min",
                               eps=0.0, k_cap=16, seed=0),
    # the same setting with the paper's Matern kernel of order 1 (Sec. 6.2,
    # beta - d/2 = 1), unscaled: phi = r K_1(r), normalised to phi(0) = 1
    "halton2d_n512k_k16_matern": dict(n=1 << 19, d=2, points="halton", kernel=2,
                                      ell=1.0, leaf=2048, eta=1.5, adm="min",
                                      eps=0.0, k_cap=16, seed=0),
}


def workload_points(name: str, n: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    if w["points"] == "uniform":
        return uniform_points(n, w["d"], w["seed"])
    if w["points"] == "halton":
        return halton_points(n, w["d"])
    return mixture_points(n, w["d"], w["seed"])
