"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module generates point sets and workload descriptions only.  It holds none
of the eigenvalue method's arithmetic (no kernel evaluation, no factorization,
no counting), so that the CPU oracle and the CUDA path can both consume the
same inputs without sharing any code of the method itself.

Random numbers come from SplitMix64 (S. Vigna's public-domain generator, the
mixing function of Java's SplittableRandom, Steele/Lea/Flood 2014), written out
with numpy uint64 arithmetic so that the same seed gives the same bits on any
machine.  Uniform doubles take the top 53 bits; Gaussians use Box-Muller.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of SplitMix64 started at state ``seed``."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.arange(
            1, count + 1, dtype=np.uint64)
        z = state
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """``count`` doubles uniform in [0, 1): top 53 bits of SplitMix64 × 2^-53."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, count: int) -> np.ndarray:
    """``count`` standard normal doubles by the Box-Muller transform."""
    half = (count + 1) // 2
    u = uniform(seed, 2 * half)
    u1 = 1.0 - u[0::2]            # in (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * half)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def uniform_cube(n: int, d: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1]^d, row-major n×d (the unit square for d=2)."""
    return uniform(seed, n * d).reshape(n, d)


def cylinder_lattice(n: int, seed: int, radius: float = 5.0, spacing: float = 0.14,
                     jitter: float = 0.01) -> np.ndarray:
    """Rings of round(2πR/spacing) points, rings ``spacing`` apart along z,
    first n points in z-major order, Gaussian jitter of std ``jitter``."""
    per_ring = int(round(2.0 * math.pi * radius / spacing))
    idx = np.arange(n)
    ring, k = idx // per_ring, idx % per_ring
    theta = 2.0 * np.pi * k / per_ring
    pts = np.stack([radius * np.cos(theta), radius * np.sin(theta), spacing * ring], axis=1)
    return pts + jitter * gaussian(seed, 3 * n).reshape(n, 3)


def unit_circle(n: int, seed: int) -> np.ndarray:
    """n points uniformly distributed on the circumference of the unit circle
    (angles 2 pi U), n x 2: the synthetic Laplace workload of the paper's
    Sec. 5.1."""
    t = 2.0 * math.pi * uniform(seed, n)
    return np.stack([np.cos(t), np.sin(t)], axis=1)


def line_points(n: int) -> np.ndarray:
    """Points 1, 2, ..., n on a line (n×1): the closed-form test matrices."""
    return np.arange(1, n + 1, dtype=np.float64).reshape(n, 1)


# Kernel kinds.  The numbering is the C ABI's (include/h2eig.h).
LAPLACE_EPS = 0      # 1/(r + p0)
YUKAWA_EPS = 1       # exp(-r)/(r + p0)
GAUSS_PLUS_INV = 2   # exp(-r^2/2) + p0/(r + p1)
TRIDIAG_TEST = 3     # 2 at r = 0, -1 at r = 1, else 0   (points on the integers)
MIN_TEST = 4         # min(x_i, x_j) of the first coordinates


@dataclass
class Workload:
    """One synthetic problem: points plus the H^2 parameters."""
    name: str
    points: np.ndarray
    kernel: int
    kparams: tuple = (1e-3, 0.0, 0.0, 0.0)
    leaf: int = 64
    rank: int = 16
    eta: float = 1.0
    ks: list = field(default_factory=list)
    tol: float = 1e-8


def c1_laplace_square(seed: int = 1, n: int = 1024) -> Workload:
    """n points uniform in the unit square, 1/(r+1e-3), leaf 64, rank 16, k = n/2."""
    return Workload("laplace2d_n%d" % n, uniform_cube(n, 2, seed), LAPLACE_EPS,
                    (1e-3, 0, 0, 0), 64, 16, 1.0, [n // 2], 1e-8)


def c2_yukawa_cube(seed: int = 2, n: int = 65536) -> Workload:
    """n points uniform in the unit cube, exp(-r)/(r+1e-3), leaf 256, rank 32,
    k in {1, n/4, n/2, 3n/4, n}."""
    return Workload("yukawa3d_n%d" % n, uniform_cube(n, 3, seed), YUKAWA_EPS,
                    (1e-3, 0, 0, 0), 256, 32, 1.0, [1, n // 4, n // 2, 3 * n // 4, n], 1e-8)


def cp_cylinder(seed: int = 4, n: int = 262144) -> Workload:
    """Cylindrical lattice, exp(-r^2/2) + 1e-2/(r+0.1), leaf 256, rank 48,
    32 interior k around n/2."""
    return Workload("cylinder_n%d" % n, cylinder_lattice(n, seed), GAUSS_PLUS_INV,
                    (1e-2, 0.1, 0, 0), 256, 48, 1.0, list(range(n // 2 - 16, n // 2 + 16)), 1e-8)


def batch_members(count: int = 512, seed: int = 3) -> list:
    """The many-matrix configuration: ``count`` independent problems with
    n = floor(2048 * 16^U) (log-uniform in [2048, 32768]), dimension 2 or 3
    with probability 1/2, points uniform in the unit square or cube (point
    seed 1000 * seed + i), kernel 1/(r + 1e-3), leaf/rank 64/16 in 2D and
    256/32 in 3D, and k uniform in 1..n.  Returns Workload descriptions."""
    u = uniform(seed, 3 * count)
    out = []
    for i in range(count):
        n = int(2048.0 * 16.0 ** u[3 * i])
        d = 2 if u[3 * i + 1] < 0.5 else 3
        k = 1 + int(u[3 * i + 2] * n)
        leaf, rank = (64, 16) if d == 2 else (256, 32)
        out.append(Workload("batch%d_d%d_n%d" % (i, d, n), uniform_cube(n, d, 1000 * seed + i), LAPLACE_EPS,
                            (1e-3, 0, 0, 0), leaf, rank, 1.0, [k], 1e-8))
    return out
