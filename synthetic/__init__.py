"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no kernel evaluation, ordering, selection or fill).

Generator: the SplitMix64 sequence (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Its n-th output is a pure
function of (state, n) -- the Weyl increment n*0x9E3779B97F4A7C15 followed by
the published 64-bit finaliser -- so it is counter based and vectorises over n.
A uniform double in [0, 1) keeps the top 53 bits: (z >> 11) * 2**-53.

Streams: every draw is addressed by (seed, stream, n); the key of a stream is
finalise(finalise(seed) + stream), so streams of one seed do not overlap in any
way that matters for these workloads.

The workloads echo the point clouds of the paper's experiments (Section 6.1:
points in the unit square or cube with a Matern kernel).  `PRESETS` lists the
five configurations this library is measured on, with their sizes.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "GOLDEN_GAMMA", "mix64", "uniform", "normal", "points", "clustered_points", "planted_factor", "PRESETS",
    "STREAM_POINTS", "STREAM_NORMAL", "STREAM_PLANTED", "STREAM_CLUSTER",
]

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_POINTS = 1
STREAM_NORMAL = 2
STREAM_PLANTED = 3
STREAM_CLUSTER = 4


def mix64(z):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _key(seed: int, stream: int) -> np.uint64:
    s = mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    with np.errstate(over="ignore"):
        k = mix64(s + np.uint64(stream & 0xFFFFFFFFFFFFFFFF))
    return k[0]


def raw64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` SplitMix64 outputs of stream (seed, stream), starting at index `offset`."""
    n = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(_key(seed, stream) + n * GOLDEN_GAMMA)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (raw64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, stream: int = STREAM_NORMAL) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform of consecutive uniform pairs."""
    pairs = (count + 1) // 2
    u = uniform(seed, stream, 2 * pairs)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def points(n: int, dim: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^dim, row-major float64 (point i, coordinate c = draw i*dim+c)."""
    return uniform(seed, STREAM_POINTS, n * dim).reshape(n, dim)


def clustered_points(n: int, dim: int, seed: int, frac: float = 0.5, width: float = 0.05) -> np.ndarray:
    """An inhomogeneous cloud: `points(n, dim, seed)`, with each point moved, when its own
    extra uniform draw is below `frac`, into the cube of side `width` centred in [0,1)^dim
    (same relative position inside it).  About frac * n points crowd the small cube; the rest
    stay spread over the unit cube."""
    p = points(n, dim, seed)
    pick = uniform(seed, STREAM_CLUSTER, n) < frac
    p[pick] = 0.5 + width * (p[pick] - 0.5)
    return p


def planted_factor(n: int, s: int, seed: int, diag: float = 10.0) -> np.ndarray:
    """Dense lower-triangular factor for the planted-recovery workload (Section 6.5).

    Column c gets `diag` on the diagonal and min(s, n-1-c) distinct strictly-lower rows
    chosen uniformly (partial Fisher-Yates on the rows below c) with N(0,1) values.
    """
    L = np.zeros((n, n))
    u = uniform(seed, STREAM_PLANTED, n * n)
    z = normal(seed, n * s, stream=STREAM_PLANTED + 100)
    zi = 0
    for c in range(n):
        L[c, c] = diag
        rows = list(range(c + 1, n))
        take = min(s, len(rows))
        for t in range(take):
            r = t + int(u[c * n + t] * (len(rows) - t))
            rows[t], rows[r] = rows[r], rows[t]
            L[rows[t], c] = z[zi]
            zi += 1
    return L


# Workload presets.  `nu_x2` is twice the Matern smoothness (1, 3, 5 -> 1/2, 3/2, 5/2).
PRESETS = {
    "cfg1_single_fp64": dict(n=4096, dim=2, seed=0, nu_x2=3, length_scale=0.1, variance=1.0,
                             nugget=1e-8, n_cand=256, k=16, mode="single"),
    "cfg2_single_batched": dict(n=65536, dim=3, seed=0, nu_x2=5, length_scale=0.05, variance=1.0,
                                nugget=1e-6, n_cand=512, k=32, mode="single"),
    "cfg3_aggregated": dict(n=1 << 20, dim=2, seed=0, nu_x2=3, length_scale=0.02, variance=1.0,
                            nugget=1e-6, n_cand=1024, k=64, m_min=8, m_max=64, mode="aggregated"),
    "cfg4_learned": dict(n=1 << 20, dim=2, seed=0, nu_x2=3, length_scale=0.02, variance=1.0,
                         nugget=1e-6, n_cand=1024, k=64, m_min=8, m_max=64, top=256, mode="learned"),
    "cfg5_pcg": dict(n=1 << 20, dim=2, seed=0, nu_x2=3, length_scale=0.02, variance=1.0,
                     nugget=1e-6, shift=1e-4, nrhs=8, tol=1e-8, k=64, mode="pcg"),
}
