"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no lattice Boltzmann arithmetic: it only draws numbers.
Every draw is counter based (SplitMix64, Steele, Lea & Flood, OOPSLA 2014),
so a value depends only on (seed, stream, index) and any process can
regenerate any part of a field without generating the rest.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function of the states x (uint64 array)."""
    z = np.asarray(x, dtype=np.uint64) + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform [0, 1) doubles for the given element indices of one stream."""
    idx = np.asarray(index, dtype=np.uint64)
    key = splitmix64(np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        z = splitmix64(idx * _GOLDEN + key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_field(seed: int, stream: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    return uniform(seed, stream, np.arange(n, dtype=np.uint64)).reshape(shape)


def random_fields(shape, seed: int, drho: float = 1e-3, du: float = 0.03, dT: float = 0.5):
    """rho = 1 + drho (2xi - 1), each velocity component du (2xi - 1),
    T = dT (2xi - 1); shape = (nz, ny, nx).  Returns rho, u (3, ...), T."""
    rho = 1.0 + drho * (2.0 * uniform_field(seed, 1, shape) - 1.0)
    u = np.stack([du * (2.0 * uniform_field(seed, 2 + a, shape) - 1.0) for a in range(3)])
    T = dT * (2.0 * uniform_field(seed, 5, shape) - 1.0)
    return rho, u, T


def noise(shape, seed: int, stream: int, amp: float) -> np.ndarray:
    """amp (2xi - 1) on an array of the given shape."""
    return amp * (2.0 * uniform_field(seed, stream, shape) - 1.0)


def rb_initial_temperature(nx: int, ny: int, nz: int, seed: int, delta: float = 1e-3) -> np.ndarray:
    """Linear conduction profile between T = +1/2 (bottom wall) and -1/2 (top
    wall) at the node centres z = k + 1/2, plus a uniform random perturbation
    of amplitude delta; shape (nz, ny, nx)."""
    k = np.arange(nz, dtype=np.float64)
    base = 0.5 - (k + 0.5) / nz
    T = np.broadcast_to(base[:, None, None], (nz, ny, nx)).copy()
    return T + noise((nz, ny, nx), seed, 11, delta)


def cell_candidates(seed: int, count: int, edges=(33, 49, 65, 81, 97)):
    """A seeded stream of cell draws for a batched sweep: edge length drawn
    from `edges`, Ra log-uniform in [1e4, 1e7], Pr from {0.71, 7}.  Returns
    a list of (edge, Ra, Pr) tuples; callers skip draws they cannot use."""
    k = np.arange(count, dtype=np.uint64)
    e = uniform(seed, 31, k)
    r = uniform(seed, 32, k)
    p = uniform(seed, 33, k)
    out = []
    for i in range(count):
        edge = edges[min(int(e[i] * len(edges)), len(edges) - 1)]
        out.append((edge, float(10.0 ** (4.0 + 3.0 * r[i])), 0.71 if p[i] < 0.5 else 7.0))
    return out


def warmstart_pairs(seed: int, count: int, ra_range=(1e5, 1e7), pr_range=(0.5, 7.0), stream: int = 41):
    """Seeded (Ra, Pr) draws for the learned warm start: Ra log-uniform and Pr
    uniform over the given ranges."""
    k = np.arange(count, dtype=np.uint64)
    r = uniform(seed, stream, k)
    p = uniform(seed, stream + 1, k)
    lo, hi = np.log10(ra_range[0]), np.log10(ra_range[1])
    return [(float(10.0 ** (lo + (hi - lo) * r[i])), float(pr_range[0] + (pr_range[1] - pr_range[0]) * p[i]))
            for i in range(count)]
