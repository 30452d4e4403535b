"""Seeded workload generators for the octahedron KPZ simulator.

The paper's own workloads are synthetic: a flat start on an L x L periodic
lattice, p = 1, q = 0 (arXiv:1204.5072, Sec. 2.1 and Sec. 3.1). This module
holds the workload shapes, the sampling times and random *valid* surfaces
used to exercise the height and width code on states other than the flat one.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One single-lattice workload: lattice size, rates, run length, RNG key."""
    name: str
    L: int
    p: float
    q: float
    mcs: int
    seed: int = 1
    sample: int = 0
    bx: int = 128
    by: int = 128


# Single-lattice workloads of the benchmark suite.
L256_1000 = Workload("octahedron L=256 p=1 q=0 1000 MCS", 256, 1.0, 0.0, 1000)
L4096_P1 = Workload("octahedron L=4096 p=1 q=0 10^4 MCS", 4096, 1.0, 0.0, 10_000)
L4096_P095 = Workload("octahedron L=4096 p=0.95 q=0.05 10^4 MCS", 4096, 0.95, 0.05, 10_000)
L65536_2000 = Workload("octahedron L=65536 p=1 q=0 2000 MCS", 65536, 1.0, 0.0, 2000)


def sample_times(T: int, n: int = 64) -> list[int]:
    """Log-spaced sampling times t_k = ceil(10^(k log10(T) / (n-1))), k = 0..n-1,
    deduplicated, with t = 0 prepended (the paper samples W^2 'at certain
    sampling times', Sec. 2.1)."""
    if T <= 0:
        return [0]
    ts = {0}
    for k in range(n):
        ts.add(min(T, int(math.ceil(10 ** (k * math.log10(T) / (n - 1)) - 1e-9))))
    ts.add(T)
    return sorted(ts)


@dataclasses.dataclass(frozen=True)
class EnsembleSpec:
    """One realisation of the batched ensemble."""
    L: int
    p: float
    q: float
    mcs: int
    sample: int


def ensemble_specs(n: int = 512, seed: int = 1, cap: int = 100_000,
                   log2_lmin: int = 8, log2_lmax: int = 13) -> list[EnsembleSpec]:
    """Batched-ensemble workload: L = 2^U{log2_lmin..log2_lmax} (log-uniform),
    p ~ U[0.5, 1], q = 1 - p, run length min(ceil(4 L^1.6), cap) MCS."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = 1 << int(rng.integers(log2_lmin, log2_lmax + 1))
        p = float(rng.uniform(0.5, 1.0))
        T = int(min(math.ceil(4 * L ** 1.6), cap))
        out.append(EnsembleSpec(L, p, 1.0 - p, T, k))
    return out


def _periodic_walk(n: int, rng: np.random.Generator) -> np.ndarray:
    steps = np.array([1] * (n // 2) + [0] * (n // 2), np.uint8)
    rng.shuffle(steps)
    return steps


def separable_surface(L: int, seed: int):
    """A random valid surface h(i,j) = f(i) + g(j) with f, g periodic +-1 walks.

    Returns (sx, sy) as uint8 arrays [j, i] (1 = slope +1). Every row of sx is
    the same walk and every column of sy is the same walk, so neighbour
    heights differ by one and all loop sums vanish."""
    rng = np.random.default_rng(seed)
    f = _periodic_walk(L, rng)
    g = _periodic_walk(L, rng)
    sx = np.tile(f[None, :], (L, 1))
    sy = np.tile(g[:, None], (1, L))
    return np.ascontiguousarray(sx), np.ascontiguousarray(sy)


def valid_heights_4x4():
    """All height functions on the 4x4 torus with h(0,0) = 0 and |dh| = 1 on
    every nearest-neighbour bond (periodic), found by brute force over the
    +-1 steps of a spanning tree."""
    L = 4
    out = []
    # spanning tree: column 0 from (0,j-1) to (0,j), then each row from (i-1,j)
    for bits in range(1 << 15):
        h = np.zeros((L, L), np.int64)
        b = bits
        for j in range(1, L):
            h[j, 0] = h[j - 1, 0] + (1 if b & 1 else -1)
            b >>= 1
        for j in range(L):
            for i in range(1, L):
                h[j, i] = h[j, i - 1] + (1 if b & 1 else -1)
                b >>= 1
        dx = np.roll(h, -1, axis=1) - h
        dy = np.roll(h, -1, axis=0) - h
        if np.all(np.abs(dx) == 1) and np.all(np.abs(dy) == 1):
            out.append(h)
    return out
