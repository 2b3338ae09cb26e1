"""Seeded synthetic QUBO instances shaped like the paper's benchmark sets.

The paper evaluates on the Beasley set (n = 2500, sparse, integer weights)
and the Palubeckis set (n = 5000 / 7000, dense) (Section 4.1).  Neither is
shipped here; these generators stand in for them with the same shapes:
symmetric integer Q with entries in [-100, 100] at a chosen density.

This module holds input generation only -- none of the solver's arithmetic --
so the tests can feed the same instance to the CUDA library and to the CPU
oracle.  Generator: numpy PCG64 seeded with ``seed``.

Recipe (for i <= j, mirrored to Q_ji):
  * density == 1: Q_ij uniform on the integers of [lo, hi];
  * density  < 1: Q_ij present with probability ``density``, and when present
    uniform on the non-zero integers of [lo, hi]; absent entries are 0.
"""
from __future__ import annotations

import numpy as np


def make_qubo(n: int, density: float = 1.0, seed: int = 0, lo: int = -100, hi: int = 100) -> np.ndarray:
    """Symmetric int8 [n, n] QUBO matrix."""
    if not (-128 <= lo <= hi <= 127):
        raise ValueError("entries must fit int8")
    if n < 1:
        raise ValueError("n must be positive")
    rng = np.random.Generator(np.random.PCG64(seed))
    if density >= 1.0:
        V = rng.integers(lo, hi + 1, size=(n, n), dtype=np.int16)
    else:
        if lo <= 0 <= hi:
            V = rng.integers(lo, hi, size=(n, n), dtype=np.int16)  # lo..hi-1
            V[V >= 0] += 1                                        # -> lo..-1, 1..hi
        else:
            V = rng.integers(lo, hi + 1, size=(n, n), dtype=np.int16)
        keep = rng.random(size=(n, n)) < density
        V = np.where(keep, V, 0).astype(np.int16)
    U = np.triu(V)
    Q = U + np.triu(U, 1).T
    return Q.astype(np.int8)


def random_solutions(n: int, z: int, seed: int) -> np.ndarray:
    """Uniform random binary [z, n] uint8 rows (for tests that start from a
    given state rather than the solver's own initial set)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    return rng.integers(0, 2, size=(z, n), dtype=np.uint8)


def random_subsets(n: int, sizes, seed: int) -> np.ndarray:
    """Disjoint index groups of the given sizes, each sorted ascending,
    concatenated (int32).  Used to drive the anneal kernel directly."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5B5E7))
    perm = rng.permutation(n).astype(np.int32)
    out, off = [], 0
    for m in sizes:
        out.append(np.sort(perm[off:off + m]))
        off += m
    return np.concatenate(out).astype(np.int32) if out else np.zeros(0, np.int32)


# Workloads named after the paper's instance families, with the sizes the
# benchmark and the parity tests use.
WORKLOADS = {
    "dense-n64-m16-z8": dict(n=64, density=1.0, m=16, z=8, K=1, sweeps=256, iters=200),
    "beasley-like-n2500-d0.1-m64-z128": dict(n=2500, density=0.1, m=64, z=128, K=1, sweeps=1024),
    "palubeckis-like-n5000-d0.5-uneven32-256-z32k16": dict(n=5000, density=0.5, m_min=32, m_max=256,
                                                           z=32, K=16),
    "palubeckis-like-n7000-d1.0-R256": dict(n=7000, density=1.0, z=256),
    "n10000-d0.5": dict(n=10000, density=0.5),
}
