"""Seeded random numbers for the synthetic workloads.

Every random draw used by the scene generators comes from here, so that the oracle and the
CUDA path are always fed bit-identical inputs.  Nothing in this module knows about voxels,
covariances or residuals.

Generator: numpy's Philox 4x64 counter-based bit generator (Salmon et al., "Parallel random
numbers: as easy as 1, 2, 3", SC 2011), one independent stream per (seed, name): the Philox
key is derived from the seed and a 64-bit FNV-1a hash of the stream name.  Uniform doubles
use the top 53 bits; normals use numpy's ziggurat sampler.
"""
from __future__ import annotations

import numpy as np


def _name_id(name: str) -> int:
    """Stable 64-bit id of a stream name (FNV-1a)."""
    h = 0xCBF29CE484222325
    for ch in name.encode():
        h ^= ch
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


class Stream:
    """One independent stream of random numbers, addressed by (seed, name)."""

    def __init__(self, seed: int, name: str):
        key = np.array([int(seed) & 0xFFFFFFFFFFFFFFFF, _name_id(name)], dtype=np.uint64)
        self.gen = np.random.Generator(np.random.Philox(key=key))

    def u64(self, n: int) -> np.ndarray:
        return self.gen.integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """U[lo, hi) in FP64."""
        return lo + (hi - lo) * self.gen.random(n)

    def normal(self, n: int) -> np.ndarray:
        """Standard normal draws."""
        return self.gen.standard_normal(n)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers in [lo, hi)."""
        return self.gen.integers(lo, hi, size=n, dtype=np.int64)

    def unit_vectors(self, n: int) -> np.ndarray:
        v = self.normal(3 * n).reshape(n, 3)
        return v / np.linalg.norm(v, axis=1, keepdims=True)
