"""Counter-based seeded random numbers for the synthetic workloads.

Every random draw used by the scene generators comes from here, so that the
oracle and the CUDA path are always fed bit-identical inputs.  Nothing in this
module knows about voxels, covariances or residuals.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter mode: draw ``i`` of stream
``s`` is ``mix(key(seed, s) + (i + 1) * GAMMA)``, so any slice of a stream can
be produced independently and in any order.  Uniform doubles take the top 53
bits; normals use the Box-Muller transform in FP64.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (a bijection on uint64)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


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
        base = np.array([(int(seed) * 0x9E3779B97F4A7C15 + _name_id(name)) & 0xFFFFFFFFFFFFFFFF],
                        dtype=np.uint64)
        self.key = _mix(base)[0]
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """U[lo, hi) in FP64 from the top 53 bits."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """Standard normal by Box-Muller (u1 in (0, 1], so the log is finite)."""
        m = (n + 1) // 2
        bits = self.u64(2 * m)
        u1 = ((bits[:m] >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
        u2 = (bits[m:] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return z[:n]

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers in [lo, hi) (multiply-shift; bias below 2^-40 for the ranges used here)."""
        u = self.uniform(n)
        return np.minimum(lo + np.floor(u * (hi - lo)).astype(np.int64), hi - 1)

    def unit_vectors(self, n: int) -> np.ndarray:
        v = self.normal(3 * n).reshape(n, 3)
        return v / np.linalg.norm(v, axis=1, keepdims=True)
