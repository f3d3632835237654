"""Exact FP32 arithmetic by rational numbers, for pinning the voxel-key rule.

Each operation is evaluated exactly with ``fractions.Fraction`` and rounded once
to the nearest binary32 value (ties to even), which is the IEEE 754 definition of
a correctly rounded multiply or fused multiply-add.  Used only by the tests, on
small inputs.
"""
from fractions import Fraction

import numpy as np


def _even(v: np.float32) -> bool:
    return (np.array(v, dtype=np.float32).view(np.uint32) & 1) == 0


def round_f32(x: Fraction) -> np.float32:
    if x == 0:
        return np.float32(0.0)
    c = np.float32(float(x))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    best, bd = None, None
    for v in cands:
        if not np.isfinite(v):
            continue
        d = abs(Fraction(float(v)) - x)
        if bd is None or d < bd or (d == bd and _even(v) and not _even(best)):
            best, bd = v, d
    return np.float32(best)


def f(v) -> Fraction:
    return Fraction(float(np.float32(v)))


def mul(a, b) -> np.float32:
    return round_f32(f(a) * f(b))


def fma(a, b, c) -> np.float32:
    return round_f32(f(a) * f(b) + f(c))


def sub(a, b) -> np.float32:
    return round_f32(f(a) - f(b))


def transform_axis(Rrow, t, mu) -> np.float32:
    """q = fma(R2, mu_z, fma(R1, mu_y, fma(R0, mu_x, t)))."""
    return fma(Rrow[2], mu[2], fma(Rrow[1], mu[1], fma(Rrow[0], mu[0], t)))


def key(coord, inv_r):
    """floor(coord * inv_r) with one FP32 multiply; None if outside [-2^20, 2^20)."""
    p = mul(coord, inv_r)
    k = int(np.floor(np.float64(p)))
    if k < -(1 << 20) or k >= (1 << 20):
        return None
    return k
