"""Exact-rational float32 helpers for pinning the oracle's quantization.

fma(a, b, c) is defined by IEEE 754 as the exact a*b + c rounded once to the
nearest float32 (ties to even); these helpers compute it with Fractions, a
technique independent of the oracle's std::fmaf.
"""
from fractions import Fraction
import math

import numpy as np


def f32_round(fr: Fraction) -> np.float32:
    """Nearest float32 to an exact rational, ties to even."""
    c = np.float32(float(fr))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    best = None
    for cand in cands:
        d = abs(Fraction(float(cand)) - fr)
        even = (int(np.float32(cand).view(np.uint32)) & 1) == 0
        if best is None or d < best[0] or (d == best[0] and even):
            best = (d, cand)
    return np.float32(best[1])


def fma32(a, b, c) -> np.float32:
    return f32_round(Fraction(float(np.float32(a))) * Fraction(float(np.float32(b)))
                     + Fraction(float(np.float32(c))))


def quantize_axis(v, scale, offset, bits) -> int:
    f = math.floor(float(fma32(v, scale, offset)))
    return min(max(f, 0), (1 << bits) - 1)


def quantize_query_axis(v, scale, offset) -> int:
    f = math.floor(float(fma32(v, scale, offset)))
    return min(max(f, -(1 << 30)), 1 << 30)


def transform(xform12, p):
    R = [np.float32(v) for v in xform12[:9]]
    t = [np.float32(v) for v in xform12[9:]]
    out = []
    for r in range(3):
        inner = fma32(R[3 * r + 2], p[2], t[r])
        mid = fma32(R[3 * r + 1], p[1], inner)
        out.append(fma32(R[3 * r + 0], p[0], mid))
    return out
