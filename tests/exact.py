"""Exact rational helpers for the tests (no multicomponent arithmetic here).

Every binary64/binary32 value is a dyadic rational, so sums and products of
components are exact as Python Fractions or as big integers at a common scale.
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

SCALE_BITS = 1100  # every binary64 value (>= 2^-1074) times 2^1100 is an integer


def frac(x) -> Fraction:
    return Fraction(float(x))


def mp_value(col) -> Fraction:
    """Exact value of one K-component number (iterable of components)."""
    return sum((Fraction(float(c)) for c in col), Fraction(0))


def mp_values(arr) -> list:
    """Exact values of a K-array of shape (K, n)."""
    a = np.asarray(arr)
    return [mp_value(a[:, i]) for i in range(a.shape[1])]


def to_int(x: float) -> int:
    """x * 2^SCALE_BITS as an exact integer."""
    num, den = float(x).as_integer_ratio()
    return num * ((1 << SCALE_BITS) // den)


def mp_ints(arr) -> np.ndarray:
    """Object array of exact integers: value * 2^SCALE_BITS, shape arr.shape[1:]."""
    a = np.asarray(arr, dtype=np.float64)
    flat = a.reshape(a.shape[0], -1)
    out = np.empty(flat.shape[1], dtype=object)
    for i in range(flat.shape[1]):
        out[i] = sum(to_int(c) for c in flat[:, i])
    return out.reshape(a.shape[1:])


def int_to_float(v: int, scale_bits: int) -> float:
    """v / 2^scale_bits, correctly rounded."""
    return v / (1 << scale_bits) if v.bit_length() < 1000 else float(Fraction(v, 1 << scale_bits))


def rel_err(approx: Fraction, exact: Fraction) -> float:
    if exact == 0:
        return 0.0 if approx == 0 else math.inf
    return float(abs(approx - exact) / abs(exact))


def to_mp(q: Fraction, K: int, dtype=np.float64) -> np.ndarray:
    """Greedy K-component expansion of a rational: c_j = round(q - sum_{i<j} c_i)."""
    out = np.zeros(K, dtype=dtype)
    r = Fraction(q)
    for j in range(K):
        c = dtype(float(r)) if dtype is np.float64 else np.float32(float(r))
        out[j] = c
        r -= Fraction(float(c))
    return out


def isqrt_frac(q: Fraction, bits: int) -> Fraction:
    """sqrt(q) truncated to `bits` fractional bits (q >= 0)."""
    s = 2 * bits
    v = (q.numerator << s) // q.denominator
    return Fraction(math.isqrt(v), 1 << bits)
