"""Input families shared by the oracle pins and the GPU parity tests."""

from fractions import Fraction

import numpy as np

from exact import mp_value, to_mp
from paper_2603_14926_gb300 import inputs


def families(oracle, prec, n=600, seed=0, limits=False):
    """(name, a, b) pairs of K-arrays: random nonoverlapping numbers, exponent gaps,
    near-cancellation (b = -(a + eps) re-expanded exactly), zero lower components;
    with limits=True (binary64 only) also operands near the ends of the binary64
    range, where intermediate error terms are subnormal or sums approach overflow
    (no error bound of the paper applies there; the GPU must still reproduce the
    oracle's bits)."""
    K, dt = oracle.PRECS[prec]
    f32 = dt == np.float32
    rng = np.random.default_rng(100 + seed)
    out = []
    a = inputs.mp_uniform(seed, n, K, dt, stream=41)
    b = inputs.mp_uniform(seed, n, K, dt, stream=42)
    out.append(("random", a, b))
    gap = rng.integers(-12, 13, n) if f32 else rng.integers(-60, 61, n)
    out.append(("exponent-gap", a, (b * np.exp2(gap)).astype(dt)))
    # near-cancellation: b = -(a + eps) re-expanded exactly into K components
    m = n // 3
    eps = inputs.mp_uniform(seed, m, K, dt, stream=43)
    sh = rng.integers(5, 40 if f32 else 150, m)
    bb = np.zeros((K, m), dtype=dt)
    for i in range(m):
        q = -(mp_value(a[:, i]) + mp_value(eps[:, i]) * Fraction(2) ** int(-sh[i]))
        bb[:, i] = to_mp(q, K, dt)
    out.append(("cancellation", a[:, :m].copy(), bb))
    z = b.copy()
    z[1:, : n // 4] = 0
    z[2:, n // 4: n // 2] = 0
    out.append(("zero-components", a, z))
    if limits and not f32:
        lo, hi = a.copy(), b.copy()
        lo[:, 0::3] *= 2.0 ** -1000
        lo[:, 1::3] *= 2.0 ** 1000
        hi[:, 1::3] *= 2.0 ** 22
        hi[:, 2::3] *= 2.0 ** -60
        out.append(("range-limits", lo, hi))
    return out


