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




def strassen_one_level_entry(oracle, prec, A, B, i, j):
    """Entry (i, j) of one level of Strassen's recursion (Section 3.1; the seven
    products and four combinations of Strassen's original formulas) computed from
    the rows and columns that entry needs, with the oracle's add, negation-add and
    sequential-fold GEMM; quadrants are ceil-halves, zero-padded.  Equals entry
    (i, j) of oracle.gemm_strassen when exactly one level recurses (the leaves
    are the classical fold), so full-size Strassen products can be checked one
    entry at a time."""
    K = A.shape[0]
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    hm, hk, hn = (m + 1) // 2, (k + 1) // 2, (n + 1) // 2
    qi, qj = int(i >= hm), int(j >= hn)
    ii, jj = i - qi * hm, j - qj * hn

    def arow(r, c):  # row ii of quadrant A_rc (1-based quadrant indices), padded to hk
        out = np.zeros((K, 1, hk), dtype=A.dtype)
        gi, c0 = (r - 1) * hm + ii, (c - 1) * hk
        if gi < m:
            w = min(hk, k - c0)
            out[:, 0, :w] = A[:, gi, c0:c0 + w]
        return out

    def bcol(r, c):  # column jj of quadrant B_rc, padded to hk
        out = np.zeros((K, hk, 1), dtype=B.dtype)
        gj, r0 = (c - 1) * hn + jj, (r - 1) * hk
        if gj < n:
            w = min(hk, k - r0)
            out[:, :w, 0] = B[:, r0:r0 + w, gj]
        return out

    def add(x, y):
        return oracle.add(prec, x.reshape(K, -1), y.reshape(K, -1)).reshape(x.shape)

    def sub(x, y):
        return oracle.add(prec, x.reshape(K, -1), (-y).reshape(K, -1)).reshape(x.shape)

    def prod(s, t):
        return oracle.gemm(prec, s, t)[:, 0, 0]

    def comb(first, *rest):
        acc = first[:, None]
        for sign, v in rest:
            acc = (add if sign > 0 else sub)(acc, v[:, None])
        return acc[:, 0]

    if (qi, qj) == (0, 0):
        M1 = prod(add(arow(1, 1), arow(2, 2)), add(bcol(1, 1), bcol(2, 2)))
        M4 = prod(arow(2, 2), sub(bcol(2, 1), bcol(1, 1)))
        M5 = prod(add(arow(1, 1), arow(1, 2)), bcol(2, 2))
        M7 = prod(sub(arow(1, 2), arow(2, 2)), add(bcol(2, 1), bcol(2, 2)))
        return comb(M1, (1, M4), (-1, M5), (1, M7))
    if (qi, qj) == (0, 1):
        M3 = prod(arow(1, 1), sub(bcol(1, 2), bcol(2, 2)))
        M5 = prod(add(arow(1, 1), arow(1, 2)), bcol(2, 2))
        return comb(M3, (1, M5))
    if (qi, qj) == (1, 0):
        M2 = prod(add(arow(2, 1), arow(2, 2)), bcol(1, 1))
        M4 = prod(arow(2, 2), sub(bcol(2, 1), bcol(1, 1)))
        return comb(M2, (1, M4))
    M1 = prod(add(arow(1, 1), arow(2, 2)), add(bcol(1, 1), bcol(2, 2)))
    M2 = prod(add(arow(2, 1), arow(2, 2)), bcol(1, 1))
    M3 = prod(arow(1, 1), sub(bcol(1, 2), bcol(2, 2)))
    M6 = prod(sub(arow(2, 1), arow(1, 1)), add(bcol(1, 1), bcol(1, 2)))
    return comb(M1, (-1, M2), (1, M3), (1, M6))
