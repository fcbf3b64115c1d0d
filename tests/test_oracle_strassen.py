"""Pins for the oracle's Strassen recursion (Section 3.1's matrix-multiplication
scheme, Strassen's seven products, zero padding for odd sizes).

- Integer matrices: every product, sum and difference is exact, so any cutoff
  and any padding must give the exact integer product; a wrong sign, operand or
  quadrant in any of the seven products or four combinations does not.
- A cutoff above min(m, n, k) is the classical fold itself.
- Random nonoverlapping entries: the result is within a Strassen-type bound of
  the exact product and is not the classical fold's bits (the recursion ran).
- The Eq. 1 matrices at cutoff 32: at least the accuracy the paper prints for
  its Strassen runs (29.0 / 45.5 / 61.7 decimal digits, DD / TD / QD).
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from exact import SCALE_BITS, isqrt_frac, mp_ints, mp_value, to_mp
from paper_2603_14926_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def int_matrix(rng, shape, K, dt, lim=40):
    X = np.zeros((K,) + shape, dtype=dt)
    X[0] = rng.integers(-lim, lim + 1, shape)
    return X


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "tf", "qf"])
@pytest.mark.parametrize("m,n,k,cutoff", [(7, 7, 7, 2), (13, 9, 11, 3), (33, 20, 17, 4), (16, 16, 16, 2),
                                          (5, 12, 9, 2), (40, 40, 40, 5)])
def test_strassen_exact_on_integer_matrices(oracle, prec, m, n, k, cutoff):
    K, dt = oracle.PRECS[prec]
    rng = np.random.default_rng(m * 1000 + n * 10 + k)
    A = int_matrix(rng, (m, k), K, dt)
    B = int_matrix(rng, (k, n), K, dt)
    C = oracle.gemm_strassen(prec, A, B, cutoff)
    exact = A[0].astype(np.int64) @ B[0].astype(np.int64)
    got = mp_ints(C)
    assert all(got[i, j] == int(exact[i, j]) << SCALE_BITS for i in range(m) for j in range(n))


@pytest.mark.parametrize("prec", ["dd", "qd", "qf"])
def test_strassen_cutoff_above_sizes_is_classical(oracle, prec):
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(1, (9, 12), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(2, (12, 10), K, dt, stream=inputs.STREAM_B)
    assert np.array_equal(oracle.gemm_strassen(prec, A, B, 10), oracle.gemm(prec, A, B))


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_strassen_random_within_bound(oracle, prec):
    """n = 40 at cutoff 5: three levels (40 -> 20 -> 10 -> 5).  Each level at most
    doubles the operands' magnitudes in its sums and adds up to four products, so
    |C - AB| <= 2^-p (n + 16) 8^L n max|a| max|b| with room to spare; a wrong
    formula errs by O(max|a| max|b|)."""
    K, dt = oracle.PRECS[prec]
    n, cutoff, L = 40, 5, 3
    A = inputs.mp_uniform(3, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(4, (n, n), K, dt, stream=inputs.STREAM_B)
    C = oracle.gemm_strassen(prec, A, B, cutoff)
    assert not np.array_equal(C, oracle.gemm(prec, A, B))
    exact = mp_ints(A).dot(mp_ints(B))
    Ci = mp_ints(C)
    amax = float(np.abs(A[0]).max()) * 1.01
    bmax = float(np.abs(B[0]).max()) * 1.01
    p = K * 53
    bound = 2.0 ** -p * (n + 16) * 8 ** L * n * amax * bmax
    worst = 0.0
    for i in range(n):
        for j in range(n):
            err = float(Fraction(abs(Ci[i, j] * (1 << SCALE_BITS) - exact[i, j]), 1 << (2 * SCALE_BITS)))
            worst = max(worst, err)
    assert 0 < worst <= bound, (worst, bound)


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
@pytest.mark.parametrize("n", [65, 96])
def test_strassen_eq1_accuracy_digits(oracle, prec, n):
    """Eq. 1 matrices a_ij = sqrt5 (i+j-1), b_ij = sqrt3 (n-i+1) at the paper's
    cutoff 32 (two levels here; n = 65 pads at both): at least the lower end of
    the digits Section 3.1 reports for its Strassen runs, at most the format's."""
    g = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    lo, _ = g["real_gemm_digits"][prec]
    K, dt = oracle.PRECS[prec]
    s5 = to_mp(isqrt_frac(Fraction(5), 400), K)
    s3 = to_mp(isqrt_frac(Fraction(3), 400), K)
    ints = np.zeros((K, 2 * n), dtype=dt)
    ints[0] = np.arange(2 * n)
    r5 = oracle.mul(prec, np.repeat(s5[:, None], 2 * n, 1), ints)
    r3 = oracle.mul(prec, np.repeat(s3[:, None], 2 * n, 1), ints)
    I, J = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    A = np.ascontiguousarray(r5[:, I + J - 1])
    B = np.ascontiguousarray(r3[:, n - I + 1])
    C = oracle.gemm_strassen(prec, A, B, 32)
    s15 = isqrt_frac(Fraction(15), 400)
    digits = math.inf
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            S = (i - 1) * n * (n + 1) // 2 + sum(k * (n - k + 1) for k in range(1, n + 1))
            ex = s15 * S
            digits = min(digits, -math.log10(float(abs(mp_value(C[:, i - 1, j - 1]) - ex) / ex)))
    assert digits >= lo, digits
    assert digits <= K * 53 * math.log10(2) + 1.5, digits


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "qdc"])
@pytest.mark.parametrize("shape", [(65, 65, 65), (70, 67, 69), (64, 66, 65)])
def test_one_level_entry_helper_matches_recursion(oracle, prec, shape):
    """The entry-at-a-time form of one Strassen level (tests/cases.py), used to
    check full-size GPU products one entry at a time, equals the oracle's
    recursion bit for bit in every quadrant, odd and even sizes."""
    from cases import strassen_one_level_entry

    m, n, k = shape
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(31, (m, k), K, dt)
    B = inputs.mp_uniform(32, (k, n), K, dt)
    cutoff = min(shape)  # one level: the halves drop below it
    C = oracle.gemm_strassen(prec, A, B, cutoff)
    for i, j in [(0, 0), (0, n - 1), (m - 1, 0), (m - 1, n - 1), (m // 2, n // 2), (3, 40), (40, 3)]:
        got = strassen_one_level_entry(oracle, prec, A, B, i, j)
        assert np.array_equal(got.view(np.uint64), C[:, i, j].view(np.uint64)), (i, j)
