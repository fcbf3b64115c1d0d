"""Pins for the oracle's AXPY, dot, GEMV and GEMM (sequential folds).

Checked against exact results (big-integer long accumulators over the exact
component values), exact special cases (permutation and power-of-two diagonal
matrices, transposed storage), and the accuracy the paper prints for the Eq. 1
test matrices (Section 3.1).
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


def pbits(oracle, prec):
    K, dt = oracle.PRECS[prec]
    return K * (53 if dt == np.float64 else 24)


def reduction_bound(n, p):
    """|fold - exact| <= (4n + 16) 2^-p sum |x_k y_k|: one multiply (<= 2^-(p-4)
    relative) per term plus one add (<= 2^-(p-2) relative to the partial sum) per step."""
    return (4 * n + 16) * 2.0 ** -p


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd"])
def test_gemm_vs_exact_config0(oracle, prec):
    """QD GEMM n = 64 on the seed-0 nonoverlapping generator, every entry vs exact."""
    K, dt = oracle.PRECS[prec]
    n = 64
    A = inputs.mp_uniform(0, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(0, (n, n), K, dt, stream=inputs.STREAM_B)
    C = oracle.gemm(prec, A, B)
    Ai, Bi, Ci = mp_ints(A), mp_ints(B), mp_ints(C)
    exact = Ai.dot(Bi)  # value * 2^(2 SCALE_BITS)
    absA = np.abs(A.astype(np.float64)).sum(0)
    absB = np.abs(B.astype(np.float64)).sum(0)
    mag = absA @ absB
    p = pbits(oracle, prec)
    bound = reduction_bound(n, p) if prec != "ddc" else reduction_bound(n, p) * 4
    worst = 0.0
    for i in range(n):
        for j in range(n):
            err = abs(Ci[i, j] * (1 << SCALE_BITS) - exact[i, j])
            e = float(Fraction(err, 1 << (2 * SCALE_BITS))) / mag[i, j]
            worst = max(worst, e)
            assert e <= bound, (i, j, e)
    assert worst > 0


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "tf", "qf"])
def test_gemm_permutation_and_scaling_exact(oracle, prec):
    """A P and P A permute A exactly; A diag(2^e) scales columns exactly (add(x,0) = x
    and mul(x,1) = x hold bit for bit).  Fails for swapped indices or operands."""
    K, dt = oracle.PRECS[prec]
    m, k = 13, 9
    rng = np.random.default_rng(5)
    A = inputs.mp_uniform(3, (m, k), K, dt)
    perm = rng.permutation(k)
    P = np.zeros((K, k, k), dtype=dt)
    P[0, np.arange(k), perm] = 1  # P[i, perm[i]] = 1: (A P)[:, perm[i]] = A[:, i]
    AP = oracle.gemm(prec, A, P)
    want = np.zeros_like(A)
    want[:, :, perm] = A
    assert np.array_equal(AP, want)
    permr = rng.permutation(m)
    Q = np.zeros((K, m, m), dtype=dt)
    Q[0, np.arange(m), permr] = 1  # (Q A)[i] = A[permr[i]]
    assert np.array_equal(oracle.gemm(prec, Q, A), A[:, permr, :])
    e = rng.integers(-5, 6, k)
    D = np.zeros((K, k, k), dtype=dt)
    D[0, np.arange(k), np.arange(k)] = np.exp2(e)
    assert np.array_equal(oracle.gemm(prec, A, D), (A * np.exp2(e)[None, None, :]).astype(dt))


@pytest.mark.parametrize("prec", ["dd", "qd", "qf"])
def test_gemm_transposed_storage(oracle, prec):
    """op(X) = X^T reads the transposed storage: same fold, same bits."""
    K, dt = oracle.PRECS[prec]
    m, n, k = 7, 11, 5
    A = inputs.mp_uniform(1, (m, k), K, dt)
    B = inputs.mp_uniform(2, (k, n), K, dt)
    C = oracle.gemm(prec, A, B)
    At = np.ascontiguousarray(A.transpose(0, 2, 1))
    Bt = np.ascontiguousarray(B.transpose(0, 2, 1))
    assert np.array_equal(oracle.gemm(prec, At, B, opA=1), C)
    assert np.array_equal(oracle.gemm(prec, A, Bt, opB=1), C)
    assert np.array_equal(oracle.gemm(prec, At, Bt, opA=1, opB=1), C)
    # row ranges used by the CPU-baseline sample
    assert np.array_equal(oracle.gemm(prec, A, B, rows=(2, 5)), C[:, 2:5])
    assert np.array_equal(oracle.gemm(prec, At, B, opA=1, rows=(2, 5)), C[:, 2:5])


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_gemm_eq1_accuracy_digits(oracle, prec):
    """Eq. 1 matrices a_ij = sqrt5 (i+j-1), b_ij = sqrt3 (n-i+1): the paper reports
    29.0-30.4 / 45.5-47.5 / 61.7-63.5 correct decimal digits for DD/TD/QD
    (Section 3.1).  The classical fold at n = 48 must reach at least the lower end
    and cannot exceed the format's precision."""
    g = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    lo, hi = g["real_gemm_digits"][prec]
    K, dt = oracle.PRECS[prec]
    n = 48
    s5 = to_mp(isqrt_frac(Fraction(5), 400), K)
    s3 = to_mp(isqrt_frac(Fraction(3), 400), K)
    ints = np.zeros((K, 2 * n), dtype=dt)
    ints[0] = np.arange(2 * n)
    s5v = np.repeat(s5[:, None], 2 * n, 1)
    s3v = np.repeat(s3[:, None], 2 * n, 1)
    r5 = oracle.mul(prec, s5v, ints)  # sqrt5 * t, t = 0 .. 2n-1
    r3 = oracle.mul(prec, s3v, ints)
    I, J = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    A = r5[:, I + J - 1]
    B = r3[:, n - I + 1]
    C = oracle.gemm(prec, A, B)
    s15 = isqrt_frac(Fraction(15), 400)
    digits = math.inf
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            S = sum((i + k - 1) * (n - k + 1) for k in range(1, n + 1))
            ex = s15 * S
            got = mp_value(C[:, i - 1, j - 1])
            digits = min(digits, -math.log10(float(abs(got - ex) / ex)))
    assert digits >= lo, digits
    assert digits <= K * 53 * math.log10(2) + 1.5, digits


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "ds", "qf"])
def test_dot_gemv_axpy_vs_exact(oracle, prec):
    K, dt = oracle.PRECS[prec]
    p = pbits(oracle, prec)
    n = 700
    x = inputs.mp_uniform(11, n, K, dt, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(11, n, K, dt, stream=inputs.STREAM_Y)
    xi, yi = mp_ints(x), mp_ints(y)
    s = oracle.dot(prec, x, y)
    exact = int(xi.dot(yi))
    mag = float(np.abs(x.astype(np.float64)).sum(0) @ np.abs(y.astype(np.float64)).sum(0))
    err = abs(int(mp_ints(s[:, None])[0]) * (1 << SCALE_BITS) - exact)
    assert float(Fraction(err, 1 << (2 * SCALE_BITS))) <= reduction_bound(n, p) * mag
    # gemv
    m = 9
    A = inputs.mp_uniform(12, (m, n), K, dt)
    yv = oracle.gemv(prec, A, x)
    Ai = mp_ints(A)
    absA = np.abs(A.astype(np.float64)).sum(0)
    absx = np.abs(x.astype(np.float64)).sum(0)
    for i in range(m):
        ex = int(Ai[i].dot(xi))
        got = int(mp_ints(yv[:, i:i + 1])[0])
        e = float(Fraction(abs(got * (1 << SCALE_BITS) - ex), 1 << (2 * SCALE_BITS)))
        assert e <= reduction_bound(n, p) * float(absA[i] @ absx)
        # gemv row == dot of the row (same fold)
        assert np.array_equal(yv[:, i], oracle.dot(prec, A[:, i, :], x))
    # axpy: one multiply and one add per element
    alpha = inputs.mp_uniform(13, 1, K, dt)[:, 0]
    r = oracle.axpy(prec, alpha, x, y)
    ai = mp_ints(alpha[:, None])[0]
    ri = mp_ints(r)
    for i in range(n):
        ex = ai * xi[i] + yi[i] * (1 << SCALE_BITS)
        e = abs(ri[i] * (1 << SCALE_BITS) - ex)
        magi = abs(float(alpha[0]) * float(x[0, i])) + abs(float(y[0, i]))
        assert float(Fraction(e, 1 << (2 * SCALE_BITS))) <= 2.0 ** -(p - 5) * magi * 1.01


@pytest.mark.parametrize("prec", ["qd"])
def test_reductions_edge_cases(oracle, prec):
    K, dt = oracle.PRECS[prec]
    z = np.zeros((K, 0), dtype=dt)
    assert np.array_equal(oracle.dot(prec, z, z), np.zeros(K))
    A = inputs.mp_uniform(1, (3, 4), K, dt)
    B = np.zeros((K, 4, 0), dtype=dt)
    assert oracle.gemm(prec, A, B).shape == (K, 3, 0)
    E = np.zeros((K, 3, 0), dtype=dt)
    F = np.zeros((K, 0, 5), dtype=dt)
    assert np.array_equal(oracle.gemm(prec, E, F), np.zeros((K, 3, 5)))


def eq2_matrices(oracle, prec, seed, n):
    """Eq. 2 entries U * exp(r_n), the product formed with the oracle's multiply."""
    K, dt = oracle.PRECS[prec]
    Ur, Er, Ui, Ei = inputs.complex_eq2(seed, (n, n), K, dt)
    mk = lambda U, E: oracle.mul(prec, U.reshape(K, -1),  # noqa: E731
                                 inputs.mp_from_double(E.reshape(-1), K, dt)).reshape(K, n, n)
    return mk(Ur, Er), mk(Ui, Ei)


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_cgemm3m_vs_exact_and_paper_digits(oracle, prec):
    """3M complex GEMM (Eq. 3) on Eq. 2 matrices.  Every entry within the bound of
    its three real products and two subtractions; the worst entry keeps at least
    the lower end of the digits the paper reports (Section 3.2: DD 23.2, TD 39.2,
    QD 55.8 -- measured there with Strassen up to n = 2049) and no more than the
    format holds."""
    g = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    lo, hi = g["complex_gemm_digits"][prec]
    K = oracle.PRECS[prec][0]
    p = pbits(oracle, prec)
    n = 32
    Ar, Ai = eq2_matrices(oracle, prec, 1, n)
    Br, Bi = eq2_matrices(oracle, prec, 2, n)
    Cr, Ci = oracle.cgemm(prec, Ar, Ai, Br, Bi)
    iar, iai, ibr, ibi = (mp_ints(x) for x in (Ar, Ai, Br, Bi))
    er = iar.dot(ibr) - iai.dot(ibi)
    ei = iar.dot(ibi) + iai.dot(ibr)
    f = lambda X: np.abs(X.astype(np.float64)).sum(0)  # noqa: E731
    sa, sb = f(Ar) + f(Ai), f(Br) + f(Bi)
    mag = sa @ sb  # bounds |Re A||Re B| + |Im A||Im B| + |Re A + Im A||Re B + Im B| sums
    digits = math.inf
    for got, ex in ((mp_ints(Cr), er), (mp_ints(Ci), ei)):
        for i in range(n):
            for j in range(n):
                e = abs(got[i, j] * (1 << SCALE_BITS) - ex[i, j])
                assert float(Fraction(e, 1 << (2 * SCALE_BITS))) <= 3 * reduction_bound(n, p) * mag[i, j]
                if e:
                    digits = min(digits, -math.log10(float(Fraction(e, abs(ex[i, j])))))
    assert lo <= digits <= K * 53 * math.log10(2) + 1.5, digits


def test_cgemm3m_structure(oracle):
    """Re C = C1 - C2 and Im C = (C3 - C1) - C2 with C1, C2, C3 the oracle's real GEMMs,
    in transposed storage too; a real input (Im = 0) reduces to the real GEMM."""
    prec, K = "qd", 4
    m, n, k = 5, 7, 6
    Ar, Ai = inputs.mp_uniform(1, (m, k), K), inputs.mp_uniform(2, (m, k), K)
    Br, Bi = inputs.mp_uniform(3, (k, n), K), inputs.mp_uniform(4, (k, n), K)
    Cr, Ci = oracle.cgemm(prec, Ar, Ai, Br, Bi)
    C1 = oracle.gemm(prec, Ar, Br)
    C2 = oracle.gemm(prec, Ai, Bi)
    C3 = oracle.gemm(prec, oracle.add(prec, Ar, Ai), oracle.add(prec, Br, Bi))
    assert np.array_equal(Cr, oracle.add(prec, C1, -C2))
    assert np.array_equal(Ci, oracle.add(prec, oracle.add(prec, C3, -C1), -C2))
    tr = lambda X: np.ascontiguousarray(X.transpose(0, 2, 1))  # noqa: E731
    Tr, Ti = oracle.cgemm(prec, tr(Ar), tr(Ai), tr(Br), tr(Bi), opA=1, opB=1)
    assert np.array_equal(Tr, Cr) and np.array_equal(Ti, Ci)
    Z = np.zeros_like(Ai)
    Rr, Ri = oracle.cgemm(prec, Ar, Z, Br, np.zeros_like(Bi))
    assert np.array_equal(Rr, oracle.gemm(prec, Ar, Br)) and not np.any(Ri)
