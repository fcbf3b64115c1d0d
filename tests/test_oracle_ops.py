"""Pins for the oracle's EFT primitives and K-component add/multiply.

The oracle restates Algorithms 1-14 (Section 2).  These tests check it against
things fixed independently of its code: exact rational arithmetic (Python
Fractions), the operation counts printed in Tables 1 and 2, the identity of
Algorithms 7 and 8, error bounds, the nonoverlap property, and algebraic
identities that exact round-to-nearest arithmetic guarantees.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from cases import families
from exact import mp_value, mp_values, rel_err, to_mp
from paper_2603_14926_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BF_PRECS = ["dd", "td", "qd", "ds", "tf", "qf"]
ALL_PRECS = ["dd", "ddc", "td", "qd", "ds", "tf", "qf"]


def prec_bits(oracle, prec):
    K, dt = oracle.PRECS[prec]
    return K * (53 if dt == np.float64 else 24)


# ---------------------------------------------------------------------------
# Algorithms 1-3
# ---------------------------------------------------------------------------

def _pairs(f32=False, n=4000, seed=1):
    rng = np.random.default_rng(seed)
    dt = np.float32 if f32 else np.float64
    a = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(dt)
    b = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(dt)
    edge = [(1.0, 1.0), (1.0, -1.0), (1.0, 2.0 ** -60), (2.0 ** -60, 1.0), (0.0, 3.0),
            (1.5, -1.5), (1 + 2.0 ** -52, -1.0), (3.0, 2.0 ** -52), (-0.0, 0.0)]
    ea = np.array([e[0] for e in edge], dtype=dt)
    eb = np.array([e[1] for e in edge], dtype=dt)
    return np.concatenate([a, ea]), np.concatenate([b, eb])


@pytest.mark.parametrize("f32", [False, True])
def test_two_sum_exact(oracle, f32):
    a, b = _pairs(f32)
    for x, y in zip(a, b):
        s, e = oracle.two_sum(float(x), float(y), f32)
        assert Fraction(s) + Fraction(e) == Fraction(float(x)) + Fraction(float(y))
        assert s == float(np.float32(float(x) + float(y))) if f32 else s == float(x) + float(y)


@pytest.mark.parametrize("f32", [False, True])
def test_quick_two_sum_exact_when_ordered(oracle, f32):
    a, b = _pairs(f32, seed=2)
    for x, y in zip(a, b):
        x, y = float(x), float(y)
        if abs(x) < abs(y):
            x, y = y, x
        s, e = oracle.quick_two_sum(x, y, f32)
        assert Fraction(s) + Fraction(e) == Fraction(x) + Fraction(y)


def test_quick_two_sum_needs_its_precondition(oracle):
    # |a| < |b|: the three-operation form loses the error term (Algorithm 1's
    # precondition); TwoSum (Algorithm 2) recovers it.
    a, b = 2.0 ** -60, 1.0 + 2.0 ** -52
    s, e = oracle.quick_two_sum(a, b)
    assert Fraction(s) + Fraction(e) != Fraction(a) + Fraction(b)
    s, e = oracle.two_sum(a, b)
    assert Fraction(s) + Fraction(e) == Fraction(a) + Fraction(b)


@pytest.mark.parametrize("f32", [False, True])
def test_two_prod_exact(oracle, f32):
    a, b = _pairs(f32, seed=3)
    for x, y in zip(a, b):
        p, e = oracle.two_prod(float(x), float(y), f32)
        assert Fraction(p) + Fraction(e) == Fraction(float(x)) * Fraction(float(y))


# ---------------------------------------------------------------------------
# Tables 1 and 2
# ---------------------------------------------------------------------------

def test_op_counts_match_tables(oracle):
    g = json.load(open(os.path.join(GOLDEN, "op_counts.json")))
    for name, row in g["rows"].items():
        add, sub, mul, div, fma = row["counts"]
        got = oracle.op_counts(row["prec"], row["op"])
        assert got == (add, sub, mul, fma), (name, got)
        assert div == 0
        f32 = {"td": "tf", "qd": "qf"}[row["prec"]]
        assert oracle.op_counts(f32, row["op"]) == got


def test_op_counts_double_word(oracle):
    # Algorithm 6: 2 TwoSum + 2 QuickTwoSum + 2 adds; Algorithm 4: TwoSum + 2 adds +
    # QuickTwoSum; Algorithms 7/8: TwoProd + 2 mul + 2 add + QuickTwoSum.
    assert oracle.op_counts("dd", "add") == (8, 12, 0, 0)
    assert oracle.op_counts("ddc", "add") == (5, 6, 0, 0)
    assert oracle.op_counts("dd", "mul") == (3, 2, 3, 1)
    assert oracle.op_counts("ddc", "mul") == (3, 2, 3, 1)


# ---------------------------------------------------------------------------
# Inputs: random nonoverlapping numbers, exponent gaps, near-cancellation, zeros
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", BF_PRECS)
@pytest.mark.parametrize("op", ["add", "mul"])
def test_relative_error_bound(oracle, prec, op):
    """|c - exact| <= 2^-(p-2) |exact| for add, 2^-(p-4) |exact| for mul, where
    p = K * (component precision): the bound adopted for the branch-free algorithms
    (the paper quotes no bound; observed maxima are about 2^-(p-1) and 2^-(p-3))."""
    p = prec_bits(oracle, prec)
    bound = 2.0 ** -(p - 2) if op == "add" else 2.0 ** -(p - 4)
    worst = 0.0
    for name, a, b in families(oracle, prec):
        if op == "mul" and name == "cancellation":
            continue
        c = getattr(oracle, op)(prec, a, b)
        for x, y, z in zip(mp_values(a), mp_values(b), mp_values(c)):
            ex = x + y if op == "add" else x * y
            e = rel_err(z, ex)
            worst = max(worst, e)
            assert e <= bound, (name, prec, op, e)
    assert worst > 0  # the inputs do exercise rounding


def test_sloppy_add_absolute_bound(oracle):
    """Algorithm 4 has no relative bound under cancellation; its error is
    bounded by 2^-104 (|a| + |b|)."""
    for name, a, b in families(oracle, "ddc"):
        c = oracle.add("ddc", a, b)
        for x, y, z in zip(mp_values(a), mp_values(b), mp_values(c)):
            assert abs(z - (x + y)) <= Fraction(1, 2 ** 104) * (abs(x) + abs(y)), name


def test_sloppy_add_loses_under_cancellation(oracle):
    """The accurate add (Algorithm 6) keeps a relative bound where the sloppy one
    (Algorithm 4) does not: both must see at least one such input."""
    fams = dict((n, (a, b)) for n, a, b in families(oracle, "ddc"))
    a, b = fams["cancellation"]
    cs = oracle.add("ddc", a, b)
    cb = oracle.add("dd", a, b)
    es = max(rel_err(z, x + y) for x, y, z in zip(mp_values(a), mp_values(b), mp_values(cs)))
    eb = max(rel_err(z, x + y) for x, y, z in zip(mp_values(a), mp_values(b), mp_values(cb)))
    assert eb <= 2.0 ** -104 and es > 2.0 ** -90


def test_dwmul_equals_dwbfmul(oracle):
    """Reading "QuickTwoProd" in Algorithm 7 as QuickTwoSum makes Algorithms 7 and 8
    the same sequence of operations: results must agree bit for bit."""
    for name, a, b in families(oracle, "dd", n=3000):
        assert np.array_equal(oracle.mul("ddc", a, b), oracle.mul("dd", a, b)), name


@pytest.mark.parametrize("prec", ALL_PRECS)
def test_nonoverlap(oracle, prec):
    """Weak nonoverlap for every component pair of every result: |c[j+1]| <= ulp(c[j]),
    and c[j] == 0 implies c[j+1] == 0; strict for the last pair, written by a final
    QuickTwoSum: fl(c[K-2] + c[K-1]) == c[K-2]."""
    K, dt = oracle.PRECS[prec]
    for name, a, b in families(oracle, prec):
        for op in ("add", "mul"):
            c = getattr(oracle, op)(prec, a, b)
            for j in range(K - 1):
                hi, lo = c[j].astype(np.float64), c[j + 1].astype(np.float64)
                ulp = np.spacing(np.abs(c[j])).astype(np.float64)
                assert np.all(np.abs(lo) <= ulp + (hi == 0) * 0), (name, op, j)
                assert np.all((hi != 0) | (lo == 0)), (name, op, j)
            s = (c[K - 2] + c[K - 1]).astype(dt)
            assert np.array_equal(s, c[K - 2]), (name, op)


@pytest.mark.parametrize("prec", ALL_PRECS)
def test_identities(oracle, prec):
    """Exact round-to-nearest arithmetic makes these hold bit for bit: a+0 = 0+a = a,
    a*1 = 1*a = a, a*2^-3 scales every component, a+(-a) = 0, add and mul commute,
    and both are odd under sign changes.  Commutativity fails for most wrongly
    wired operands (an A-side term paired with a B-side one)."""
    K, dt = oracle.PRECS[prec]
    for name, a, b in families(oracle, prec, n=1500, seed=7):
        z = np.zeros_like(a)
        one = np.zeros_like(a)
        one[0] = 1
        p2 = np.zeros_like(a)
        p2[0] = 0.125
        add, mul = oracle.add, oracle.mul
        assert np.array_equal(add(prec, a, z), a)
        assert np.array_equal(add(prec, z, a), a)
        assert np.array_equal(mul(prec, a, one), a)
        assert np.array_equal(mul(prec, one, a), a)
        assert np.array_equal(mul(prec, a, p2), (a * dt(0.125)).astype(dt))
        assert np.array_equal(add(prec, a, -a), z)
        assert np.array_equal(add(prec, a, b), add(prec, b, a)), name
        assert np.array_equal(mul(prec, a, b), mul(prec, b, a)), name
        assert np.array_equal(add(prec, -a, -b), -add(prec, a, b)), name
        assert np.array_equal(mul(prec, -a, b), -mul(prec, a, b)), name


def test_generator_nonoverlapping():
    for dt, mant in ((np.float64, 53), (np.float32, 24)):
        a = inputs.mp_uniform(0, 5000, 4, dt)
        for j in range(3):
            hi, lo = a[j].astype(np.float64), a[j + 1].astype(np.float64)
            assert np.all(np.abs(lo) <= np.where(hi == 0, 0, np.spacing(np.abs(a[j])) / 2))
        assert np.all(np.abs(a[0]) < 1)
        b = inputs.mp_uniform(0, 5000, 4, dt)
        assert np.array_equal(a, b)
