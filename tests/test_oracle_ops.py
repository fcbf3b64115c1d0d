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
ALL_PRECS = ["dd", "ddc", "td", "qd", "tdc", "qdc", "ds", "tf", "qf"]
CONV_PRECS = ["tdc", "qdc"]


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
# Conventional triple and quad word (Tables 1 and 2, the renormalising rows)
# ---------------------------------------------------------------------------

# building blocks as (add, sub, mul, fma): Algorithms 1-3 and the plain operations
TS, QTS, TP, ADD_, MUL_ = (2, 4, 0, 0), (1, 2, 0, 0), (0, 0, 1, 1), (1, 0, 0, 0), (0, 0, 1, 0)


def _blocks(**n):
    parts = {"ts": TS, "qts": QTS, "tp": TP, "add": ADD_, "mul": MUL_}
    return tuple(sum(n.get(k, 0) * v[i] for k, v in parts.items()) for i in range(4))


def _typical(oracle, prec):
    K, dt = oracle.PRECS[prec]
    return (inputs.mp_uniform(0, 1, K, dt, stream=41), inputs.mp_uniform(0, 1, K, dt, stream=42))


def test_conventional_tw_mul_counts_match_table1(oracle):
    """Algorithm 10 (six TwoProds, sixteen TwoSums, five adds) plus TWRenormalize
    (five QuickTwoSums on every path) gives Table 1's TWxTW row exactly, on a
    typical input and on one whose lower components are zero."""
    g = json.load(open(os.path.join(GOLDEN, "op_counts.json")))["conventional_rows"]
    add, sub, mul, div, fma = g["TWxTW"]["counts"]
    assert div == 0
    assert _blocks(tp=6, ts=16, add=5, qts=5) == (add, sub, mul, fma)
    assert oracle.op_counts("tdc", "mul") == (add, sub, mul, fma)
    assert oracle.op_counts("tdc", "mul", *_typical(oracle, "tdc")) == (add, sub, mul, fma)


def test_conventional_tw_add_counts_against_table1(oracle):
    """Algorithm 9 as printed: three written-out TwoSums, four TwoSums, two adds,
    then TWRenormalize (five QuickTwoSums, the count Table 1's TWxTW row fixes).
    That is one TwoSum (2 adds, 4 subtractions) more than Table 1's TW+TW row,
    which matches Algorithm 9 with its last TwoSum replaced by a plain add; the
    algorithm is followed as printed."""
    g = json.load(open(os.path.join(GOLDEN, "op_counts.json")))["conventional_rows"]
    add, sub, mul, _, fma = g["TW+TW"]["counts"]
    want = _blocks(ts=7, add=2, qts=5)
    assert want == (add + 2, sub + 4, mul, fma)
    assert oracle.op_counts("tdc", "add") == want
    assert oracle.op_counts("tdc", "add", *_typical(oracle, "tdc")) == want


def test_conventional_qw_counts(oracle):
    """The QD library's quad-word add (ten TwoSums, three adds) and accurate
    multiply (ten TwoProds, three products, twenty TwoSums, eighteen adds), each
    with QWRenormalize: four QuickTwoSums, then three more, or two and an add
    when every error term is nonzero (the typical path).  Table 2's QWxQW row
    has the same 94 subtractions on the seven-QuickTwoSum path.  Its QW+QW row
    (26 adds, 58 subtractions) cannot come from TwoSums, QuickTwoSums and plain
    adds at all, since each of these has at most twice as many subtractions as
    additions."""
    g = json.load(open(os.path.join(GOLDEN, "op_counts.json")))["conventional_rows"]
    assert oracle.op_counts("qdc", "add") == _blocks(ts=10, add=3, qts=7)
    assert oracle.op_counts("qdc", "add", *_typical(oracle, "qdc")) == _blocks(ts=10, add=4, qts=6)
    assert oracle.op_counts("qdc", "mul") == _blocks(tp=10, mul=3, ts=20, add=18, qts=7)
    assert oracle.op_counts("qdc", "mul", *_typical(oracle, "qdc")) == _blocks(tp=10, mul=3, ts=20, add=19,
                                                                               qts=6)
    assert oracle.op_counts("qdc", "mul")[1] == g["QWxQW"]["counts"][1]
    add, sub = g["QW+QW"]["counts"][:2]
    assert sub > 2 * add


@pytest.mark.parametrize("prec", CONV_PRECS)
@pytest.mark.parametrize("op", ["add", "mul"])
def test_conventional_error_bound(oracle, prec, op):
    """The renormalising algorithms keep the same adopted bounds as the
    branch-free ones (2^-(p-2) relative for add and 2^-(p-4) for multiply); the
    accurate multiply keeps every term down to order eps^4 and is held to
    2^-(p-2).  Observed: add 2^-(p+2), multiply 2^-(p+0.6) (TD) and 2^-(p+3) (QD)."""
    p = prec_bits(oracle, prec)
    bound = 2.0 ** -(p - 2)
    worst = 0.0
    for name, a, b in families(oracle, prec):
        c = getattr(oracle, op)(prec, a, b)
        for x, y, z in zip(mp_values(a), mp_values(b), mp_values(c)):
            e = rel_err(z, x + y if op == "add" else x * y)
            worst = max(worst, e)
            assert e <= bound, (name, prec, op, e)
    assert worst > 0


@pytest.mark.parametrize("prec", CONV_PRECS)
def test_conventional_agrees_with_branch_free(oracle, prec):
    """Both families approximate the same exact result: conventional and
    branch-free sums and products differ by no more than their two bounds."""
    bf = prec[:-1]
    p = prec_bits(oracle, prec)
    for name, a, b in families(oracle, prec, n=300, seed=3):
        for op in ("add", "mul"):
            c1 = mp_values(getattr(oracle, op)(prec, a, b))
            c2 = mp_values(getattr(oracle, op)(bf, a, b))
            for x, y in zip(c1, c2):
                assert abs(x - y) <= Fraction(2) ** -(p - 5) * max(abs(x), abs(y)), (name, op)


def test_renormalisation_compacts_exact_sums(oracle):
    """Sums whose exact value needs fewer components than K come out with the
    zeros last (the zero tests of the renormalisation): 1 + 2^-k in QD, and
    products of two one-component numbers, which TwoProd makes exact."""
    K = 4
    for k in (1, 30, 60, 110, 170):
        a = np.zeros((K, 1))
        b = np.zeros((K, 1))
        a[0, 0] = 1.0
        b[0, 0] = 2.0 ** -k
        for prec in ("qdc", "tdc"):
            Kp = oracle.PRECS[prec][0]
            c = oracle.add(prec, a[:Kp], b[:Kp])
            assert mp_value(c[:, 0]) == 1 + Fraction(2) ** -k
            nz = [float(v) != 0 for v in c[:, 0]]
            assert nz == sorted(nz, reverse=True), (prec, k, c[:, 0])
    rng = np.random.default_rng(4)
    for prec in CONV_PRECS:
        Kp = oracle.PRECS[prec][0]
        a = np.zeros((Kp, 50))
        b = np.zeros((Kp, 50))
        a[0] = rng.standard_normal(50)
        b[0] = rng.standard_normal(50)
        c = oracle.mul(prec, a, b)
        for i in range(50):
            assert mp_value(c[:, i]) == Fraction(float(a[0, i])) * Fraction(float(b[0, i]))
            assert not c[2:, i].any()


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
