"""Plant plausible transcription mistakes in the oracle (on the CPU) and check
that its pins catch every one.

Each mutant edits one line of the oracle's C source: a wrong operand, TwoSum
swapped for QuickTwoSum, a dropped term, a swapped component index, a sign
slip, transposed GEMM indices, an off-by-one Horner coefficient, a Newton sign
error, a Durand-Kerner product that includes j = i, a mis-wired Estrin tree, a
Strassen product, combination or quadrant gone wrong, a dropped term, wrong
partner or component in the conventional triple- and quad-word algorithms or
their renormalisation.
The pin battery below
(exact rationals, the op counts of Tables 1 and 2, error bounds, identities,
permutation GEMM, known roots) must pass on the real oracle and fail on every
mutant.
"""

import json
import os
from fractions import Fraction

import numpy as np
import pytest

from cases import families
from exact import SCALE_BITS, mp_ints, mp_value, mp_values, rel_err
from paper_2603_14926_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CORE, DK = "mpref_core.inc", "mpref_dk.inc"

MUTANTS = [
    ("Alg13 wrong operand", CORE, "b2 = ADD(b1, h1);", "b2 = ADD(b1, f1);"),
    ("Alg13 dropped term", CORE, "e8 = ADD(e6, g3);", "e8 = e6;"),
    ("Alg13 TwoSum->QuickTwoSum", CORE, "F(two_sum)(b5, c4, &b6, &c6);", "F(quick_two_sum)(b5, c4, &b6, &c6);"),
    ("Alg13 swapped final operands", CORE, "F(quick_two_sum)(c11, d10, &r2, &r3);",
     "F(quick_two_sum)(d10, c11, &r2, &r3);"),
    ("Alg14 component index", CORE, "F(two_prod)(A[1], B[1], &h0, &k0);", "F(two_prod)(A[1], B[0], &h0, &k0);"),
    ("Alg14 dropped term", CORE, "f3 = ADD(f2, m2);", "f3 = f2;"),
    ("Alg14 wrong low product", CORE, "m0 = MUL(A[0], B[3]);", "m0 = MUL(A[0], B[2]);"),
    ("Alg14 wrong partner", CORE, "F(two_sum)(e2, g1, &e3, &g3);", "F(two_sum)(e2, i1, &e3, &g3);"),
    ("Alg12 dropped term", CORE, "g2 = ADD(g1, h0);", "g2 = g1;"),
    ("Alg12 TwoSum->QuickTwoSum", CORE, "g1 = ADD(g0, i0);\n    F(two_sum)(b0, c1, &b2, &c2);",
     "g1 = ADD(g0, i0);\n    F(quick_two_sum)(b0, c1, &b2, &c2);"),
    ("Alg11 dropped term", CORE, "c7 = ADD(c6, d5);", "c7 = c6;"),
    ("Alg11 wrong operand", CORE, "c4 = ADD(c3, e2);", "c4 = ADD(c3, d2);"),
    ("Alg6 dropped term", CORE, "g5 = ADD(g4, g3e);", "g5 = g4;"),
    ("Alg8 component index", CORE, "p10 = MUL(A[1], B[0]);", "p10 = MUL(A[1], B[1]);"),
    ("Alg4 dropped low sum", CORE, "REAL t = ADD(A[1], B[1]);\n    e = ADD(e, t);", "REAL t = ADD(A[1], B[1]);\n    e = ADD(e, 0 * t);"),
    ("Alg9 dropped term", CORE, "t0 = ADD(ADD(t0, t1), t2);", "t0 = ADD(t0, t1);"),
    ("Alg9 wrong partner", CORE, "F(two_sum)(t1, i1, &s2, &i3);", "F(two_sum)(t0, i1, &s2, &i3);"),
    ("Alg10 component index", CORE, "x[4], o[4];\n    F(two_prod)(A[0], B[0], &p0, &q0);\n    F(two_prod)(A[0], B[1], &p1, &q1);\n    F(two_prod)(A[1], B[0], &p2, &q2);\n    F(two_prod)(A[0], B[2], &p3, &q3);\n    F(two_prod)(A[1], B[1], &p4, &q4);",
     "x[4], o[4];\n    F(two_prod)(A[0], B[0], &p0, &q0);\n    F(two_prod)(A[0], B[1], &p1, &q1);\n    F(two_prod)(A[1], B[0], &p2, &q2);\n    F(two_prod)(A[0], B[2], &p3, &q3);\n    F(two_prod)(A[1], B[0], &p4, &q4);"),
    ("Alg10 wrong renormalisation input", CORE, "x[0] = p0; x[1] = p1; x[2] = s0; x[3] = t0;\n    F(renorm)(x, 4, 4, o);",
     "x[0] = p0; x[1] = p1; x[2] = p2; x[3] = t0;\n    F(renorm)(x, 4, 4, o);"),
    ("QW add dropped term", CORE, "t[0] = ADD(ADD(t[0], t[1]), t[3]);", "t[0] = ADD(t[0], t[1]);"),
    ("QW mul wrong eps^3 product", CORE, "F(two_prod)(A[3], B[0], &p9, &q9);", "F(two_prod)(A[3], B[1], &p9, &q9);"),
    ("Renormalisation drops the last term", CORE, "r = ADD(r, t[i]);\n            continue;", "continue;"),
    ("Renormalisation sweep operand order", CORE, "F(quick_two_sum)(x[i], s, &s, &t[i + 1]);",
     "F(quick_two_sum)(s, x[i], &s, &t[i + 1]);"),
    ("TwoSum wrong operand", CORE, "REAL t3 = SUB(b, v);", "REAL t3 = SUB(b, s_);"),
    ("TwoProd sign", CORE, "*e = FMA(a, b, -p_);", "*e = FMA(a, b, p_);"),
    ("QuickTwoSum order", CORE, "REAL t = SUB(s_, a);\n    *e = SUB(b, t);", "REAL t = SUB(s_, b);\n    *e = SUB(a, t);"),
    ("GEMM transposed index", CORE, "int64_t ib = opB ? (j * ldb + l) : (l * ldb + j);",
     "int64_t ib = opB ? (j * ldb + l) : (j * ldb + l);"),
    ("Horner off-by-one", CORE, "        F(load)(P, coef, pc, i, a);\n        P->mul(h, x, h);",
     "        F(load)(P, coef, pc, i + 1, a);\n        P->mul(h, x, h);"),
    ("Newton sign", CORE, "        F(mp_sub)(P, one, t, e);", "        F(mp_sub)(P, t, one, e);"),
    ("Estrin lo/hi swapped", CORE, "                P->mul(hi_r, pr, t1);\n                P->add(t1, lo_r, vr + 4 * j);",
     "                P->mul(lo_r, pr, t1);\n                P->add(t1, hi_r, vr + 4 * j);"),
    ("Estrin lost pass-through", CORE, "                vr[4 * half + c] = vr[4 * (len - 1) + c];",
     "                vr[4 * half + c] = 0;"),
    ("Estrin power doubled, not squared", CORE, "                P->mul(pr, pr, pr);", "                P->add(pr, pr, pr);"),
    ("Strassen M4 operands swapped", CORE, "T = F(msum)(P, B21, B11, nb, 1);", "T = F(msum)(P, B11, B21, nb, 1);"),
    ("Strassen C22 sign", CORE, "F(load)(P, M[2], nc, t, b); F(mp_sub)(P, a, b, a);",
     "F(load)(P, M[2], nc, t, b); P->add(a, b, a);"),
    ("Strassen quadrant offset", CORE, "*A21 = F(block)(P, A, lda, pA, m, k, hm, 0, hm, hk)",
     "*A21 = F(block)(P, A, lda, pA, m, k, hm - 1, 0, hm, hk)"),
    ("DK product includes j == i", DK, "                if (j == i) continue;\n                load_d(P, z, pz, j, zjr);",
     "                load_d(P, z, pz, j, zjr);"),
    ("DK wrong update sign", DK, "            mp_sub_d(P, zr, wr, yr);", "            P->add(zr, wr, yr);"),
]


def battery(oracle):
    """Run a compact set of the oracle's pins; return the names of those that fail
    (a pin that raises, e.g. on a NaN result, counts as failed)."""
    bad = []
    for part in (_counts_and_eft, _ops, _blas_poly, _roots):
        try:
            part(oracle, bad)
        except Exception as e:  # noqa: BLE001 -- any exception is a caught mutant
            bad.append(f"{part.__name__}: {type(e).__name__}")
    return bad


def _counts_and_eft(oracle, bad):

    def check(name, ok):
        if not ok and name not in bad:
            bad.append(name)

    # Tables 1 and 2 and the double-word counts
    g = json.load(open(os.path.join(GOLDEN, "op_counts.json")))
    for row in g["rows"].values():
        a, s, m, _, f = row["counts"]
        check("op counts", oracle.op_counts(row["prec"], row["op"]) == (a, s, m, f))
    check("op counts", oracle.op_counts("dd", "add") == (8, 12, 0, 0))
    check("op counts", oracle.op_counts("ddc", "add") == (5, 6, 0, 0))
    check("op counts", oracle.op_counts("dd", "mul") == (3, 2, 3, 1))
    conv = g["conventional_rows"]
    a, s, m, _, f = conv["TWxTW"]["counts"]
    check("op counts", oracle.op_counts("tdc", "mul") == (a, s, m, f))
    a, s, m, _, f = conv["TW+TW"]["counts"]
    check("op counts", oracle.op_counts("tdc", "add") == (a + 2, s + 4, m, f))
    check("op counts", oracle.op_counts("qdc", "add") == (30, 54, 0, 0))
    check("op counts", oracle.op_counts("qdc", "mul") == (65, 94, 13, 10))
    # EFT exactness
    rng = np.random.default_rng(0)
    xs = rng.standard_normal(200) * np.exp2(rng.integers(-20, 20, 200))
    ys = rng.standard_normal(200) * np.exp2(rng.integers(-20, 20, 200))
    for x, y in zip(xs, ys):
        s, e = oracle.two_sum(float(x), float(y))
        check("TwoSum exact", Fraction(s) + Fraction(e) == Fraction(float(x)) + Fraction(float(y)))
        p, e = oracle.two_prod(float(x), float(y))
        check("TwoProd exact", Fraction(p) + Fraction(e) == Fraction(float(x)) * Fraction(float(y)))
        big, small = (x, y) if abs(x) >= abs(y) else (y, x)
        s, e = oracle.quick_two_sum(float(big), float(small))
        check("QuickTwoSum exact", Fraction(s) + Fraction(e) == Fraction(float(big)) + Fraction(float(small)))


def _check(bad):
    def check(name, ok):
        if not ok and name not in bad:
            bad.append(name)
    return check


def _ops(oracle, bad):
    check = _check(bad)
    # per-op error bounds and identities
    for prec in ("dd", "ddc", "td", "qd", "tdc", "qdc", "tf", "qf"):
        K, dt = oracle.PRECS[prec]
        p = K * (53 if dt == np.float64 else 24)
        for name, a, b in families(oracle, prec, n=120, seed=5):
            for op in ("add", "mul"):
                if op == "mul" and name == "cancellation":
                    continue
                c = getattr(oracle, op)(prec, a, b)
                for x, y, z in zip(mp_values(a), mp_values(b), mp_values(c)):
                    ex = x + y if op == "add" else x * y
                    if prec == "ddc" and op == "add":
                        check("sloppy add bound", abs(z - ex) <= Fraction(1, 2 ** 104) * (abs(x) + abs(y)))
                    else:
                        lim = 2.0 ** -(p - 2) if op == "add" or prec in ("tdc", "qdc") else 2.0 ** -(p - 4)
                        check(f"{op} error bound", rel_err(z, ex) <= lim)
            check("commutativity", np.array_equal(oracle.add(prec, a, b), oracle.add(prec, b, a)))
            check("commutativity", np.array_equal(oracle.mul(prec, a, b), oracle.mul(prec, b, a)))
    a, b = families(oracle, "dd", n=300)[0][1:]
    check("Alg7 == Alg8", np.array_equal(oracle.mul("ddc", a, b), oracle.mul("dd", a, b)))


def _blas_poly(oracle, bad):
    check = _check(bad)
    # GEMM vs exact and under a column permutation
    K = 4
    A = inputs.mp_uniform(1, (6, 5), K)
    B = inputs.mp_uniform(2, (5, 7), K)
    C = oracle.gemm("qd", A, B)
    ex = mp_ints(A).dot(mp_ints(B))
    Ci = mp_ints(C)
    for i in range(6):
        for j in range(7):
            err = abs(Ci[i, j] * (1 << SCALE_BITS) - ex[i, j])
            check("GEMM vs exact", float(Fraction(err, 1 << (2 * SCALE_BITS))) <= 2.0 ** -200)
    perm = np.array([2, 0, 4, 1, 3])
    Pm = np.zeros((K, 5, 5))
    Pm[0, np.arange(5), perm] = 1
    want = np.zeros_like(A)
    want[:, :, perm] = A
    check("GEMM permutation", np.array_equal(oracle.gemm("qd", A, Pm), want))
    # Strassen on integer matrices (odd sizes, three levels): exact
    rng = np.random.default_rng(12)
    Ai = np.zeros((K, 13, 11))
    Bi = np.zeros((K, 11, 9))
    Ai[0] = rng.integers(-40, 41, (13, 11))
    Bi[0] = rng.integers(-40, 41, (11, 9))
    Cs = oracle.gemm_strassen("qd", Ai, Bi, 3)
    check("Strassen exact", np.array_equal(Cs[0], Ai[0] @ Bi[0]) and not Cs[1:].any())
    # Horner vs exact
    off = np.array([0, 9], dtype=np.int64)
    coef = inputs.mp_uniform(3, 9, K, stream=inputs.STREAM_C)
    xv = inputs.mp_uniform(4, 3, K, stream=inputs.STREAM_X)
    y = oracle.polyeval("qd", off, coef, 3, xv)
    cv = mp_values(coef)
    for m in range(3):
        x = mp_value(xv[:, m])
        ex = sum(cv[i] * x ** i for i in range(9))
        check("Horner vs exact", abs(mp_value(y[:, m]) - ex) <= Fraction(2) ** -200)
    # Estrin on exactly representable cases (integer coefficients, x = 2 and -3/2)
    rng = np.random.default_rng(11)
    for n in (4, 5, 6, 7, 12):
        a = rng.integers(-15, 16, n + 1)
        cf = np.zeros((K, n + 1))
        cf[0] = a
        for xq in (Fraction(2), Fraction(-3, 2)):
            xe = np.zeros((K, 1))
            xe[0, 0] = float(xq)
            ye = oracle.polyeval_estrin("qd", np.array([0, n + 1], dtype=np.int64), cf, 1, xe)
            check("Estrin exact", mp_value(ye[:, 0]) == sum(int(a[i]) * xq ** i for i in range(n + 1)))
    # reciprocal
    r = oracle.recip("qd", xv)
    for v, w in zip(mp_values(xv), mp_values(r)):
        check("recip bound", abs(v * w - 1) <= Fraction(2) ** -206)


def _roots(oracle, bad):
    check = _check(bad)
    # Durand-Kerner on exactly known roots
    prob = inputs.dk_problem_from_roots([([0.5 + 0.25j, -0.75 + 0.5j], -0.125)])
    c = oracle.poly_from_roots("qd", prob)
    rr, it, st = oracle.roots("qd", prob.coef_off, c)
    check("DK known roots", st[0] in (1, 2))
    got = [complex(float(mp_value(rr[:4, j])), float(mp_value(rr[4:, j]))) for j in range(5)]
    want_r = list(prob.roots_of(0))
    check("DK known roots", all(min(abs(g_ - w) for w in want_r) < 1e-30 for g_ in got))


def test_battery_passes_on_the_oracle(oracle):
    assert battery(oracle) == []


@pytest.mark.parametrize("name,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle, name, fname, old, new):
    with oracle.mutant([(fname, old, new)]):
        failed = battery(oracle)
    assert failed, f"mutant '{name}' survived every pin"
