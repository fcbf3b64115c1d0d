"""Pins for the oracle's polynomial evaluation (Section 4.1), its adjoint,
the reciprocal, the Aberth starting values (Eq. 5) and the Durand-Kerner
iteration (Eq. 4), against exact rational arithmetic, closed forms and
finite differences.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

from exact import isqrt_frac, mp_value, mp_values, to_mp
from paper_2603_14926_gb300 import inputs

DPRECS = ["dd", "ddc", "td", "qd"]


def pbits(oracle, prec):
    return oracle.PRECS[prec][0] * 53


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def poly_problem(seed, npoly, dmin, dmax, K, dt=np.float64):
    """Random real coefficients (generator numbers) with ragged degrees."""
    rng = np.random.default_rng(seed)
    deg = rng.integers(dmin, dmax + 1, npoly)
    off = np.zeros(npoly + 1, dtype=np.int64)
    np.cumsum(deg + 1, out=off[1:])
    coef = inputs.mp_uniform(seed, int(off[-1]), K, dt, stream=inputs.STREAM_C)
    return off, coef


# ---------------------------------------------------------------------------
# Horner
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["dd", "td", "qd", "qf"])
def test_horner_real_and_complex_vs_exact(oracle, prec):
    K, dt = oracle.PRECS[prec]
    p = K * (53 if dt == np.float64 else 24)
    npts = 7
    off, coef = poly_problem(1, 5, 0, 17, K, dt)
    npoly = len(off) - 1
    xr = inputs.mp_uniform(2, npoly * npts, K, dt, stream=inputs.STREAM_X)
    xi = inputs.mp_uniform(3, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    yr = oracle.polyeval(prec, off, coef, npts, xr)
    cr, ci = oracle.polyeval(prec, off, coef, npts, xr, xi)
    cv = mp_values(coef)
    for b in range(npoly):
        a = cv[off[b]:off[b + 1]]
        n = len(a) - 1
        for m in range(npts):
            idx = b * npts + m
            x = mp_value(xr[:, idx])
            z = (x, mp_value(xi[:, idx]))
            ex = sum(a[i] * x ** i for i in range(n + 1))
            mag = sum(abs(a[i]) * abs(x) ** i for i in range(n + 1))
            bound = Fraction(8 * n + 16) * Fraction(2) ** -p * mag
            assert abs(mp_value(yr[:, idx]) - ex) <= bound
            # exact complex value
            h = (Fraction(0), Fraction(0))
            for i in range(n, -1, -1):
                h = cmul(h, z)
                h = (h[0] + a[i], h[1])
            zabs = abs(complex(float(z[0]), float(z[1])))
            magc = sum(abs(float(a[i])) * zabs ** i for i in range(n + 1))
            bc = (16 * n + 16) * 2.0 ** -p * magc
            assert float(abs(mp_value(cr[:, idx]) - h[0])) <= bc
            assert float(abs(mp_value(ci[:, idx]) - h[1])) <= bc
            # real Horner == complex Horner at zero imaginary part
        yr0, yi0 = oracle.polyeval(prec, off, coef, npts, xr, np.zeros_like(xr))
        assert np.array_equal(yr0, yr)
        assert not np.any(yi0)


# ---------------------------------------------------------------------------
# Estrin
# ---------------------------------------------------------------------------

def _estrin_exact_cases(prec, dt):
    """(n, a, x) with small integer coefficients where every value any evaluation
    order forms is exactly representable in one component of the type."""
    bits = 50 if dt == np.float64 else 22
    rng = np.random.default_rng(7)
    for n in range(0, 41):
        a = [int(v) for v in rng.integers(-15, 16, n + 1)]
        for x in (Fraction(2), Fraction(-2), Fraction(1, 2), Fraction(-3, 2)):
            # numerators over the common denominator stay below 2^bits
            num = 15 * sum(abs(x.numerator) ** i * x.denominator ** (n - i) for i in range(n + 1))
            top = abs(x.numerator) ** (1 << max(0, (n).bit_length()))
            if num < 2 ** bits and top < 2 ** bits:
                yield n, a, x


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "qf"])
def test_estrin_exact_on_representable_cases(oracle, prec):
    """Integer coefficients at x in {2, -2, 1/2, -3/2} (and x = 1 + i below): every
    intermediate of any order is exact, so the result must be the exact value.  A
    wrong pairing, power or pass-through of the tree changes it."""
    K, dt = oracle.PRECS[prec]
    count = 0
    for n, a, x in _estrin_exact_cases(prec, dt):
        cf = np.zeros((K, n + 1), dtype=dt)
        cf[0] = a
        xe = np.zeros((K, 1), dtype=dt)
        xe[0, 0] = float(x)
        y = oracle.polyeval_estrin(prec, np.array([0, n + 1], dtype=np.int64), cf, 1, xe)
        assert mp_value(y[:, 0]) == sum(a[i] * x ** i for i in range(n + 1)), (n, x)
        count += 1
    assert count > 40
    # complex argument 1 + i: Gaussian integers
    for n in range(0, 21 if dt == np.float64 else 9):
        a = [int(v) for v in np.random.default_rng(n).integers(-15, 16, n + 1)]
        cf = np.zeros((K, n + 1), dtype=dt)
        cf[0] = a
        one = np.zeros((K, 1), dtype=dt)
        one[0, 0] = 1.0
        yr, yi = oracle.polyeval_estrin(prec, np.array([0, n + 1], dtype=np.int64), cf, 1, one, one)
        h = (Fraction(0), Fraction(0))
        for i in range(n, -1, -1):
            h = cmul(h, (Fraction(1), Fraction(1)))
            h = (h[0] + a[i], h[1])
        assert (mp_value(yr[:, 0]), mp_value(yi[:, 0])) == h, n


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "qf"])
def test_estrin_vs_exact_and_horner(oracle, prec):
    """Random coefficients and points: within the evaluation bound of the exact
    value (real and complex arguments); degrees 0 and 1 equal Horner bit for bit
    (the same single operation)."""
    K, dt = oracle.PRECS[prec]
    p = K * (53 if dt == np.float64 else 24)
    npts = 5
    off, coef = poly_problem(21, 7, 0, 40, K, dt)
    npoly = len(off) - 1
    xr = inputs.mp_uniform(22, npoly * npts, K, dt, stream=inputs.STREAM_X)
    xi = inputs.mp_uniform(23, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    yr = oracle.polyeval_estrin(prec, off, coef, npts, xr)
    cr, ci = oracle.polyeval_estrin(prec, off, coef, npts, xr, xi)
    cv = mp_values(coef)
    for b in range(npoly):
        a = cv[off[b]:off[b + 1]]
        n = len(a) - 1
        for m in range(npts):
            idx = b * npts + m
            x = mp_value(xr[:, idx])
            z = (x, mp_value(xi[:, idx]))
            ex = sum(a[i] * x ** i for i in range(n + 1))
            mag = sum(abs(a[i]) * abs(x) ** i for i in range(n + 1))
            assert abs(mp_value(yr[:, idx]) - ex) <= Fraction(8 * n + 16) * Fraction(2) ** -p * mag
            h = (Fraction(0), Fraction(0))
            for i in range(n, -1, -1):
                h = cmul(h, z)
                h = (h[0] + a[i], h[1])
            zabs = abs(complex(float(z[0]), float(z[1])))
            bc = (16 * n + 16) * 2.0 ** -p * sum(abs(float(a[i])) * zabs ** i for i in range(n + 1))
            assert float(abs(mp_value(cr[:, idx]) - h[0])) <= bc
            assert float(abs(mp_value(ci[:, idx]) - h[1])) <= bc
    low = np.array([0, 1, 3, 4], dtype=np.int64)  # degrees 0, 1, 0
    cl = inputs.mp_uniform(24, 4, K, dt, stream=inputs.STREAM_C)
    xl = inputs.mp_uniform(25, 3 * npts, K, dt, stream=inputs.STREAM_X)
    assert np.array_equal(oracle.polyeval_estrin(prec, low, cl, npts, xl), oracle.polyeval(prec, low, cl, npts, xl))


# ---------------------------------------------------------------------------
# Adjoint of Horner evaluation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_polyeval_backward_vs_exact(oracle, prec):
    K, dt = oracle.PRECS[prec]
    p = pbits(oracle, prec)
    npts = 6
    off, coef = poly_problem(4, 4, 0, 12, K)
    npoly = len(off) - 1
    x = inputs.mp_uniform(5, npoly * npts, K, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(6, npoly * npts, K, stream=inputs.STREAM_Y)
    dc, dx = oracle.polyeval_backward(prec, off, coef, npts, x, dy)
    cv, xv, gv = mp_values(coef), mp_values(x), mp_values(dy)
    for b in range(npoly):
        a = cv[off[b]:off[b + 1]]
        n = len(a) - 1
        for i in range(n + 1):
            ex = sum(gv[b * npts + m] * xv[b * npts + m] ** i for m in range(npts))
            mag = sum(abs(gv[b * npts + m]) * abs(xv[b * npts + m]) ** i for m in range(npts))
            bound = Fraction(4 * (npts + i) + 16) * Fraction(2) ** -p * mag
            assert abs(mp_value(dc[:, off[b] + i]) - ex) <= bound
        for m in range(npts):
            idx = b * npts + m
            xx = xv[idx]
            der = sum(i * a[i] * xx ** (i - 1) for i in range(1, n + 1))
            magd = sum(i * abs(a[i]) * abs(xx) ** (i - 1) for i in range(1, n + 1))
            bound = Fraction(8 * n + 32) * Fraction(2) ** -p * magd * abs(gv[idx])
            assert abs(mp_value(dx[:, idx]) - gv[idx] * der) <= bound


def test_polyeval_backward_finite_differences(oracle):
    """QD central differences, h = 2^-70: truncation ~h^2, rounding ~2^-212/h."""
    prec, K = "qd", 4
    npts = 5
    off, coef = poly_problem(8, 3, 3, 20, K)
    npoly = len(off) - 1
    x = inputs.mp_uniform(9, npoly * npts, K, stream=inputs.STREAM_X)
    dy = np.zeros((K, npoly * npts))
    dy[0] = 1.0
    dc, dx = oracle.polyeval_backward(prec, off, coef, npts, x, dy)
    h = np.zeros_like(x)
    h[0] = 2.0 ** -70
    yp = oracle.polyeval(prec, off, coef, npts, oracle.add(prec, x, h))
    ym = oracle.polyeval(prec, off, coef, npts, oracle.add(prec, x, -h))
    fd = oracle.add(prec, yp, -ym) * 2.0 ** 69
    for idx in range(npoly * npts):
        scale = 1 + abs(float(dx[0, idx]))
        assert abs(float(mp_value(fd[:, idx]) - mp_value(dx[:, idx]))) <= 2.0 ** -120 * scale
    # coefficient gradient: p is linear in a, so differences are exact up to rounding
    for b in range(npoly):
        for i in (0, int(off[b + 1] - off[b]) - 1):
            e = np.zeros_like(coef)
            e[0, off[b] + i] = 2.0 ** -70
            yp = oracle.polyeval(prec, off, oracle.add(prec, coef, e), npts, x)
            ym = oracle.polyeval(prec, off, oracle.add(prec, coef, -e), npts, x)
            fd = oracle.add(prec, yp, -ym) * 2.0 ** 69
            g = sum(mp_value(fd[:, b * npts + m]) for m in range(npts))
            assert abs(float(g - mp_value(dc[:, off[b] + i]))) <= 2.0 ** -120


# ---------------------------------------------------------------------------
# Reciprocal and the elementary functions of the starting values
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", DPRECS + ["tf", "qf"])
def test_recip_bound(oracle, prec):
    K, dt = oracle.PRECS[prec]
    p = K * (53 if dt == np.float64 else 24)
    x = inputs.mp_uniform(21, 400, K, dt)
    x = x * np.exp2(np.arange(400) % 41 - 20).astype(dt)
    r = oracle.recip(prec, x)
    for xv, rv in zip(mp_values(x), mp_values(r)):
        if xv == 0:
            continue
        assert abs(rv * xv - 1) <= Fraction(2) ** -(p - 6)


def test_dk_cos_sin_and_nthroot(oracle):
    for th in np.linspace(0, 2 * math.pi, 997, endpoint=False):
        c, s = oracle.dk_cos_sin(float(th))
        assert abs(c - math.cos(th)) < 1e-14 and abs(s - math.sin(th)) < 1e-14
    rng = np.random.default_rng(0)
    for v, m in zip(np.exp2(rng.uniform(-300, 300, 500)), rng.integers(1, 600, 500)):
        r = oracle.dk_nthroot(float(v), int(m))
        want = math.exp(math.log(v) / m)
        assert abs(r / want - 1) < 1e-13, (v, m)
    assert oracle.dk_nthroot(8.0, 3) == pytest.approx(2.0, rel=1e-15)


# ---------------------------------------------------------------------------
# Polynomials from roots (the root-solving workload's builder)
# ---------------------------------------------------------------------------

def exact_poly(prob, b, magnitude=False):
    """Exact coefficients of polynomial b; with magnitude=True those of
    prod (x + |r|) (x^2 + 2|Re r| x + |r|^2), which bound every partial product."""
    n = int(prob.degrees[b])
    d = prob.rootdata[prob.root_off[b]:prob.root_off[b + 1]]
    poly = [Fraction(1)]
    sgn = 1 if magnitude else -1
    if n % 2:
        r = Fraction(float(d[n - 1]))
        poly = [sgn * (abs(r) if magnitude else r) * poly[0], poly[0]]
    for k in range(n // 2):
        re, im = Fraction(float(d[2 * k])), Fraction(float(d[2 * k + 1]))
        B, C = (2 * abs(re) if magnitude else -2 * re), re * re + im * im
        new = [Fraction(0)] * (len(poly) + 2)
        for i, c in enumerate(poly):
            new[i] += C * c
            new[i + 1] += B * c
            new[i + 2] += c
        poly = new
    if magnitude:
        return poly
    dl = prob.delta[prob.root_off[b]:prob.root_off[b + 1]]
    return [c * (1 + Fraction(float(dl[i]))) if i < n else c for i, c in enumerate(poly)]


@pytest.mark.parametrize("prec", DPRECS)
def test_poly_from_roots_vs_exact(oracle, prec):
    K = oracle.PRECS[prec][0]
    p = pbits(oracle, prec)
    prob = inputs.dk_problem(3, 6, 1, 14)
    coef = oracle.poly_from_roots(prec, prob)
    assert coef.shape == (K, int(prob.coef_off[-1]))
    for b in range(prob.npoly):
        ex = exact_poly(prob, b)
        n = len(ex) - 1
        absprob = exact_poly(prob, b, magnitude=True)
        got = mp_values(coef[:, prob.coef_off[b]:prob.coef_off[b + 1]])
        assert got[n] == 1
        for i in range(n + 1):
            assert abs(got[i] - ex[i]) <= Fraction(16 * n + 16) * Fraction(2) ** -p * absprob[i]


# ---------------------------------------------------------------------------
# Aberth starting values (Eq. 5)
# ---------------------------------------------------------------------------

def test_aberth_matches_formula(oracle):
    prob = inputs.dk_problem(5, 4, 5, 40)
    coef = oracle.poly_from_roots("qd", prob)
    for b in range(prob.npoly):
        c = coef[:, prob.coef_off[b]:prob.coef_off[b + 1]]
        n = c.shape[1] - 1
        z = oracle.aberth("qd", c)
        lead = c[0]
        nnz = int(np.count_nonzero(lead[:n]))
        r = max(abs(nnz * lead[i]) ** (1.0 / (n - i)) for i in range(n) if lead[i] != 0)
        i = np.arange(1, n + 1)
        want = -lead[n - 1] / n + r * np.exp(1j * (2 * (i - 1) * np.pi / n + 3 / (2 * n)))
        assert np.allclose(z[0], want.real, rtol=0, atol=1e-12 * (1 + r))
        assert np.allclose(z[4], want.imag, rtol=0, atol=1e-12 * (1 + r))
        assert not np.any(z[1:4]) and not np.any(z[5:8])


# ---------------------------------------------------------------------------
# Durand-Kerner (Eq. 4)
# ---------------------------------------------------------------------------

def roots_of(oracle, prec, r, K, lo, hi):
    re = np.array([float(mp_value(r[:K, j])) for j in range(lo, hi)])
    im = np.array([float(mp_value(r[K:, j])) for j in range(lo, hi)])
    return re + 1j * im


def match_sets(a, b):
    """Greedy nearest matching; returns the largest distance."""
    b = list(b)
    worst = 0.0
    for x in a:
        d = [abs(x - y) for y in b]
        k = int(np.argmin(d))
        worst = max(worst, d[k])
        b.pop(k)
    return worst


@pytest.mark.parametrize("prec", DPRECS)
def test_dk_known_roots(oracle, prec):
    K = oracle.PRECS[prec][0]
    p = pbits(oracle, prec)
    cases = [([], 2.0), ([1j], None), ([0.5 + 0.25j, -0.75 + 0.5j], -0.125),
             ([0.3 + 0.4j, 0.3 - 0.9j, -0.6 + 0.1j], 0.7)]
    prob = inputs.dk_problem_from_roots(cases)
    coef = oracle.poly_from_roots(prec, prob)
    r, iters, st = oracle.roots(prec, prob.coef_off, coef)
    assert np.all(st == oracle.DK_CONVERGED), st
    for b in range(prob.npoly):
        lo, hi = prob.root_off[b], prob.root_off[b + 1]
        got = [(mp_value(r[:K, j]), mp_value(r[K:, j])) for j in range(lo, hi)]
        want = list(prob.roots_of(b))
        for g in got:
            gz = complex(float(g[0]), float(g[1]))
            k = int(np.argmin([abs(gz - w) for w in want]))
            w = want.pop(k)
            err = abs(g[0] - Fraction(w.real)) + abs(g[1] - Fraction(w.imag))
            tol = 2.0 ** -(p - 12) if prec != "ddc" else 2.0 ** -(p - 16)
            assert float(err) <= tol, (b, float(err))


@pytest.mark.parametrize("prec", ["td", "qd"])
def test_dk_chebyshev_small(oracle, prec):
    """Chebyshev quadrature nodes: n = 2 gives x^2 - 1/3 (nodes +-1/sqrt3), n = 3 gives
    x^3 - x/2 (nodes 0, +-1/sqrt2); coefficients rounded to K components."""
    K = oracle.PRECS[prec][0]
    p = pbits(oracle, prec)
    c2 = np.stack([to_mp(Fraction(-1, 3), K), np.zeros(K), to_mp(Fraction(1), K)], 1)
    c3 = np.stack([np.zeros(K), to_mp(Fraction(-1, 2), K), np.zeros(K), to_mp(Fraction(1), K)], 1)
    coef = np.concatenate([c2, c3], 1)
    off = np.array([0, 3, 7])
    r, it, st = oracle.roots(prec, off, coef)
    assert np.all(st == oracle.DK_CONVERGED)
    s3 = isqrt_frac(Fraction(1, 3), 300)
    s2 = isqrt_frac(Fraction(1, 2), 300)
    want = [[s3, -s3], [Fraction(0), s2, -s2]]
    rof = [0, 2, 5]
    for b in range(2):
        got = sorted(mp_value(r[:K, j]) for j in range(rof[b], rof[b + 1]))
        for g, w in zip(got, sorted(want[b])):
            assert float(abs(g - w)) <= 2.0 ** -(p - 8)
        assert all(abs(float(mp_value(r[K:, j]))) <= 2.0 ** -(p - 8) for j in range(rof[b], rof[b + 1]))


def test_dk_one_step_vs_exact(oracle):
    """One Jacobi step (max_iter = 1) from the Aberth values equals the exact
    rational update z - q(z) / prod_{j != i} (z - z_j) within rounding."""
    prec, K = "qd", 4
    prob = inputs.dk_problem(9, 1, 7, 7)
    coef = oracle.poly_from_roots(prec, prob)
    z0 = oracle.aberth(prec, coef)
    r, it, st = oracle.roots(prec, prob.coef_off, coef, max_iter=1)
    assert it[0] == 1 and st[0] == oracle.DK_CAP
    a = mp_values(coef)
    z = [(mp_value(z0[:K, i]), mp_value(z0[K:, i])) for i in range(7)]
    for i in range(7):
        q = (Fraction(0), Fraction(0))
        for c in reversed(a):
            q = cmul(q, z[i])
            q = (q[0] + c, q[1])
        den = (Fraction(1), Fraction(0))
        for j in range(7):
            if j != i:
                den = cmul(den, (z[i][0] - z[j][0], z[i][1] - z[j][1]))
        d2 = den[0] ** 2 + den[1] ** 2
        w = cmul(q, (den[0], -den[1]))
        new = (z[i][0] - w[0] / d2, z[i][1] - w[1] / d2)
        err = abs(mp_value(r[:K, i]) - new[0]) + abs(mp_value(r[K:, i]) - new[1])
        assert float(err) <= 2.0 ** -190 * (1 + float(abs(w[0] / d2) + abs(w[1] / d2)))


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_dk_random_backward_error_and_planted_roots(oracle, prec):
    K = oracle.PRECS[prec][0]
    p = pbits(oracle, prec)
    prob = inputs.dk_problem(3, 6, 10, 30)
    coef = oracle.poly_from_roots(prec, prob)
    r, it, st = oracle.roots(prec, prob.coef_off, coef)
    # a rounding floor above tol ends the iteration as "stagnated": quality is judged
    # by the backward error below
    assert np.all((st == oracle.DK_CONVERGED) | (st == oracle.DK_STAGNATED)), st
    for b in range(prob.npoly):
        a = mp_values(coef[:, prob.coef_off[b]:prob.coef_off[b + 1]])
        n = len(a) - 1
        lo = prob.root_off[b]
        for j in range(lo, lo + n):
            z = (mp_value(r[:K, j]), mp_value(r[K:, j]))
            q = (Fraction(0), Fraction(0))
            for c in reversed(a):
                q = cmul(q, z)
                q = (q[0] + c, q[1])
            za = abs(complex(float(z[0]), float(z[1])))
            mag = sum(abs(float(c)) * za ** i for i, c in enumerate(a))
            res = math.hypot(float(q[0]), float(q[1]))
            assert res <= (32 * n) * 2.0 ** -p * mag, (b, j, res, mag)
        got = roots_of(oracle, prec, r, K, lo, lo + n)
        assert match_sets(got, prob.roots_of(b)) < 1e-12


def test_dk_status_cases(oracle):
    prec, K = "td", 3
    prob = inputs.dk_problem(4, 3, 12, 20)
    coef = oracle.poly_from_roots(prec, prob)
    r, it, st = oracle.roots(prec, prob.coef_off, coef, max_iter=3)
    assert np.all(st == oracle.DK_CAP) and np.all(it == 3)
    # explicit z0 equal to the Aberth values gives the same bits as z0 = NULL
    z0 = np.concatenate([oracle.aberth(prec, coef[:, prob.coef_off[b]:prob.coef_off[b + 1]])
                         for b in range(prob.npoly)], 1)
    r1, it1, st1 = oracle.roots(prec, prob.coef_off, coef)
    r2, it2, st2 = oracle.roots(prec, prob.coef_off, coef, z0=z0)
    assert np.array_equal(r1, r2) and np.array_equal(it1, it2) and np.array_equal(st1, st2)
    # a non-finite coefficient ends in breakdown, not a hang
    bad = coef.copy()
    bad[0, 1] = np.nan
    _, it3, st3 = oracle.roots(prec, prob.coef_off, bad)
    assert st3[0] == oracle.DK_BREAKDOWN and it3[0] == 1
    # degree 0 and degree 1
    off = np.array([0, 1, 3])
    c = np.zeros((K, 3))
    c[0] = [5.0, 0.25, 1.0]
    r4, it4, st4 = oracle.roots(prec, off, c)
    assert st4[0] == oracle.DK_CONVERGED and it4[0] == 0
    assert st4[1] == oracle.DK_CONVERGED and r4[0, 0] == -0.25 and not np.any(r4[1:, 0])


def test_dk_non_monic(oracle):
    """q_n = p_n / a_n: scaling every coefficient by 3 leaves the roots unchanged
    (up to the rounding of the division)."""
    prec, K = "qd", 4
    prob = inputs.dk_problem(6, 2, 8, 12)
    coef = oracle.poly_from_roots(prec, prob)
    three = np.zeros_like(coef)
    three[0] = 3.0
    c3 = oracle.mul(prec, coef, three)
    r1, _, s1 = oracle.roots(prec, prob.coef_off, coef)
    r3, _, s3 = oracle.roots(prec, prob.coef_off, c3)
    assert np.all(s1 == 1) and np.all(s3 == 1)
    for b in range(prob.npoly):
        lo, hi = prob.root_off[b], prob.root_off[b + 1]
        assert match_sets(roots_of(oracle, prec, r1, K, lo, hi),
                          roots_of(oracle, prec, r3, K, lo, hi)) < 1e-28


def test_dk_high_degree_extended_exponent(oracle):
    """Degree 160 from a radius-1.1 circle: |q(z)| and |prod (z_i - z_j)| leave binary64's
    range during the iteration (carried with explicit exponents), the solve still ends
    at the rounding floor and finds the planted roots.  The roots of this polynomial
    are ill-conditioned in the monomial basis: double-double loses them (error ~0.2),
    triple- and quad-double recover them."""
    rng = np.random.default_rng(11)
    m = 80
    rho = 0.5 + 0.45 * rng.random(m)
    th = np.pi * (np.arange(m) + 0.5) / m  # upper half plane, well separated
    prob = inputs.dk_problem_from_roots([(list(rho * np.exp(1j * th)), None)])
    for prec, tol in (("td", 1e-12), ("qd", 1e-15)):
        K = oracle.PRECS[prec][0]
        coef = oracle.poly_from_roots(prec, prob)
        r, it, st = oracle.roots(prec, prob.coef_off, coef, radius=1.1)
        assert st[0] in (oracle.DK_CONVERGED, oracle.DK_STAGNATED), (st, it)
        got = roots_of(oracle, prec, r, K, 0, 2 * m)
        assert match_sets(got, prob.roots_of(0)) < tol
        # the start Eq. 5 gives without the explicit radius is far larger
        z0 = oracle.aberth(prec, coef)
        assert np.max(np.abs(z0[0] + 1j * z0[K])) > 2.0


def test_chebyshev_coefficients_closed_forms():
    """The reading of Eq. 6 (Newton's identities on the power sums n/(k+1)) gives the
    classical Chebyshev quadrature polynomials for n = 2..5."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "chebyshev_quadrature.json")))
    for n, coefs in g["coefficients_low_to_high"].items():
        assert inputs.chebyshev_quadrature(int(n)) == [Fraction(c) for c in coefs], n
    # power sums of the n = 64 polynomial's roots are n/(k+1) (even k) and 0 (odd k):
    # checked through the Newton identities in reverse for the first ten
    a = inputs.chebyshev_quadrature(64)
    n = 64
    e = [Fraction(1)] + [(-1) ** k * a[n - k] for k in range(1, 11)]  # elementary symmetric
    p = [None]
    for k in range(1, 11):
        pk = (-1) ** (k - 1) * k * e[k] + sum((-1) ** (k - 1 + i) * e[k - i] * p[i] for i in range(1, k))
        p.append(pk)
        assert pk == (Fraction(n, k + 1) if k % 2 == 0 else 0), k


@pytest.mark.parametrize("prec", ["td", "qd"])
def test_dk_chebyshev_n4_nodes(oracle, prec):
    """x^4 - 2/3 x^2 + 1/45 has the nodes +-sqrt(1/3 +- 2/(3 sqrt5)) (the paper's problem
    at n = 4, started from Eq. 5 as printed)."""
    K = oracle.PRECS[prec][0]
    p = pbits(oracle, prec)
    c = inputs.rational_to_mp(inputs.chebyshev_quadrature(4), K)
    r, it, st = oracle.roots(prec, np.array([0, 5]), c)
    assert st[0] in (oracle.DK_CONVERGED, oracle.DK_STAGNATED)
    s5 = isqrt_frac(Fraction(5), 400)
    nodes = []
    for sgn in (1, -1):
        x2 = Fraction(1, 3) + sgn * Fraction(2, 3) / s5
        x = isqrt_frac(x2, 300)
        nodes += [x, -x]
    got = sorted(mp_value(r[:K, j]) for j in range(4))
    for g_, w in zip(got, sorted(nodes)):
        assert float(abs(g_ - w)) <= 2.0 ** -(p - 10)
    assert all(float(abs(mp_value(r[K:, j]))) <= 2.0 ** -(p - 10) for j in range(4))
