"""GPU: the Durand-Kerner cluster solve (mp_roots_P mode 2) -- one polynomial per
thread-block cluster, its roots spread over the cluster's SMs and each complex
step split over a lane quad (degrees <= 128) or pair -- gives the bits of the one-block solver and of
the oracle: roots, sweep counts and statuses (Section 4.2, Eq. 4)."""

import numpy as np
import pytest

from paper_2603_14926_gb300 import inputs
from test_gpu_blas import dev, host, same_bits

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,n", [("qd", 64), ("td", 64), ("dd", 32), ("qd", 20)])
def test_cluster_chebyshev_bit_exact(mp, oracle, prec, n):
    """The paper's problem (Eq. 6, Table 6 at n = 64) from Eq. 5's start: alone and as
    3 copies (3 clusters), equal to the oracle and to the one-block solver."""
    K = oracle.PRECS[prec][0]
    c = inputs.rational_to_mp(inputs.chebyshev_quadrature(n), K)
    off = np.array([0, n + 1])
    wr, wit, wst = oracle.roots(prec, off, c)
    r, it, st = mp.roots(prec, dev(off), dev(c), n, mode=2)
    assert host(it)[0] == wit[0] and host(st)[0] == wst[0]
    assert same_bits(host(r), wr)
    cb = np.tile(c, 3)
    ob = np.arange(0, (n + 1) * 4, n + 1, dtype=np.int64)
    rb, itb, stb = mp.roots(prec, dev(ob), dev(cb), n, mode=2, engine=2)
    assert np.all(host(itb) == wit[0]) and np.all(host(stb) == wst[0])
    assert same_bits(host(rb), np.tile(wr, 3))


@pytest.mark.parametrize("engine", [0, 2])
@pytest.mark.parametrize("dmax", [128, 256])
def test_cluster_random_batch_matches_block_solver(mp, oracle, engine, dmax):
    """Random-root polynomials of degrees 1..dmax (lane quads per root and one CTA
    per 16 roots up to degree 128, lane pairs and one CTA per 32 roots above;
    ragged root counts per CTA, CTAs owning no root): every root, sweep count and
    status equal to the persistent one-block solve's; the three smallest also to
    the oracle's."""
    prec = "qd"
    prob = inputs.dk_problem(6, 12, 1, dmax)
    coef = oracle.poly_from_roots(prec, prob)
    md = int(prob.degrees.max())
    kw = dict(radius=1.1, max_iter=40)
    r0, i0, s0 = mp.roots(prec, dev(prob.coef_off), dev(coef), md, mode=0, engine=engine, **kw)
    r2, i2, s2 = mp.roots(prec, dev(prob.coef_off), dev(coef), md, mode=2, engine=engine, **kw)
    assert np.array_equal(host(i0), host(i2)) and np.array_equal(host(s0), host(s2))
    assert same_bits(host(r0), host(r2))
    small = np.argsort(prob.degrees, kind="stable")[:3]
    for b in small:
        sub = inputs.DKProblem([prob.degrees[b]], prob.rootdata[prob.root_off[b]:prob.root_off[b + 1]],
                               prob.delta[prob.root_off[b]:prob.root_off[b + 1]])
        c = oracle.poly_from_roots(prec, sub)
        wr, wit, wst = oracle.roots(prec, sub.coef_off, c, **kw)
        assert host(i2)[b] == wit[0] and host(s2)[b] == wst[0]
        assert same_bits(np.ascontiguousarray(host(r2)[:, prob.root_off[b]:prob.root_off[b + 1]]), wr)


def test_cluster_edge_cases(mp, oracle):
    """Degree 0 and 1, a non-monic polynomial, explicit starting values, a sweep cap,
    a one-cycle watchdog (status 3 after one sweep on every CTA of the cluster),
    and the degree bound of the mode (256)."""
    prec, K = "qd", 4
    prob = inputs.dk_problem(4, 3, 12, 20)
    base = oracle.poly_from_roots(prec, prob)
    three = np.zeros_like(base)
    three[0] = 3.0
    scaled = oracle.mul(prec, base, three)
    lin = np.zeros((K, 3))
    lin[0] = [5.0, 0.25, 1.0]
    coef = np.concatenate([lin, scaled], 1)
    off = np.concatenate([[0, 1, 3], 3 + prob.coef_off[1:]])
    md = int(np.diff(off).max() - 1)
    for kw in ({}, {"max_iter": 4}):
        r0, i0, s0 = mp.roots(prec, dev(off), dev(coef), md, mode=0, **kw)
        r2, i2, s2 = mp.roots(prec, dev(off), dev(coef), md, mode=2, **kw)
        assert np.array_equal(host(i0), host(i2)) and np.array_equal(host(s0), host(s2)), kw
        assert same_bits(host(r0), host(r2)), kw
    z0 = mp.roots_init(prec, dev(off), dev(coef), md, radius=0.9)
    ra, ia, sa = mp.roots(prec, dev(off), dev(coef), md, z0=z0, mode=0)
    rb, ib, sb = mp.roots(prec, dev(off), dev(coef), md, z0=z0, mode=2)
    assert same_bits(host(ra), host(rb)) and np.array_equal(host(ia), host(ib))
    rw0, iw0, sw0 = mp.roots(prec, dev(off), dev(coef), md, mode=0, watchdog_cycles=1)
    rw2, iw2, sw2 = mp.roots(prec, dev(off), dev(coef), md, mode=2, watchdog_cycles=1)
    assert np.array_equal(host(iw0), host(iw2)) and np.array_equal(host(sw0), host(sw2))
    assert np.sum(host(sw2) == mp.DK_TIMEOUT) == 4 and np.all(host(iw2) <= 1)  # all but degree 0
    assert same_bits(host(rw0), host(rw2))
    with pytest.raises(mp.MPError, match="invalid"):
        mp.roots(prec, dev(off), dev(coef), 257, mode=2)
