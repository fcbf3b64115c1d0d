"""GPU parity: polynomial evaluation (Section 4.1), its adjoint, the
polynomial builder, Aberth starting values (Eq. 5) and the Durand-Kerner solver
(Eq. 4) through the C ABI against the CPU oracle -- all bit for bit (roots,
iteration counts and statuses included)."""

import numpy as np
import pytest

from paper_2603_14926_gb300 import inputs
from test_gpu_blas import dev, host, same_bits

pytestmark = pytest.mark.gpu


def ragged(seed, npoly, dmin, dmax, K, dt):
    rng = np.random.default_rng(seed)
    deg = rng.integers(dmin, dmax + 1, npoly)
    off = np.zeros(npoly + 1, dtype=np.int64)
    np.cumsum(deg + 1, out=off[1:])
    coef = inputs.mp_uniform(seed, int(off[-1]), K, dt, stream=inputs.STREAM_C)
    return off, coef


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd", "ds", "tf", "qf"])
def test_polyeval_bit_exact(mp, oracle, prec):
    K, dt = oracle.PRECS[prec]
    off, coef = ragged(1, 9, 0, 45, K, dt)
    npts = 33
    npoly = len(off) - 1
    xr = inputs.mp_uniform(2, npoly * npts, K, dt, stream=inputs.STREAM_X)
    xi = inputs.mp_uniform(3, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    doff, dcoef = dev(off), dev(coef)
    y = mp.polyeval(prec, doff, dcoef, npts, dev(xr))
    assert same_bits(host(y), oracle.polyeval(prec, off, coef, npts, xr))
    yr, yi = mp.polyeval(prec, doff, dcoef, npts, dev(xr), dev(xi))
    wr, wi = oracle.polyeval(prec, off, coef, npts, xr, xi)
    assert same_bits(host(yr), wr) and same_bits(host(yi), wi)


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd", "ds", "tf", "qf"])
def test_polyeval_estrin_bit_exact(mp, oracle, prec):
    """Estrin's scheme: the GPU's streamed binary-counter form against the oracle's
    level-by-level tree, ragged degrees 0..300 (every pass-through pattern up to
    nine levels), real and complex arguments."""
    K, dt = oracle.PRECS[prec]
    off, coef = ragged(31, 12, 0, 300, K, dt)
    off[3] = off[2]  # an empty polynomial
    npts = 9
    npoly = len(off) - 1
    xr = inputs.mp_uniform(32, npoly * npts, K, dt, stream=inputs.STREAM_X)
    xi = inputs.mp_uniform(33, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    doff, dcoef = dev(off), dev(coef)
    y = mp.polyeval(prec, doff, dcoef, npts, dev(xr), scheme="estrin")
    assert same_bits(host(y), oracle.polyeval_estrin(prec, off, coef, npts, xr))
    yr, yi = mp.polyeval(prec, doff, dcoef, npts, dev(xr), dev(xi), scheme="estrin")
    wr, wi = oracle.polyeval_estrin(prec, off, coef, npts, xr, xi)
    assert same_bits(host(yr), wr) and same_bits(host(yi), wi)
    if dt == np.float64:  # points near 2^-1000: the per-point FP64 recomputation
        xr[:, 0::5] *= 2.0 ** -1000
        y = mp.polyeval(prec, doff, dcoef, npts, dev(xr), scheme="estrin")
        assert same_bits(host(y), oracle.polyeval_estrin(prec, off, coef, npts, xr))


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "qf"])
@pytest.mark.parametrize("npts", [0, 1, 64, 77])
@pytest.mark.parametrize("dmax", [70, 200])
def test_polyeval_backward_bit_exact(mp, oracle, prec, npts, dmax):
    """Degrees 0..70 run the coefficient sweep with padded point periods (fewer
    than 32 coefficients) and full ones; degrees 90..200 have more coefficients
    than points.  64 points fill two groups of 32 exactly, 77 leave a ragged
    last group, 1 a single lane, 0 an empty fold."""
    K, dt = oracle.PRECS[prec]
    off, coef = ragged(4, 7, 0 if dmax == 70 else 90, dmax, K, dt)
    off[2] = off[1]  # an empty polynomial (no coefficients)
    npoly = len(off) - 1
    x = inputs.mp_uniform(5, npoly * npts, K, dt, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(6, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    dc, dx = mp.polyeval_backward(prec, dev(off), dev(coef), npts, dev(x), dev(dy))
    wc, wx = oracle.polyeval_backward(prec, off, coef, npts, x, dy)
    used = np.zeros(coef.shape[1], dtype=bool)
    for b in range(npoly):
        used[off[b]:off[b + 1]] = True
    assert same_bits(host(dc)[:, used], wc[:, used])
    assert same_bits(host(dx), wx)


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_horner_range_limits_bit_exact(mp, oracle, prec):
    """Points and adjoint seeds near the bottom of the binary64 range send the
    default hybrid engine to its FP64 recomputation (per point for values and
    dx); the coefficient sweep's engine packs the subnormal error terms
    itself.  Every result stays bit-identical to the oracle."""
    K, dt = oracle.PRECS[prec]
    off, coef = ragged(8, 6, 0, 70, K, dt)
    npoly, npts = len(off) - 1, 40
    x = inputs.mp_uniform(9, npoly * npts, K, dt, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(10, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    x[:, 0::7] *= 2.0 ** -1000
    dy[:, 2 * npts:3 * npts] *= 2.0 ** -1000
    doff, dcoef = dev(off), dev(coef)
    assert same_bits(host(mp.polyeval(prec, doff, dcoef, npts, dev(x))), oracle.polyeval(prec, off, coef, npts, x))
    dc, dx = mp.polyeval_backward(prec, doff, dcoef, npts, dev(x), dev(dy))
    wc, wx = oracle.polyeval_backward(prec, off, coef, npts, x, dy)
    assert same_bits(host(dc), wc) and same_bits(host(dx), wx)


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_dcoef_restart_on_fp64_pipe_bit_exact(mp, oracle, prec):
    """One adjoint seed of 1.5 * 2^1023 puts TwoSum operands of the coefficient
    sweep above the hybrid engine's exponent bound: that polynomial restarts
    on the FP64 pipe from its first point, and the coefficient gradient equals
    the oracle's bit for bit (points in [0, 1), so no running power overflows)."""
    K, dt = oracle.PRECS[prec]
    off, coef = ragged(8, 6, 0, 70, K, dt)
    npoly, npts = len(off) - 1, 40
    x = np.abs(inputs.mp_uniform(9, npoly * npts, K, dt, stream=inputs.STREAM_X))
    dy = inputs.mp_uniform(10, npoly * npts, K, dt, stream=inputs.STREAM_Y)
    dy[:, 2 * npts + 5] = 0.0
    dy[0, 2 * npts + 5] = 1.5 * 2.0 ** 1023
    dc, _ = mp.polyeval_backward(prec, dev(off), dev(coef), npts, dev(x), dev(dy), want_dx=False)
    wc, _ = oracle.polyeval_backward(prec, off, coef, npts, x, dy, want_dx=False)
    assert np.isfinite(wc).all()
    assert same_bits(host(dc), wc)


def test_polyeval_backward_needs_no_workspace(mp, oracle):
    """The coefficient sweep keeps its partial sums in dcoef itself: the size
    query answers 0 and a call without a workspace equals the oracle."""
    K, dt = 4, np.float64
    off, coef = ragged(4, 3, 5, 40, K, dt)
    x = inputs.mp_uniform(5, 3 * 40, K, dt)
    assert mp.polyeval_backward_workspace("qd", 3, 40) == 0
    dc, dx = mp.polyeval_backward("qd", dev(off), dev(coef), 40, dev(x), dev(x))
    wc, wx = oracle.polyeval_backward("qd", off, coef, 40, x, x)
    assert same_bits(host(dc), wc) and same_bits(host(dx), wx)


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd"])
def test_poly_from_roots_bit_exact(mp, oracle, prec):
    prob = inputs.dk_problem(3, 11, 1, 75)
    want = oracle.poly_from_roots(prec, prob)
    got = mp.poly_from_roots(prec, dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta),
                             int(prob.degrees.max()), int(prob.coef_off[-1]))
    assert same_bits(host(got), want)


def test_roots_one_sweep_host_loop_equals_batched(mp):
    """The per-polynomial baseline of the benchmark: a host loop of one-sweep
    launches (max_iter 1, z0 = the previous iterate, the status read after each)
    ends, after the batched solve's sweep count, on the batched solve's bits."""
    import torch

    prob = inputs.dk_problem(14, 6, 10, 60)
    coef = mp.poly_from_roots("qd", dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta), 60,
                              int(prob.coef_off[-1]))
    r, it, st = mp.roots("qd", dev(prob.coef_off), coef, 60, radius=1.1, max_iter=200, sort=1)
    r, it, st = host(r), host(it), host(st)
    hc = host(coef)
    for b in range(prob.npoly):
        n = int(prob.degrees[b])
        oq = dev(np.array([0, n + 1], dtype=np.int64))
        cq = dev(hc[:, prob.coef_off[b]:prob.coef_off[b + 1]])
        z = mp.roots_init("qd", oq, cq, n, radius=1.1)
        zb = torch.empty_like(z)
        for k in range(int(it[b])):
            zb, _, sq = mp.roots("qd", oq, cq, n, z0=z, max_iter=1, mode=1, out=zb)
            flag = int(sq.item())
            z, zb = zb, z
            if flag == 1:  # converged: only at the batched solve's last sweep
                assert k + 1 == it[b] and st[b] == 1
        assert same_bits(host(z), r[:, prob.root_off[b]:prob.root_off[b + 1]]), b


@pytest.mark.parametrize("prec", ["dd", "qd"])
@pytest.mark.parametrize("radius", [0.0, 1.1])
def test_roots_init_bit_exact(mp, oracle, prec, radius):
    K = oracle.PRECS[prec][0]
    prob = inputs.dk_problem(5, 7, 2, 90)
    coef = oracle.poly_from_roots(prec, prob)
    z = host(mp.roots_init(prec, dev(prob.coef_off), dev(coef), int(prob.degrees.max()), radius))
    for b in range(prob.npoly):
        c = coef[:, prob.coef_off[b]:prob.coef_off[b + 1]]
        want = oracle.aberth(prec, c, radius)
        assert same_bits(np.ascontiguousarray(z[:, prob.root_off[b]:prob.root_off[b + 1]]), want), b


def _solve_both(mp, oracle, prec, prob, coef, **kw):
    maxdeg = int(prob.degrees.max())
    r, it, st = mp.roots(prec, dev(prob.coef_off), dev(coef), maxdeg, **kw)
    okw = {k: v for k, v in kw.items() if k in ("tol", "max_iter", "stag_window", "stag_min_iter",
                                                  "radius")}
    wr, wit, wst = oracle.roots(prec, prob.coef_off, coef, **okw)
    return (host(r), host(it), host(st)), (wr, wit, wst)


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd"])
@pytest.mark.parametrize("engine", [0, 2])
def test_roots_bit_exact(mp, oracle, prec, engine):
    prob = inputs.dk_problem(3, 6, 10, 40)
    coef = oracle.poly_from_roots(prec, prob)
    (r, it, st), (wr, wit, wst) = _solve_both(mp, oracle, prec, prob, coef, engine=engine)
    assert np.array_equal(it, wit) and np.array_equal(st, wst)
    assert same_bits(np.ascontiguousarray(r), wr)
    assert np.all((st == 1) | (st == 2))


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_roots_range_limits_bit_exact(mp, oracle, prec):
    """Hybrid engine (the default).  One starting value per polynomial placed
    near 2^-1000 makes the first sweep's Horner products produce subnormal TwoSum
    error terms, which the solver's hybrid engine packs exactly on the integer
    pipes (no FP64 recomputation): roots, sweep counts and statuses stay
    bit-identical to the oracle.  (Two such starting values would make a
    difference underflow to zero and the solve break down.)"""
    K = oracle.PRECS[prec][0]
    prob = inputs.dk_problem(5, 4, 12, 30)
    coef = oracle.poly_from_roots(prec, prob)
    z0 = np.zeros((2 * K, int(prob.degrees.sum())))
    for b in range(prob.npoly):
        c = coef[:, prob.coef_off[b]:prob.coef_off[b + 1]]
        z = oracle.aberth(prec, c, radius=1.1)
        z[:, :1] *= 2.0 ** -1000
        z0[:, prob.root_off[b]:prob.root_off[b + 1]] = z
    before = mp.roots_hybrid_fallbacks()
    r, it, st = mp.roots(prec, dev(prob.coef_off), dev(coef), int(prob.degrees.max()), z0=dev(z0), max_iter=40,
                         engine=1)
    wr, wit, wst = oracle.roots(prec, prob.coef_off, coef, z0=z0, max_iter=40)
    assert np.array_equal(host(it), wit) and np.array_equal(host(st), wst)
    assert np.isfinite(wr).all() and np.all(wst != 4)
    assert same_bits(np.ascontiguousarray(host(r)), wr)
    assert mp.roots_hybrid_fallbacks() == before


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_roots_fp64_recomputation_bit_exact(mp, oracle, prec):
    """Starting values near 2^1023 for linear polynomials put TwoSum operands
    above the hybrid engine's exponent bound (Horner's z + a_0 and the update
    z - w): those roots are recomputed on the FP64 pipe (counted), and the
    results, sweep counts and statuses equal the oracle's."""
    K = oracle.PRECS[prec][0]
    prob = inputs.dk_problem_from_roots([([], 0.25), ([], -0.75), ([], 0.125)])
    coef = oracle.poly_from_roots(prec, prob)
    z0 = np.zeros((2 * K, int(prob.degrees.sum())))
    z0[0, :] = [2.0 ** 1023, -(2.0 ** 1022) * 1.5, 1.75 * 2.0 ** 1023]
    before = mp.roots_hybrid_fallbacks()
    r, it, st = mp.roots(prec, dev(prob.coef_off), dev(coef), int(prob.degrees.max()), z0=dev(z0), max_iter=60,
                         engine=1)
    wr, wit, wst = oracle.roots(prec, prob.coef_off, coef, z0=z0, max_iter=60)
    assert np.array_equal(host(it), wit) and np.array_equal(host(st), wst)
    assert same_bits(np.ascontiguousarray(host(r)), wr)
    assert mp.roots_hybrid_fallbacks() > before


@pytest.mark.parametrize("mode,sort,threads,engine", [(0, 0, 64, 2), (0, 1, 256, 2), (1, 0, 128, 2), (1, 1, 32, 2),
                                                      (0, 1, 256, 1), (1, 0, 64, 1), (0, 0, 128, 0)])
def test_roots_modes_identical(mp, oracle, mode, sort, threads, engine):
    """Persistent batched launch and the per-polynomial launch loop, sorted or not,
    any block size: identical bits, equal to the oracle."""
    prec = "td"
    prob = inputs.dk_problem(8, 9, 3, 70)
    coef = oracle.poly_from_roots(prec, prob)
    (r, it, st), (wr, wit, wst) = _solve_both(mp, oracle, prec, prob, coef, mode=mode, sort=sort,
                                              threads=threads, radius=1.1, engine=engine)
    assert np.array_equal(it, wit) and np.array_equal(st, wst)
    assert same_bits(np.ascontiguousarray(r), wr)


def test_roots_edge_cases(mp, oracle):
    """Degree 0 and 1, a non-monic polynomial, an iteration cap, a non-finite
    coefficient (breakdown), explicit starting values."""
    prec, K = "qd", 4
    prob = inputs.dk_problem(4, 3, 12, 20)
    base = oracle.poly_from_roots(prec, prob)
    three = np.zeros_like(base)
    three[0] = 3.0
    scaled = oracle.mul(prec, base, three)
    lin = np.zeros((K, 3))
    lin[0] = [5.0, 0.25, 1.0]  # degree 0 (a_0 = 5) and degree 1 (x + 0.25)
    coef = np.concatenate([lin, scaled, base], 1)
    off = np.concatenate([[0, 1, 3], 3 + prob.coef_off[1:], 3 + prob.coef_off[-1] + prob.coef_off[1:]])
    bad = coef.copy()
    bad[0, off[3] + 2] = np.nan

    class Prob:
        coef_off = off
        degrees = np.diff(off) - 1
    for c, kw in ((coef, {}), (coef, {"max_iter": 4}), (bad, {})):
        (r, it, st), (wr, wit, wst) = _solve_both(mp, oracle, prec, Prob, c, **kw)
        assert np.array_equal(it, wit) and np.array_equal(st, wst), (kw, it, wit, st, wst)
        ok = np.ones(r.shape[1], dtype=bool)
        for b in np.nonzero(st == mp.DK_BREAKDOWN)[0]:  # NaN payloads are not compared
            ok[off[b] - b:off[b + 1] - b - 1] = False
        assert same_bits(np.ascontiguousarray(r[:, ok]), np.ascontiguousarray(wr[:, ok]))
    assert np.sum(st == mp.DK_BREAKDOWN) == 1
    z0 = mp.roots_init(prec, dev(off), dev(coef), int(Prob.degrees.max()))
    r1, i1, s1 = mp.roots(prec, dev(off), dev(coef), int(Prob.degrees.max()))
    r2, i2, s2 = mp.roots(prec, dev(off), dev(coef), int(Prob.degrees.max()), z0=z0)
    assert same_bits(host(r1), host(r2)) and np.array_equal(host(i1), host(i2))


def test_roots_watchdog_and_degree_bound(mp, oracle):
    """A one-cycle watchdog ends every solve after its first sweep with status 3;
    a polynomial above max_degree is skipped with status 4.  No fault, no hang."""
    prec = "dd"
    prob = inputs.dk_problem(6, 5, 20, 30)
    coef = dev(oracle.poly_from_roots(prec, prob))
    r, it, st = mp.roots(prec, dev(prob.coef_off), coef, int(prob.degrees.max()), watchdog_cycles=1)
    assert np.all(host(st) == mp.DK_TIMEOUT) and np.all(host(it) == 1)
    small = int(prob.degrees.min())
    r, it, st = mp.roots(prec, dev(prob.coef_off), coef, small)
    st = host(st)
    assert np.all(st[prob.degrees > small] == mp.DK_BREAKDOWN)
    assert np.all(st[prob.degrees == small] != mp.DK_BREAKDOWN)
    with pytest.raises(mp.MPError, match="invalid"):
        mp.roots(prec, dev(prob.coef_off), coef, (1 << 20) + 1)
    with pytest.raises(mp.MPError, match="workspace"):  # above the shared-memory bound: slots needed
        big = mp.roots_max_degree(prec) + 1
        mp.roots(prec, dev(prob.coef_off), coef, big, ws=torch_empty(mp.roots_workspace(prec, prob.npoly)))


def torch_empty(nbytes):
    import torch

    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")


def test_roots_batch_workload_sampled(mp, oracle):
    """The batched-root workload's recipe (degrees uniform in [10, 500], roots in the
    unit disk, 1e-30 perturbation, QD, start radius 1.1, persistent sorted launch) on
    a 48-polynomial slice, 30 sweeps: GPU-built coefficients equal the oracle's on the
    sampled polynomials; the per-polynomial launch loop reproduces the batched
    launch bit for bit on the 8 lowest degrees; the 3 lowest equal the oracle's."""
    prec = "qd"
    prob = inputs.dk_problem(3, 48, 10, 500)
    maxdeg = int(prob.degrees.max())
    coef = mp.poly_from_roots(prec, dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta), maxdeg,
                              int(prob.coef_off[-1]))
    hc = host(coef)
    kw = dict(radius=1.1, max_iter=30)
    r0, i0, s0 = mp.roots(prec, dev(prob.coef_off), coef, maxdeg, mode=0, sort=1, **kw)
    r0, i0, s0 = host(r0), host(i0), host(s0)
    small = np.argsort(prob.degrees, kind="stable")[:8]
    sub_off = np.zeros(len(small) + 1, dtype=np.int64)
    np.cumsum(prob.degrees[small] + 1, out=sub_off[1:])
    sub_coef = np.concatenate([hc[:, prob.coef_off[b]:prob.coef_off[b + 1]] for b in small], 1)
    r1, i1, s1 = mp.roots(prec, dev(sub_off), dev(sub_coef), int(prob.degrees[small].max()),
                          mode=1, **kw)
    r1, i1, s1 = host(r1), host(i1), host(s1)
    for q, b in enumerate(small):
        lo, hi = prob.root_off[b], prob.root_off[b + 1]
        assert same_bits(np.ascontiguousarray(r1[:, sub_off[q] - q:sub_off[q + 1] - q - 1]),
                         np.ascontiguousarray(r0[:, lo:hi]))
        assert i1[q] == i0[b] and s1[q] == s0[b]
    for b in small[:3]:
        sub = inputs.DKProblem([prob.degrees[b]], prob.rootdata[prob.root_off[b]:prob.root_off[b + 1]],
                               prob.delta[prob.root_off[b]:prob.root_off[b + 1]])
        c = oracle.poly_from_roots(prec, sub)
        assert same_bits(np.ascontiguousarray(hc[:, prob.coef_off[b]:prob.coef_off[b + 1]]), c)
        wr, wit, wst = oracle.roots(prec, sub.coef_off, c, **kw)
        assert i0[b] == wit[0] and s0[b] == wst[0]
        assert same_bits(np.ascontiguousarray(r0[:, prob.root_off[b]:prob.root_off[b + 1]]), wr)


@pytest.mark.parametrize("prec,n", [("qd", 64), ("td", 64), ("dd", 32)])
def test_roots_chebyshev_bit_exact(mp, oracle, prec, n):
    """The paper's Durand-Kerner test problem (Section 4.2, Eq. 6; Table 6 uses n = 64),
    started from Eq. 5 as printed: roots, sweeps and status equal the oracle's, both as a
    single solve and as one member of a batch of identical problems."""
    K = oracle.PRECS[prec][0]
    c = inputs.rational_to_mp(inputs.chebyshev_quadrature(n), K)
    wr, wit, wst = oracle.roots(prec, np.array([0, n + 1]), c)
    r, it, st = mp.roots(prec, dev(np.array([0, n + 1])), dev(c), n)
    assert host(it)[0] == wit[0] and host(st)[0] == wst[0]
    assert same_bits(host(r), wr)
    copies = 5
    cb = np.tile(c, copies)
    ob = np.arange(0, (n + 1) * (copies + 1), n + 1, dtype=np.int64)
    rb, itb, stb = mp.roots(prec, dev(ob), dev(cb), n)
    assert np.all(host(itb) == wit[0]) and np.all(host(stb) == wst[0])
    assert same_bits(host(rb), np.tile(wr, copies))
