"""GPU parity at the benchmark's full sizes and launch configurations, on outputs
the oracle can compute one by one (bit-exact) or through properties that hold at
any size (reduction bounds).

Sizes: AXPY and dot at n = 2^24 and GEMV 8192 x 8192 (QD); Horner forward and
adjoint on 1024 polynomials of degree 256 at 4096 points each (QD); the 3M
complex GEMM at n = 1024 (QD); a Durand-Kerner sweep at the largest degree the
QD solver accepts.
"""

from fractions import Fraction

import numpy as np
import pytest

from exact import SCALE_BITS, mp_ints
from paper_2603_14926_gb300 import inputs
from test_gpu_blas import dev, host, same_bits

pytestmark = pytest.mark.gpu

P = 4 * 53  # QD precision in bits


def close(g, o, n, mag):
    """Two QD sums that are each within (4n + 16) 2^-p mag of the exact one."""
    diff = abs(int(mp_ints(g[:, None])[0]) - int(mp_ints(o[:, None])[0]))
    return Fraction(diff, 1 << SCALE_BITS) <= Fraction(2 * (4 * n + 16)) * Fraction(2) ** -P * Fraction(mag)


def test_axpy_dot_full_size(mp, oracle):
    n = 1 << 24
    x = inputs.mp_uniform(1, n, 4, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(1, n, 4, stream=inputs.STREAM_Y)
    alpha = inputs.mp_uniform(2, 1, 4)[:, 0]
    dx, dy = dev(x), dev(y)
    # dot: GPU tree vs the oracle's sequential fold; both are within (4n+16) 2^-p sum|xy|
    # of the exact sum, so they differ by at most twice that
    g = host(mp.dot("qd", dx, dy))
    o = oracle.dot("qd", x, y)
    mag = float(np.abs(x[0]) @ np.abs(y[0])) * (1 + 2.0 ** -50)
    assert close(g, o, n, mag)
    # AXPY in the benchmark's launch: 4096 sampled elements, bit for bit
    mp.axpy("qd", alpha, dx, dy)
    got = host(dy)
    idx = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(0).integers(0, n, 4094)]))
    want = oracle.axpy("qd", alpha, x[:, idx], y[:, idx])
    assert same_bits(np.ascontiguousarray(got[:, idx]), want)


def test_gemv_full_size_sampled_rows(mp, oracle):
    m = n = 8192
    A = inputs.mp_uniform(3, (m, n), 4)
    x = inputs.mp_uniform(4, n, 4, stream=inputs.STREAM_X)
    y = host(mp.gemv("qd", dev(A), dev(x)))
    for i in (0, 1, 4097, m - 1):
        o = oracle.dot("qd", A[:, i, :], x)
        mag = float(np.abs(A[0, i]) @ np.abs(x[0])) * (1 + 2.0 ** -50)
        assert close(y[:, i], o, n, mag), i


def test_horner_adjoint_workload_sampled(mp, oracle):
    """1024 polynomials of degree 256, 4096 points each: forward values and dx at
    sampled points, and dcoef of sampled polynomials, bit for bit."""
    npoly, deg, npts = 1024, 256, 4096
    off = np.arange(0, (npoly + 1) * (deg + 1), deg + 1, dtype=np.int64)
    coef = inputs.mp_uniform(4, npoly * (deg + 1), 4, stream=inputs.STREAM_C)
    xs = inputs.mp_uniform(5, npoly * npts, 4, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(6, npoly * npts, 4, stream=inputs.STREAM_Y)
    doff, dcoef, dxs, ddy = dev(off), dev(coef), dev(xs), dev(dy)
    y = host(mp.polyeval("qd", doff, dcoef, npts, dxs))
    dc, dxg = mp.polyeval_backward("qd", doff, dcoef, npts, dxs, ddy)
    dc, dxg = host(dc), host(dxg)
    rng = np.random.default_rng(1)
    for b in (0, 511, npoly - 1):
        sub_off = np.array([0, deg + 1], dtype=np.int64)
        c = np.ascontiguousarray(coef[:, off[b]:off[b + 1]])
        pts = np.unique(np.concatenate([[0, npts - 1], rng.integers(0, npts, 30)]))
        xb = np.ascontiguousarray(xs[:, b * npts + pts])
        yb = np.ascontiguousarray(dy[:, b * npts + pts])
        assert same_bits(np.ascontiguousarray(y[:, b * npts + pts]),
                         oracle.polyeval("qd", sub_off, c, len(pts), xb))
        _, wx = oracle.polyeval_backward("qd", sub_off, c, len(pts), xb, yb, want_dcoef=False)
        assert same_bits(np.ascontiguousarray(dxg[:, b * npts + pts]), wx)
    for b in (0, npoly - 1):  # the coefficient gradient needs all of a polynomial's points
        sub_off = np.array([0, deg + 1], dtype=np.int64)
        c = np.ascontiguousarray(coef[:, off[b]:off[b + 1]])
        xb = np.ascontiguousarray(xs[:, b * npts:(b + 1) * npts])
        yb = np.ascontiguousarray(dy[:, b * npts:(b + 1) * npts])
        wc, _ = oracle.polyeval_backward("qd", sub_off, c, npts, xb, yb, want_dx=False)
        assert same_bits(np.ascontiguousarray(dc[:, off[b]:off[b + 1]]), wc)


def test_cgemm3m_full_size_sampled(mp, oracle):
    """The complex GEMM workload: n = 1024, Eq. 2 entries U exp(r) (seed 7)."""
    n, K = 1024, 4
    Ur, Er, Ui, Ei = inputs.complex_eq2(7, (n, n), K)
    mk = lambda U, E: oracle.mul("qd", U.reshape(K, -1),  # noqa: E731
                                 inputs.mp_from_double(E.reshape(-1), K)).reshape(K, n, n)
    Ar, Ai, Br, Bi = mk(Ur, Er), mk(Ui, Ei), mk(Ur, Ei), mk(Ui, Er)
    gr, gi = mp.cgemm("qd", dev(Ar), dev(Ai), dev(Br), dev(Bi))
    gr, gi = host(gr), host(gi)
    for i, j in ((0, 0), (n - 1, n - 1), (17, 900), (700, 3)):
        wr, wi = oracle.cgemm("qd", Ar[:, i:i + 1, :], Ai[:, i:i + 1, :], Br[:, :, j:j + 1], Bi[:, :, j:j + 1])
        assert same_bits(gr[:, i, j], wr[:, 0, 0]) and same_bits(gi[:, i, j], wi[:, 0, 0]), (i, j)


def test_roots_at_max_degree(mp, oracle):
    """One sweep at the largest degree the QD solver accepts (its shared-memory bound)."""
    n = mp.roots_max_degree("qd")
    assert n > 2048
    prob = inputs.dk_problem(9, 1, n, n)
    coef = oracle.poly_from_roots("qd", prob)
    gc = dev(coef)  # above the coefficient builder's degree limit (2048)
    r, it, st = mp.roots("qd", dev(prob.coef_off), gc, n, radius=1.1, max_iter=1)
    wr, wit, wst = oracle.roots("qd", prob.coef_off, coef, radius=1.1, max_iter=1)
    assert host(it)[0] == wit[0] == 1 and host(st)[0] == wst[0]
    assert same_bits(host(r), wr)


def _sample_pairs(n, count, seed):
    """Corners, edge midpoints and random entries of an n x n result."""
    rng = np.random.default_rng(seed)
    fixed = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (n // 2, 0), (0, n // 2), (n // 2, n - 1),
             (n - 1, n // 2)]
    rand = list(zip(rng.integers(0, n, count - len(fixed)).tolist(), rng.integers(0, n, count - len(fixed)).tolist()))
    return fixed + rand


def test_gemm_backward_qd_2048_sampled(mp, oracle):
    """The GEMM adjoint at the benchmark's size (QD, n = 2048) through the
    torch.autograd.Function: 40 sampled entries each of dA = dC B^T and
    dB = A^T dC (the transposed-operand TMA path) bit for bit against the
    oracle's GEMM with op = T on the entry's row and column."""
    import torch

    from paper_2603_14926_gb300.autograd import mp_gemm

    prec, K, n = "qd", 4, 2048
    A = inputs.mp_uniform(11, (n, n), K)
    B = inputs.mp_uniform(12, (n, n), K)
    G = inputs.mp_uniform(13, (n, n), K)
    tA = dev(A).requires_grad_(True)
    tB = dev(B).requires_grad_(True)
    C = mp_gemm(prec, tA, tB)
    dA, dB = torch.autograd.grad(C, (tA, tB), dev(G))
    dA, dB = host(dA), host(dB)
    for i, j in _sample_pairs(n, 40, 1):
        want = oracle.gemm(prec, G[:, i:i + 1, :], B[:, j:j + 1, :], opB=1)[:, 0, 0]
        assert same_bits(dA[:, i, j], want), ("dA", i, j)
    for i, j in _sample_pairs(n, 40, 2):
        want = oracle.gemm(prec, A[:, :, i:i + 1], G[:, :, j:j + 1], opA=1)[:, 0, 0]
        assert same_bits(dB[:, i, j], want), ("dB", i, j)


@pytest.mark.parametrize("prec,n", [("tf", 4096), ("qf", 4096), ("td", 2048)])
def test_gemm_benchmark_sizes_sampled(mp, oracle, prec, n):
    """The square GEMM sizes the benchmark reports beyond QD 2048 / DD 4096: the
    binary32-component variants at n = 4096 and TD at n = 2048, built-in
    configuration, 32 sampled entries bit for bit."""
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(2, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(2, (n, n), K, dt, stream=inputs.STREAM_B)
    C = host(mp.gemm(prec, dev(A), dev(B), config=-1))
    for i, j in _sample_pairs(n, 32, 3):
        want = oracle.gemm(prec, A[:, i:i + 1, :], B[:, :, j:j + 1])[:, 0, 0]
        assert same_bits(C[:, i, j], want), (i, j)


@pytest.mark.parametrize("prec,n", [("qd", 2600), ("dd", 4900)])
def test_roots_above_shared_memory_bound(mp, oracle, prec, n):
    """Degrees above the shared-memory bound (QD 2421, DD 4843): each block keeps
    its coefficients and iterate in a slot of the workspace.  A polynomial above
    the bound, two sweeps, persistent launch and per-polynomial launch, equals
    the oracle; smaller polynomials solved in the same launch equal their
    shared-memory solve."""
    assert n > mp.roots_max_degree(prec)
    prob = inputs.dk_problem(9, 1, n, n)
    coef = oracle.poly_from_roots(prec, prob)
    wr, wit, wst = oracle.roots(prec, prob.coef_off, coef, radius=1.1, max_iter=2)
    for mode in (0, 1):
        r, it, st = mp.roots(prec, dev(prob.coef_off), dev(coef), n, radius=1.1, max_iter=2, mode=mode)
        assert host(it)[0] == wit[0] == 2 and host(st)[0] == wst[0], mode
        assert same_bits(host(r), wr), mode
    small = inputs.dk_problem(10, 6, 20, 200)
    cs = dev(oracle.poly_from_roots(prec, small))
    r1, i1, s1 = mp.roots(prec, dev(small.coef_off), cs, 200, radius=1.1, max_iter=30)
    r2, i2, s2 = mp.roots(prec, dev(small.coef_off), cs, n, radius=1.1, max_iter=30)  # slots
    assert np.array_equal(host(i1), host(i2)) and np.array_equal(host(s1), host(s2))
    assert same_bits(host(r1), host(r2))
