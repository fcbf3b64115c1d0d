"""GPU: torch.autograd.Function wrappers (hand-written adjoints), CUDA-graph
replay of the batched solver, and the autotuner.

Adjoints are checked bit for bit against the CPU oracle's adjoint (the same
folds: dA = dC B^T and dB = A^T dC as GEMMs with transposed operands; the
Horner adjoint of the oracle) and against QD central finite differences
computed with the oracle's arithmetic.
"""

from fractions import Fraction

import numpy as np
import pytest

from exact import mp_value
from paper_2603_14926_gb300 import inputs
from test_gpu_blas import dev, host, same_bits

pytestmark = pytest.mark.gpu


def test_mpgemm_backward_bit_exact(mp, oracle):
    import torch

    from paper_2603_14926_gb300.autograd import mp_gemm

    prec, K = "qd", 4
    m, k, n = 37, 29, 45
    A = inputs.mp_uniform(1, (m, k), K)
    B = inputs.mp_uniform(2, (k, n), K)
    G = inputs.mp_uniform(3, (m, n), K)
    tA = dev(A).requires_grad_(True)
    tB = dev(B).requires_grad_(True)
    C = mp_gemm(prec, tA, tB)
    assert same_bits(host(C), oracle.gemm(prec, A, B))
    C.backward(dev(G))
    assert same_bits(host(tA.grad), oracle.gemm(prec, G, B, opB=1))
    assert same_bits(host(tB.grad), oracle.gemm(prec, A, G, opA=1))


def test_mpgemm_backward_finite_differences(mp, oracle):
    """L(A, B) = <G, A B> is bilinear, so QD central differences (h = 2^-70, all
    arithmetic in the oracle's QD) equal the adjoint up to rounding: the QD
    rounding of L (|L| < 30, relative 2^-208) over 2h = 2^-69 is below 2^-134.
    Both sides are compared as exact K-component values (sums of their
    components as rationals), so the tolerance 2^-120 is the one tested."""
    from paper_2603_14926_gb300.autograd import mp_gemm

    prec, K = "qd", 4
    m, k, n = 6, 5, 4
    A = inputs.mp_uniform(4, (m, k), K)
    B = inputs.mp_uniform(5, (k, n), K)
    G = inputs.mp_uniform(6, (m, n), K)
    tA = dev(A).requires_grad_(True)
    tB = dev(B).requires_grad_(True)
    mp_gemm(prec, tA, tB).backward(dev(G))
    dA, dB = host(tA.grad), host(tB.grad)

    def L(A_, B_):
        C = oracle.gemm(prec, A_, B_)
        return oracle.dot(prec, G.reshape(K, -1), C.reshape(K, -1))

    h = np.zeros(K)
    h[0] = 2.0 ** -70
    for (i, j) in [(0, 0), (3, 2), (m - 1, k - 1)]:
        Ap, Am = A.copy(), A.copy()
        Ap[:, i, j] = oracle.add(prec, A[:, i, j][:, None], h[:, None])[:, 0]
        Am[:, i, j] = oracle.add(prec, A[:, i, j][:, None], -h[:, None])[:, 0]
        fd = oracle.add(prec, L(Ap, B)[:, None], -L(Am, B)[:, None])[:, 0] * 2.0 ** 69
        assert abs(mp_value(fd) - mp_value(dA[:, i, j])) <= Fraction(2) ** -120
    for (i, j) in [(0, 0), (k - 1, n - 1)]:
        Bp, Bm = B.copy(), B.copy()
        Bp[:, i, j] = oracle.add(prec, B[:, i, j][:, None], h[:, None])[:, 0]
        Bm[:, i, j] = oracle.add(prec, B[:, i, j][:, None], -h[:, None])[:, 0]
        fd = oracle.add(prec, L(A, Bp)[:, None], -L(A, Bm)[:, None])[:, 0] * 2.0 ** 69
        assert abs(mp_value(fd) - mp_value(dB[:, i, j])) <= Fraction(2) ** -120


def test_mphorner_backward_bit_exact_and_fd(mp, oracle):
    from paper_2603_14926_gb300.autograd import mp_horner

    prec, K = "qd", 4
    npoly, deg, npts = 5, 40, 24
    off = np.arange(0, (npoly + 1) * (deg + 1), deg + 1, dtype=np.int64)
    coef = inputs.mp_uniform(7, npoly * (deg + 1), K, stream=inputs.STREAM_C)
    x = inputs.mp_uniform(8, npoly * npts, K, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(9, npoly * npts, K, stream=inputs.STREAM_Y)
    tc = dev(coef).requires_grad_(True)
    tx = dev(x).requires_grad_(True)
    y = mp_horner(prec, dev(off), npts, tc, tx)
    assert same_bits(host(y), oracle.polyeval(prec, off, coef, npts, x))
    y.backward(dev(dy))
    wc, wx = oracle.polyeval_backward(prec, off, coef, npts, x, dy)
    assert same_bits(host(tc.grad), wc) and same_bits(host(tx.grad), wx)
    # QD central differences of L = <dy, p(x)> in x (h = 2^-70): the truncation
    # error (h^2 / 6 times the third derivative) and the rounding error
    # (2^-212 |p| / 2^-69) are both below 2^-120 here; compared as exact
    # K-component values
    h = np.zeros((K, 1))
    h[0] = 2.0 ** -70
    for idx in (0, npts + 3, npoly * npts - 1):
        xp, xm = x.copy(), x.copy()
        xp[:, idx] = oracle.add(prec, x[:, idx:idx + 1], h)[:, 0]
        xm[:, idx] = oracle.add(prec, x[:, idx:idx + 1], -h)[:, 0]
        yp = oracle.polyeval(prec, off, coef, npts, xp)[:, idx:idx + 1]
        ym = oracle.polyeval(prec, off, coef, npts, xm)[:, idx:idx + 1]
        d = oracle.add(prec, yp, -ym) * 2.0 ** 69
        fd = oracle.mul(prec, dy[:, idx:idx + 1], d)[:, 0]
        g = host(tx.grad)[:, idx]
        assert abs(mp_value(fd) - mp_value(g)) <= Fraction(2) ** -110 * (1 + abs(mp_value(g)))


def test_roots_graph_replay_matches_direct(mp, oracle):
    prec = "td"
    prob = inputs.dk_problem(5, 40, 5, 80)
    coef = dev(oracle.poly_from_roots(prec, prob))
    off = dev(prob.coef_off)
    md = int(prob.degrees.max())
    r0, i0, s0 = mp.roots(prec, off, coef, md, radius=1.1, max_iter=50, sort=1)
    g = mp.RootsGraph(prec, off, coef, md, radius=1.1, max_iter=50, sort=1)
    for _ in range(2):
        r1, i1, s1 = g.replay()
        assert same_bits(host(r1), host(r0))
        assert np.array_equal(host(i1), host(i0)) and np.array_equal(host(s1), host(s0))


def test_autotuner_gemm_and_roots(mp, oracle, tmp_path, monkeypatch):
    from paper_2603_14926_gb300 import tune

    monkeypatch.setenv("MPGPU_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "_cache", None)
    best, times = tune.tune_gemm("dd", 96, reps=1)
    assert 0 <= best < mp.gemm_num_configs("dd") and len(times) == mp.gemm_num_configs("dd")
    assert tune.best_gemm_config("dd", 96, 96, 96) == best
    # the tuned default computes the same bits as every other configuration
    A = inputs.mp_uniform(1, (96, 96), 2)
    B = inputs.mp_uniform(2, (96, 96), 2)
    assert same_bits(host(mp.gemm("dd", dev(A), dev(B))), oracle.gemm("dd", A, B))
    prob = inputs.dk_problem(2, 30, 10, 60)
    coef = dev(oracle.poly_from_roots("dd", prob))
    (th, bps, eng), t = tune.tune_roots("dd", dev(prob.coef_off), coef, int(prob.degrees.max()))
    assert th in (64, 128, 256) and eng in (1, 2) and (th, bps, eng) in t
    assert tune.best_roots_shape("dd", 30, int(prob.degrees.max())) == (th, bps, eng)
    assert (tmp_path / "tune.json").exists()
