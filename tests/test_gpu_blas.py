"""GPU parity: elementwise ops, AXPY, dot, GEMV and GEMM through the C ABI
against the CPU oracle on the same seeded inputs.

Elementwise ops, AXPY and GEMM (sequential k) must match bit for bit; dot and
GEMV reduce in a tree and must agree with the exact sum within
(4n + 16) 2^-p sum |x_i y_i|.
"""

from fractions import Fraction

import numpy as np
import pytest

from cases import families
from exact import SCALE_BITS, mp_ints
from paper_2603_14926_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL = ["dd", "ddc", "td", "qd", "ds", "tf", "qf"]


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def same_bits(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    if a.shape != b.shape or a.dtype != b.dtype:
        return False
    u = np.uint64 if a.dtype == np.float64 else np.uint32
    return np.array_equal(a.view(u), b.view(u))


def pbits(prec):
    from oracle.mpref import PRECS

    K, dt = PRECS[prec]
    return K * (53 if dt == np.float64 else 24)


@pytest.mark.parametrize("prec", ALL)
def test_elementwise_bit_exact(mp, oracle, prec):
    K, dt = oracle.PRECS[prec]
    for name, a, b in families(oracle, prec, n=1537, seed=3, limits=True):
        da, db = dev(a), dev(b)
        assert same_bits(host(mp.add(prec, da, db)), oracle.add(prec, a, b)), name
        assert same_bits(host(mp.mul(prec, da, db)), oracle.mul(prec, a, b)), name
    x = inputs.mp_uniform(9, 5003, K, dt) * np.exp2((np.arange(5003) % 61) - 30).astype(dt)
    assert same_bits(host(mp.recip(prec, dev(x))), oracle.recip(prec, x))


@pytest.mark.parametrize("prec", ALL)
def test_axpy_bit_exact(mp, oracle, prec):
    K, dt = oracle.PRECS[prec]
    n = 100_003
    x = inputs.mp_uniform(1, n, K, dt, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(1, n, K, dt, stream=inputs.STREAM_Y)
    alpha = inputs.mp_uniform(2, 1, K, dt)[:, 0]
    dy = dev(y)
    mp.axpy(prec, alpha, dev(x), dy)
    assert same_bits(host(dy), oracle.axpy(prec, alpha, x, y))
    if dt == np.float64:  # operands near the ends of the range: the FP64 recomputation path
        x[:, 0::5] *= 2.0 ** -1000
        y[:, 1::5] *= 2.0 ** 1000
        dy = dev(y)
        mp.axpy(prec, alpha, dev(x), dy)
        assert same_bits(host(dy), oracle.axpy(prec, alpha, x, y))


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd", "qf"])
@pytest.mark.parametrize("n", [0, 1, 255, 70_001])
def test_dot_within_bound(mp, oracle, prec, n):
    K, dt = oracle.PRECS[prec]
    x = inputs.mp_uniform(4, n, K, dt, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(4, n, K, dt, stream=inputs.STREAM_Y)
    g = host(mp.dot(prec, dev(x), dev(y)))
    if n == 0:
        assert not np.any(g)
        return
    ex = int(mp_ints(x).dot(mp_ints(y)))
    gi = int(mp_ints(g[:, None])[0])
    err = float(Fraction(abs(gi * (1 << SCALE_BITS) - ex), 1 << (2 * SCALE_BITS)))
    mag = float(np.abs(x.astype(np.float64)).sum(0) @ np.abs(y.astype(np.float64)).sum(0))
    assert err <= (4 * n + 16) * 2.0 ** -pbits(prec) * mag
    # same bound for the oracle's sequential fold, and the two agree to it
    o = oracle.dot(prec, x, y)
    oi = int(mp_ints(o[:, None])[0])
    assert float(Fraction(abs(oi - gi), 1 << SCALE_BITS)) <= 2 * (4 * n + 16) * 2.0 ** -pbits(prec) * mag


def test_dot_workspace_errors(mp):
    import torch

    x = mp.zeros("qd", 5000)
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(mp.MPError, match="workspace"):
        mp.dot("qd", x, x, ws=small)


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_dot_gemv_range_limits_match_fp64_fold(mp, oracle, prec):
    """Every fourth column of A (and element of x for the dot) scaled by 2^-1000:
    the threads whose partial folds meet them recompute on the FP64 pipe.  The
    one-column GEMM (sequential fold) matches the oracle bit for bit; GEMV and
    dot, which reduce in a tree, agree with the sequential folds to 1e-12
    relative (no error bound of the paper applies in the subnormal range, so this
    checks that the recomputed partials are the right ones, not garbage)."""
    K, dt = oracle.PRECS[prec]
    n = 700
    A = inputs.mp_uniform(21, (3, n), K)
    x = inputs.mp_uniform(22, n, K, stream=inputs.STREAM_X)
    A[:, :, 0::4] *= 2.0 ** -1000
    want = oracle.gemm(prec, A, x.reshape(K, n, 1))[:, :, 0]
    g = host(mp.gemm(prec, dev(A), dev(x.reshape(K, n, 1))))[:, :, 0]
    assert same_bits(g, want)
    y = host(mp.gemv(prec, dev(A), dev(x)))
    for i in range(3):
        assert abs(float(y[0, i]) - float(want[0, i])) <= 1e-12 * max(1.0, abs(float(want[0, i])))
    d = host(mp.dot(prec, dev(np.ascontiguousarray(A[:, 0, :])), dev(x)))
    assert abs(float(d[0]) - float(want[0, 0])) <= 1e-12 * max(1.0, abs(float(want[0, 0])))


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "tf"])
@pytest.mark.parametrize("n", [600, 1029, 2500, 5000])
def test_gemv_within_bound(mp, oracle, prec, n):
    """37 rows: n = 600, 1029, 2500, 5000 run 32, 64, 128, 256 threads per row."""
    K, dt = oracle.PRECS[prec]
    m = 37
    A = inputs.mp_uniform(5, (m, n), K, dt)
    x = inputs.mp_uniform(6, n, K, dt, stream=inputs.STREAM_X)
    g = host(mp.gemv(prec, dev(A), dev(x)))
    Ai, xi = mp_ints(A), mp_ints(x)
    absA = np.abs(A.astype(np.float64)).sum(0)
    absx = np.abs(x.astype(np.float64)).sum(0)
    for i in range(m):
        ex = int(Ai[i].dot(xi))
        gi = int(mp_ints(g[:, i:i + 1])[0])
        err = float(Fraction(abs(gi * (1 << SCALE_BITS) - ex), 1 << (2 * SCALE_BITS)))
        assert err <= (4 * n + 16) * 2.0 ** -pbits(prec) * float(absA[i] @ absx)


@pytest.mark.parametrize("prec", ALL)
def test_gemm_config0_bit_exact(mp, oracle, prec):
    """n = 64, seed 0 (the oracle's exact-rational pin uses the same inputs)."""
    K, dt = oracle.PRECS[prec]
    n = 64
    A = inputs.mp_uniform(0, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(0, (n, n), K, dt, stream=inputs.STREAM_B)
    want = oracle.gemm(prec, A, B)
    for cfg in range(mp.gemm_num_configs(prec)):
        assert same_bits(host(mp.gemm(prec, dev(A), dev(B), config=cfg)), want), cfg


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd"])
def test_gemm_hybrid_fallback_bit_exact(mp, oracle, prec):
    """Rows of A scaled by 2^-1000 drive the error terms of their products below the
    normal range: the hybrid engine's threads owning those rows fall back to the
    FP64 pipe (counted), the others do not, and every configuration stays
    bit-identical to the oracle.  A second family cancels the whole fold
    (A = [X X], B = [Y; -Y + tiny]), which exercises QuickTwoSum outside its
    exact case under configuration 6."""
    K, dt = oracle.PRECS[prec]
    m, n, k0 = 40, 36, 25
    A = inputs.mp_uniform(11, (m, 2 * k0), K)
    B = inputs.mp_uniform(12, (2 * k0, n), K)
    A[:, :5, :] *= 2.0 ** -1000
    want = oracle.gemm(prec, A, B)
    X = inputs.mp_uniform(13, (m, k0), K)
    Y = inputs.mp_uniform(14, (k0, n), K)
    A2 = np.concatenate([X, X], axis=2)
    B2 = np.concatenate([Y, -Y + inputs.mp_uniform(15, (k0, n), K) * 2.0 ** -40], axis=1)
    want2 = oracle.gemm(prec, A2, B2)
    for cfg in range(mp.gemm_num_configs(prec)):
        before = mp.gemm_hybrid_fallbacks(prec)
        assert same_bits(host(mp.gemm(prec, dev(A), dev(B), config=cfg)), want), cfg
        taken = mp.gemm_hybrid_fallbacks(prec) - before
        if "hybrid" in mp.gemm_config_name(prec, cfg):
            assert 0 < taken < m * n, (cfg, taken)
        else:
            assert taken == 0, (cfg, taken)
        assert same_bits(host(mp.gemm(prec, dev(A2), dev(B2), config=cfg)), want2), cfg


@pytest.mark.parametrize("prec", ["dd", "ddc", "qd", "qf", "tf"])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_ragged_transposed_bit_exact(mp, oracle, prec, opA, opB):
    """Ragged sizes spanning several tiles, every operand mode, every configuration."""
    K, dt = oracle.PRECS[prec]
    m, n, k = 70, 45, 133
    A = inputs.mp_uniform(7, (k, m) if opA else (m, k), K, dt)
    B = inputs.mp_uniform(8, (n, k) if opB else (k, n), K, dt)
    want = oracle.gemm(prec, A, B, opA, opB)
    for cfg in range(mp.gemm_num_configs(prec)):
        got = host(mp.gemm(prec, dev(A), dev(B), opA, opB, config=cfg))
        assert same_bits(got, want), (cfg, opA, opB)


def test_gemm_degenerate_sizes(mp, oracle):
    import torch

    prec = "qd"
    A = mp.zeros(prec, 5, 0)
    B = mp.zeros(prec, 0, 7)
    C = torch.full((4, 5, 7), 3.0, dtype=torch.float64, device="cuda")
    mp.gemm(prec, A, B, out=C)
    assert not torch.any(C)
    assert mp.gemm(prec, mp.zeros(prec, 0, 3), mp.zeros(prec, 3, 4)).shape == (4, 0, 4)
    with pytest.raises(mp.MPError, match="invalid"):
        mp.gemm(prec, mp.zeros(prec, 3, 3), mp.zeros(prec, 3, 3), opA=2)


@pytest.mark.parametrize("prec,n", [("qd", 2048), ("dd", 4096)])
def test_gemm_full_size_sampled(mp, oracle, prec, n):
    """The benchmark's size and launch configuration: 48 sampled entries recomputed
    by the oracle one by one must match bit for bit."""
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(2, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(2, (n, n), K, dt, stream=inputs.STREAM_B)
    C = host(mp.gemm(prec, dev(A), dev(B)))
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, n - 1], rng.integers(0, n, 46)])
    cols = np.concatenate([[n - 1, 0], rng.integers(0, n, 46)])
    for i, j in zip(rows, cols):
        want = oracle.gemm(prec, A[:, i:i + 1, :], B[:, :, j:j + 1])[:, 0, 0]
        assert same_bits(C[:, i, j], want), (i, j)


def test_peak_microbenchmark_runs(mp):
    rate, ms = mp.peak(0, iters=256)
    assert rate > 0 and ms > 0


@pytest.mark.parametrize("prec", ["dd", "ddc", "td", "qd", "qf"])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 1)])
def test_cgemm3m_bit_exact(mp, oracle, prec, opA, opB):
    """3M complex GEMM (Eq. 3): both parts bit for bit, ragged sizes, op modes."""
    K, dt = oracle.PRECS[prec]
    m, n, k = 37, 45, 29
    sa = (k, m) if opA else (m, k)
    sb = (n, k) if opB else (k, n)
    Ar, Ai = inputs.mp_uniform(1, sa, K, dt), inputs.mp_uniform(2, sa, K, dt)
    Br, Bi = inputs.mp_uniform(3, sb, K, dt), inputs.mp_uniform(4, sb, K, dt)
    wr, wi = oracle.cgemm(prec, Ar, Ai, Br, Bi, opA, opB)
    gr, gi = mp.cgemm(prec, dev(Ar), dev(Ai), dev(Br), dev(Bi), opA, opB)
    assert same_bits(host(gr), wr) and same_bits(host(gi), wi)


def test_cgemm3m_eq2_matrices(mp, oracle):
    """Eq. 2 matrices, QD, n = 96 (entries U * exp(r_n) formed on the GPU with mp_mul,
    which the oracle's multiply reproduces bit for bit)."""
    prec, K, n = "qd", 4, 96

    def mats(seed):
        Ur, Er, Ui, Ei = inputs.complex_eq2(seed, (n, n), K)
        out = []
        for U, E in ((Ur, Er), (Ui, Ei)):
            g = mp.mul(prec, dev(U.reshape(K, -1)), dev(inputs.mp_from_double(E.reshape(-1), K)))
            w = oracle.mul(prec, U.reshape(K, -1), inputs.mp_from_double(E.reshape(-1), K))
            assert same_bits(host(g), w)
            out.append(w.reshape(K, n, n))
        return out

    Ar, Ai = mats(1)
    Br, Bi = mats(2)
    wr, wi = oracle.cgemm(prec, Ar, Ai, Br, Bi)
    gr, gi = mp.cgemm(prec, dev(Ar), dev(Ai), dev(Br), dev(Bi))
    assert same_bits(host(gr), wr) and same_bits(host(gi), wi)


@pytest.mark.parametrize("prec", ["qd", "dd", "qf"])
def test_gemm_tma_config_layouts(mp, oracle, prec):
    """The TMA-staged configuration (4): TMA-eligible layouts (even leading dimensions)
    and ineligible ones (odd lda/ldb: the plain kernel runs instead) both give the
    oracle's bits, in every operand mode, and no TMA wait ever runs out."""
    import torch

    K, dt = oracle.PRECS[prec]
    m, n, k = 67, 53, 90
    for pad in (0, 1, 2):  # storage padded to a leading dimension of cols + pad
        for opA, opB in ((0, 0), (1, 0), (0, 1), (1, 1)):
            sa = (k, m) if opA else (m, k)
            sb = (n, k) if opB else (k, n)
            A = inputs.mp_uniform(11, sa, K, dt)
            B = inputs.mp_uniform(12, sb, K, dt)
            Ap = np.zeros((K, sa[0], sa[1] + pad), dtype=dt)
            Ap[:, :, :sa[1]] = A
            Bp = np.zeros((K, sb[0], sb[1] + pad), dtype=dt)
            Bp[:, :, :sb[1]] = B
            dA = dev(Ap)[:, :, :sa[1]]
            dB = dev(Bp)[:, :, :sb[1]]
            got = host(mp.gemm(prec, dA, dB, opA, opB, config=4))
            assert same_bits(got, oracle.gemm(prec, A, B, opA, opB)), (pad, opA, opB)
    torch.cuda.synchronize()
    assert mp.gemm_tma_timeouts(prec) == 0
