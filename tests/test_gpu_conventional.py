"""GPU parity for the conventional (renormalising) triple and quad word, tdc and
qdc: Algorithms 9 and 10 and the QD library's quad-word add and multiply, the
"standard" side of Table 4's standard / BF ratio.

Their renormalisations branch on zero tests, so besides the random families the
inputs include ones whose exact results need fewer than K components (every
branch of the renormalisation is taken).  Elementwise ops, AXPY, GEMM and
Strassen's recursion must match the oracle bit for bit; dot and GEMV agree with
the exact sum within (4n + 16) 2^-p sum |x_i y_i|.
"""

from fractions import Fraction

import numpy as np
import pytest

from cases import families
from exact import SCALE_BITS, mp_ints
from paper_2603_14926_gb300 import inputs

pytestmark = pytest.mark.gpu

CONV = ["tdc", "qdc"]


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def same_bits(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def sparse_family(K, n, seed):
    """Numbers with one or two nonzero leading components and integers: their sums
    and products often need fewer than K components, so the renormalisation's
    zero tests go both ways."""
    rng = np.random.default_rng(seed)
    a = np.zeros((K, n))
    b = np.zeros((K, n))
    a[0] = rng.integers(-8, 9, n) * np.exp2(rng.integers(-3, 4, n))
    b[0] = rng.standard_normal(n)
    b[1, ::2] = b[0, ::2] * 2.0 ** -70
    a[1, 1::3] = 2.0 ** -60
    return a, b


@pytest.mark.parametrize("prec", CONV)
def test_conventional_elementwise_bit_exact(mp, oracle, prec):
    K, dt = oracle.PRECS[prec]
    fams = families(oracle, prec, n=1537, seed=3, limits=True)
    fams.append(("sparse",) + sparse_family(K, 1537, 5))
    for name, a, b in fams:
        da, db = dev(a), dev(b)
        assert same_bits(host(mp.add(prec, da, db)), oracle.add(prec, a, b)), name
        assert same_bits(host(mp.mul(prec, da, db)), oracle.mul(prec, a, b)), name
    x = inputs.mp_uniform(9, 5003, K, dt) * np.exp2((np.arange(5003) % 61) - 30).astype(dt)
    assert same_bits(host(mp.recip(prec, dev(x))), oracle.recip(prec, x))


@pytest.mark.parametrize("prec", CONV)
def test_conventional_axpy_bit_exact(mp, oracle, prec):
    K, dt = oracle.PRECS[prec]
    n = 100_003
    x = inputs.mp_uniform(1, n, K, dt, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(1, n, K, dt, stream=inputs.STREAM_Y)
    alpha = inputs.mp_uniform(2, 1, K, dt)[:, 0]
    dy = dev(y)
    mp.axpy(prec, alpha, dev(x), dy)
    assert same_bits(host(dy), oracle.axpy(prec, alpha, x, y))


@pytest.mark.parametrize("prec", CONV)
@pytest.mark.parametrize("n", [1, 255, 70_001])
def test_conventional_dot_within_bound(mp, oracle, prec, n):
    K, dt = oracle.PRECS[prec]
    p = 53 * K
    x = inputs.mp_uniform(4, n, K, dt, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(4, n, K, dt, stream=inputs.STREAM_Y)
    g = host(mp.dot(prec, dev(x), dev(y)))
    ex = int(mp_ints(x).dot(mp_ints(y)))
    gi = int(mp_ints(g[:, None])[0])
    err = float(Fraction(abs(gi * (1 << SCALE_BITS) - ex), 1 << (2 * SCALE_BITS)))
    mag = float(np.abs(x).sum(0) @ np.abs(y).sum(0))
    assert err <= (4 * n + 16) * 2.0 ** -p * mag


@pytest.mark.parametrize("prec", CONV)
def test_conventional_gemv_within_bound(mp, oracle, prec):
    K, dt = oracle.PRECS[prec]
    p = 53 * K
    m, n = 21, 1029
    A = inputs.mp_uniform(5, (m, n), K, dt)
    x = inputs.mp_uniform(6, n, K, dt, stream=inputs.STREAM_X)
    g = host(mp.gemv(prec, dev(A), dev(x)))
    Ai, xi = mp_ints(A), mp_ints(x)
    absA, absx = np.abs(A).sum(0), np.abs(x).sum(0)
    for i in range(m):
        gi = int(mp_ints(g[:, i:i + 1])[0])
        err = float(Fraction(abs(gi * (1 << SCALE_BITS) - int(Ai[i].dot(xi))), 1 << (2 * SCALE_BITS)))
        assert err <= (4 * n + 16) * 2.0 ** -p * float(absA[i] @ absx)


@pytest.mark.parametrize("prec", CONV)
def test_conventional_gemm_every_config_bit_exact(mp, oracle, prec):
    """n = 64 (seed 0) and a ragged transposed product in every tile
    configuration, native and hybrid engines, plain and TMA-staged."""
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(0, (64, 64), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(0, (64, 64), K, dt, stream=inputs.STREAM_B)
    want = oracle.gemm(prec, A, B)
    m, n, k = 70, 45, 133
    A2 = inputs.mp_uniform(7, (k, m), K, dt)
    B2 = inputs.mp_uniform(8, (n, k), K, dt)
    want2 = oracle.gemm(prec, A2, B2, 1, 1)
    for cfg in range(mp.gemm_num_configs(prec)):
        assert same_bits(host(mp.gemm(prec, dev(A), dev(B), config=cfg)), want), cfg
        assert same_bits(host(mp.gemm(prec, dev(A2), dev(B2), 1, 1, config=cfg)), want2), cfg


@pytest.mark.parametrize("prec", CONV)
def test_conventional_gemm_fallback_and_sparse(mp, oracle, prec):
    """Rows scaled by 2^-1000 (the hybrid engine recomputes those threads on the
    FP64 pipe) and integer-valued operands (exact products, renormalisations on
    their zero branches) stay bit-identical in the built-in configuration."""
    K, dt = oracle.PRECS[prec]
    m, n, k = 40, 36, 50
    A = inputs.mp_uniform(11, (m, k), K)
    B = inputs.mp_uniform(12, (k, n), K)
    A[:, :5, :] *= 2.0 ** -1000
    before = mp.gemm_hybrid_fallbacks(prec)
    assert same_bits(host(mp.gemm(prec, dev(A), dev(B), config=-1)), oracle.gemm(prec, A, B))
    assert mp.gemm_hybrid_fallbacks(prec) > before
    rng = np.random.default_rng(3)
    Ai = np.zeros((K, m, k))
    Bi = np.zeros((K, k, n))
    Ai[0] = rng.integers(-9, 10, (m, k))
    Bi[0] = rng.integers(-9, 10, (k, n)) * 2.0 ** -3
    Bi[1, ::2] = Bi[0, ::2] * 2.0 ** -80
    assert same_bits(host(mp.gemm(prec, dev(Ai), dev(Bi), config=-1)), oracle.gemm(prec, Ai, Bi))


@pytest.mark.parametrize("prec", CONV)
def test_conventional_strassen_bit_exact(mp, oracle, prec):
    """Strassen's recursion at the paper's cutoff 32 on odd sizes (padded quadrants)."""
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(3, (65, 65), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(3, (65, 65), K, dt, stream=inputs.STREAM_B)
    got = host(mp.gemm_strassen(prec, dev(A), dev(B), cutoff=32))
    assert same_bits(got, oracle.gemm_strassen(prec, A, B, 32))


@pytest.mark.parametrize("prec", CONV)
def test_conventional_gemm_full_size_sampled(mp, oracle, prec):
    """n = 2048, the size the benchmark compares branch-free and conventional
    arithmetic at: 24 sampled entries (corners included) bit for bit."""
    K, dt = oracle.PRECS[prec]
    n = 2048
    A = inputs.mp_uniform(2, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(2, (n, n), K, dt, stream=inputs.STREAM_B)
    C = host(mp.gemm(prec, dev(A), dev(B)))
    rng = np.random.default_rng(1)
    rows = np.concatenate([[0, n - 1, 0, n - 1], rng.integers(0, n, 20)])
    cols = np.concatenate([[0, n - 1, n - 1, 0], rng.integers(0, n, 20)])
    for i, j in zip(rows, cols):
        want = oracle.gemm(prec, A[:, i:i + 1, :], B[:, :, j:j + 1])[:, 0, 0]
        assert same_bits(C[:, i, j], want), (i, j)
