"""GPU parity for Strassen's recursion (mp_gemm_strassen_P) against the oracle's
recursion: bit for bit at ragged, odd and rectangular sizes, several depths and
every precision; exact on integer matrices at n = 2048; within a Strassen-type
bound of the exact product on sampled entries of the n = 2048 random workload;
argument and workspace errors.
"""

from fractions import Fraction

import numpy as np
import pytest

from exact import SCALE_BITS, mp_ints
from paper_2603_14926_gb300 import inputs
from test_gpu_blas import ALL, dev, host, same_bits

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 64, 32), (65, 65, 65, 32), (100, 77, 90, 16), (33, 40, 35, 8), (8, 8, 8, 2),
          (31, 31, 31, 32), (1, 5, 7, 2), (48, 3, 50, 2)]


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("m,n,k,cutoff", SHAPES)
def test_strassen_bit_exact(mp, oracle, prec, m, n, k, cutoff):
    K, dt = oracle.PRECS[prec]
    A = inputs.mp_uniform(21, (m, k), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(22, (k, n), K, dt, stream=inputs.STREAM_B)
    want = oracle.gemm_strassen(prec, A, B, cutoff)
    got = host(mp.gemm_strassen(prec, dev(A), dev(B), cutoff))
    assert same_bits(got, want)


def test_strassen_strided_output_and_reuse(mp, oracle):
    """C written into a view of a wider matrix; the workspace passed in and reused."""
    import torch

    prec, K = "qd", 4
    m, n, k, cutoff = 70, 66, 45, 12
    A = inputs.mp_uniform(23, (m, k), K)
    B = inputs.mp_uniform(24, (k, n), K)
    want = oracle.gemm_strassen(prec, A, B, cutoff)
    big = torch.full((K, m, n + 5), 7.0, dtype=torch.float64, device="cuda")
    ws = torch.empty(mp.gemm_strassen_workspace(prec, m, n, k, cutoff), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        mp.gemm_strassen(prec, dev(A), dev(B), cutoff, out=big[:, :, :n], ws=ws)
        g = host(big)
        assert same_bits(np.ascontiguousarray(g[:, :, :n]), want)
        assert (g[:, :, n:] == 7.0).all()


def test_strassen_integer_matrices_full_size(mp):
    """n = 2048, cutoff 1024 (two levels, 512 x 512 leaves): integer entries make every
    step exact, so the result is the exact integer product in the leading component."""
    import torch

    n, K = 2048, 4
    rng = np.random.default_rng(31)
    A0 = rng.integers(-40, 41, (n, n))
    B0 = rng.integers(-40, 41, (n, n))
    A = torch.zeros((K, n, n), dtype=torch.float64, device="cuda")
    B = torch.zeros_like(A)
    A[0] = torch.from_numpy(A0.astype(np.float64)).cuda()
    B[0] = torch.from_numpy(B0.astype(np.float64)).cuda()
    C = mp.gemm_strassen("qd", A, B, 1024)
    # binary64 GEMM of the integer planes is exact in any order: every partial sum
    # is an integer below 40 * 40 * 2048 < 2^53
    exact = A[0] @ B[0]
    assert torch.equal(C[0], exact)
    assert not C[1:].any()


def test_strassen_random_full_size_sampled(mp):
    """The n = 2048 random QD workload at cutoff 2048 (one level, 1024 leaves):
    sampled entries within 2^-p (n + 16) 8 n max|a| max|b| of the exact product."""
    n, K = 2048, 4
    A = inputs.mp_uniform(2, (n, n), K, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(2, (n, n), K, stream=inputs.STREAM_B)
    C = host(mp.gemm_strassen("qd", dev(A), dev(B), 2048))
    amax = float(np.abs(A[0]).max()) * 1.01
    bmax = float(np.abs(B[0]).max()) * 1.01
    bound = Fraction(2) ** -212 * (n + 16) * 8 * n * Fraction(amax) * Fraction(bmax)
    for i, j in ((0, 0), (n - 1, n - 1), (5, 1500), (1024, 1023), (1023, 1024)):
        ex = mp_ints(A[:, i, :]).dot(mp_ints(B[:, :, j]))
        got = mp_ints(C[:, i, j][:, None])[0]
        err = Fraction(abs(got * (1 << SCALE_BITS) - ex), 1 << (2 * SCALE_BITS))
        assert err <= bound, (i, j, float(err))


def test_strassen_argument_errors(mp):
    import torch

    A = mp.empty("dd", 40, 40)
    B = mp.empty("dd", 40, 40)
    with pytest.raises(RuntimeError):
        mp.gemm_strassen("dd", A, B, 1)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        mp.gemm_strassen("dd", A, B, 8, ws=small)
    assert mp.gemm_strassen_workspace("dd", 40, 40, 40, 41) == 0
    C = mp.gemm_strassen("dd", mp.empty("dd", 3, 0), mp.empty("dd", 0, 4), 2)
    assert not host(C).any()
