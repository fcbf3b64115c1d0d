"""Seeded synthetic inputs for the multicomponent kernels and their oracle.

This module is the one piece of code that both the CUDA path's callers (tests,
benchmarks) and the CPU oracle's callers use.  It draws random numbers and lays
them out; it contains none of the multicomponent arithmetic itself (no TwoSum,
TwoProd, add or multiply of K-component numbers).  Everything is numpy and
deterministic for a given seed.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: output i of stream `seed`
is mix(seed + (i+1)*GAMMA), which is exactly the i-th output of a SplitMix64
generator whose state starts at `seed`.  Streams for different purposes use
different seeds derived from the caller's seed.

Number layout ("K-array"): a numpy array of shape (K, ...) whose leading axis
holds the components, component 0 the leading (largest) one.  On the device the
same array is K contiguous planes.

Generators:
  * `mp_uniform` -- nonoverlapping K-component numbers: leading component
    uniform in [-1, 1), each lower component u * ulp(previous) / 2 with u
    uniform in [-1, 1).  The scaling is by a power of two, so every component is
    exactly the drawn product (binary64 and binary32 both).
  * `dk_problem` -- real-coefficient polynomials given by their roots: degree
    uniform in [dmin, dmax], floor(n/2) complex roots uniform in the unit disk
    together with their conjugates, one real root uniform in [-1, 1) for odd n,
    and a relative coefficient perturbation delta_i = 1e-30 * g_i, g_i uniform
    in [-1, 1).  The coefficient expansion itself is multicomponent arithmetic
    and is done by the library / oracle builders, not here.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# per-purpose stream offsets, so that e.g. the A and B matrices of one seed differ
STREAM_A = 0x1000
STREAM_B = 0x2000
STREAM_C = 0x3000
STREAM_X = 0x4000
STREAM_Y = 0x5000
STREAM_POLY = 0x6000


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with initial state `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """53-bit uniform doubles in [0, 1): (z >> 11) * 2^-53 (exact)."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [-1, 1): 2u - 1, exact for 53-bit u."""
    return 2.0 * uniform01(seed, count, start) - 1.0


def uniform_pm1_f32(seed: int, count: int, start: int = 0) -> np.ndarray:
    """24-bit uniform binary32 values in [-1, 1): 2 * (z >> 40) * 2^-24 - 1 (exact)."""
    z = splitmix64(seed, count, start)
    u = (z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return (2.0 * u - 1.0).astype(np.float32)


def _ulp_half(x: np.ndarray, mant_bits: int) -> np.ndarray:
    """ulp(x)/2 for normal binary numbers with `mant_bits` significand bits; 0 where x == 0."""
    _, e = np.frexp(x.astype(np.float64))  # x = m * 2^e, 0.5 <= |m| < 1
    half = np.ldexp(np.ones_like(x, dtype=np.float64), (e - mant_bits - 1).astype(np.int32))
    return np.where(x == 0, 0.0, half)


def mp_uniform(seed: int, shape, K: int, dtype=np.float64, stream: int = STREAM_A) -> np.ndarray:
    """Nonoverlapping K-component numbers, returned as an array of shape (K, *shape).

    Component 0 is uniform in [-1, 1); component j+1 = u_j * ulp(component j) / 2
    with u_j uniform in [-1, 1).  A zero component makes all lower ones zero.
    For binary32 components, a component that would fall below the smallest normal
    binary32 number (2^-126) is set to zero together with all lower ones.
    """
    shape = tuple(int(s) for s in np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
    count = int(np.prod(shape)) if len(shape) else 1
    is32 = np.dtype(dtype) == np.float32
    mant = 24 if is32 else 53
    out = np.zeros((K, count), dtype=np.float64)
    base = (int(seed) * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF
    draw = uniform_pm1_f32 if is32 else uniform_pm1
    out[0] = draw(base, count, 0).astype(np.float64)
    for j in range(1, K):
        u = draw(base, count, j * count).astype(np.float64)
        nxt = u * _ulp_half(out[j - 1], mant)  # power-of-two scale: exact
        if is32:
            nxt = np.where(np.abs(nxt) < 2.0 ** -126, 0.0, nxt)
        nxt = np.where(out[j - 1] == 0, 0.0, nxt)
        out[j] = nxt
    return out.astype(dtype).reshape((K,) + shape)


def mp_from_double(x: np.ndarray, K: int, dtype=np.float64) -> np.ndarray:
    """K-array whose leading component is x and lower components are zero."""
    x = np.asarray(x, dtype=dtype)
    out = np.zeros((K,) + x.shape, dtype=dtype)
    out[0] = x
    return out


class DKProblem:
    """Real-coefficient polynomials described by their roots (see module docstring).

    degrees    int64 (npoly,)        degree n_p of polynomial p
    root_off   int64 (npoly+1,)      offsets into `rootdata` / `delta` (sum of degrees)
    coef_off   int64 (npoly+1,)      offsets into the coefficient array: root_off[p] + p
    rootdata   float64 (sum n_p,)    per polynomial: re_0, im_0, re_1, im_1, ... for the
                                     floor(n/2) complex roots (conjugates implied), then
                                     one real root if n is odd
    delta      float64 (sum n_p,)    per polynomial: delta_i = 1e-30 * g_i for i = 0..n-1
    """

    def __init__(self, degrees, rootdata, delta):
        self.degrees = np.asarray(degrees, dtype=np.int64)
        self.root_off = np.zeros(len(self.degrees) + 1, dtype=np.int64)
        np.cumsum(self.degrees, out=self.root_off[1:])
        self.coef_off = self.root_off + np.arange(len(self.degrees) + 1, dtype=np.int64)
        self.rootdata = np.ascontiguousarray(rootdata, dtype=np.float64)
        self.delta = np.ascontiguousarray(delta, dtype=np.float64)

    @property
    def npoly(self) -> int:
        return len(self.degrees)

    def roots_of(self, p: int) -> np.ndarray:
        """The planted roots of polynomial p as complex128 (for loose sanity checks)."""
        n = int(self.degrees[p])
        d = self.rootdata[self.root_off[p]:self.root_off[p + 1]]
        out = []
        for k in range(n // 2):
            r = complex(d[2 * k], d[2 * k + 1])
            out += [r, r.conjugate()]
        if n % 2:
            out.append(complex(d[n - 1], 0.0))
        return np.array(out, dtype=np.complex128)


def dk_problem(seed: int, npoly: int, dmin: int = 10, dmax: int = 500,
               perturb: float = 1e-30) -> DKProblem:
    """Random root sets (uniform in the unit disk, closed under conjugation)."""
    base = (int(seed) * 0x100000001B3 + STREAM_POLY) & 0xFFFFFFFFFFFFFFFF
    u = uniform01(base, npoly, 0)
    degrees = dmin + np.floor(u * (dmax - dmin + 1)).astype(np.int64)
    degrees = np.minimum(degrees, dmax)
    total = int(degrees.sum())
    u1 = uniform01(base + 1, total, 0)
    u2 = uniform01(base + 2, total, 0)
    g = uniform_pm1(base + 3, total, 0)
    rootdata = np.empty(total, dtype=np.float64)
    off = 0
    for n in degrees:
        n = int(n)
        m = n // 2
        rho = np.sqrt(u1[off:off + m])
        th = 2.0 * np.pi * u2[off:off + m]
        rootdata[off:off + 2 * m:2] = rho * np.cos(th)
        rootdata[off + 1:off + 2 * m:2] = rho * np.sin(th)
        if n % 2:
            rootdata[off + n - 1] = 2.0 * u1[off + n - 1] - 1.0
        off += n
    delta = perturb * g
    return DKProblem(degrees, rootdata, delta)


def dk_problem_from_roots(root_lists, perturb: float = 0.0) -> DKProblem:
    """Build a DKProblem from explicit root lists (complex roots given once each,
    their conjugates implied; at most one real root, listed last)."""
    degrees, data = [], []
    for cplx, real in root_lists:
        n = 2 * len(cplx) + (1 if real is not None else 0)
        degrees.append(n)
        for r in cplx:
            data += [float(np.real(r)), float(np.imag(r))]
        if real is not None:
            data.append(float(real))
    total = sum(degrees)
    return DKProblem(degrees, np.array(data, dtype=np.float64),
                     np.full(total, perturb, dtype=np.float64))


def complex_eq2(seed: int, shape, K: int, dtype=np.float64) -> tuple:
    """Factors of the complex GEMM test matrices (Section 3.2, Eq. 2):
    a = exp(r_n) (r_u - 1/2) + exp(r_n) (r_u - 1/2) sqrt(-1), every draw
    independent.  Returns (Ur, Er, Ui, Ei) for the real and imaginary parts:
    U = r_u - 1/2 as a full-precision K-component number (the nonoverlapping
    generator, halved: exact) and E = exp(r_n) in binary64 (r_n standard normal
    by Box-Muller).  The entry is the K-component product U * E, which callers
    form with their multiply (the one place multicomponent arithmetic enters)."""
    shape = tuple(np.atleast_1d(shape).tolist())
    count = int(np.prod(shape))
    base = (int(seed) * 0x100000001B3 + STREAM_C + 7) & 0xFFFFFFFFFFFFFFFF
    out = []
    for part in range(2):
        U = mp_uniform(seed, shape, K, dtype, stream=STREAM_C + 11 + part) * dtype(0.5)
        u1 = uniform01(base, count, (2 * part) * count)
        u2 = uniform01(base, count, (2 * part + 1) * count)
        rn = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
        out += [U, np.exp(rn).reshape(shape)]
    return tuple(out)


def chebyshev_quadrature(n: int):
    """Exact rational coefficients a_0..a_n of the Chebyshev integration problem
    (Section 4.2, Eq. 6), the monic polynomial whose roots are the n Chebyshev
    quadrature nodes: power sums sum x^k = n/(k+1) for even k and 0 for odd k,
    turned into coefficients by Newton's identities:
        a_n = 1,  a_{n-(2k-1)} = 0,
        a_{n-2k} = -(n / (2k)) * sum_{j=1..k} a_{n-2(k-j)} / (2j+1),  k = 1..n/2.
    (The printed Eq. 6 is garbled; this reading keeps its surviving terms and
    gives x^2 - 1/3 for n = 2 and x^3 - x/2 for n = 3.)"""
    from fractions import Fraction

    a = [Fraction(0)] * (n + 1)
    a[n] = Fraction(1)
    for k in range(1, n // 2 + 1):
        s = sum(a[n - 2 * (k - j)] / (2 * j + 1) for j in range(1, k + 1))
        a[n - 2 * k] = -Fraction(n, 2 * k) * s
    return a


def rational_to_mp(values, K: int, dtype=np.float64) -> np.ndarray:
    """K-array of the greedy K-component expansions of exact rationals
    (component j = the rounding of what components 0..j-1 leave)."""
    from fractions import Fraction

    out = np.zeros((K, len(values)), dtype=dtype)
    for i, v in enumerate(values):
        r = Fraction(v)
        for j in range(K):
            c = dtype(float(r))
            out[j, i] = c
            r -= Fraction(float(c))
    return out


def horner_points(seed: int, npoly: int, npts: int) -> np.ndarray:
    """Real evaluation points uniform in [-1, 1): shape (npoly, npts), binary64."""
    base = (int(seed) * 0x100000001B3 + STREAM_X) & 0xFFFFFFFFFFFFFFFF
    return uniform_pm1(base, npoly * npts, 0).reshape(npoly, npts)


def sqrt_fraction(v: int, bits: int = 400):
    """sqrt(v) truncated to `bits` fractional bits, as an exact Fraction (integer
    square root; no floating point)."""
    import math
    from fractions import Fraction

    return Fraction(math.isqrt(int(v) << (2 * bits)), 1 << bits)


def eq1_factors(n: int, K: int, dtype=np.float64):
    """Factors of the real GEMM test matrices of Section 3.1 (Eq. 1),
    a_ij = sqrt5 (i + j - 1) and b_ij = sqrt3 (n - i + 1), i, j = 1..n.

    Returns (s5, s3, t, ia, ib): s5 and s3 are the greedy K-component expansions
    of sqrt5 and sqrt3 (shape (K,)), t the integers 0..2n-1 as a K-array (shape
    (K, 2n)), ia and ib (n, n) index maps with ia[i-1, j-1] = i + j - 1 and
    ib[i-1, j-1] = n - i + 1.  Callers form r5 = s5 * t and r3 = s3 * t with
    their own K-component multiply (the one step of multicomponent arithmetic)
    and gather A = r5[:, ia], B = r3[:, ib]."""
    s5 = rational_to_mp([sqrt_fraction(5)], K, dtype)[:, 0]
    s3 = rational_to_mp([sqrt_fraction(3)], K, dtype)[:, 0]
    t = np.zeros((K, 2 * n), dtype=dtype)
    t[0] = np.arange(2 * n)
    i = np.arange(1, n + 1)[:, None]
    j = np.arange(1, n + 1)[None, :]
    ia = (i + j - 1).astype(np.int64)
    ib = np.broadcast_to(n - i + 1, (n, n)).astype(np.int64)
    return s5, s3, t, ia, ib


def eq1_row_sums(n: int) -> list:
    """S_i = sum_{k=1..n} (i + k - 1)(n - k + 1) for i = 1..n, exact integers: the
    exact product of Eq. 1's matrices is c_ij = sqrt15 * S_i (independent of j)."""
    base = sum(k * (n - k + 1) for k in range(1, n + 1))  # i = 1
    w = n * (n + 1) // 2                                  # sum_k (n - k + 1)
    return [base + (i - 1) * w for i in range(1, n + 1)]
