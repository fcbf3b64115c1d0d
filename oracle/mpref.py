"""ctypes/numpy wrapper around the CPU oracle (mpref.c).

TEST INFRASTRUCTURE ONLY: the oracle is a plain scalar restatement of the
paper's method (Kouya, arXiv 2603.14926) used to check the CUDA library.  Only
tests, the package smoke check and the benchmark's CPU-baseline leg import this
module; the library never does.

Arrays are numpy K-arrays: shape (K, ...) with component 0 leading, C-contiguous,
float64 for dd/ddc/td/qd and float32 for ds/tf/qf.  Complex K-arrays (roots)
have 2K planes: real components then imaginary components.
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import shutil
import subprocess
import tempfile
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "lib")
SRC = [os.path.join(HERE, f) for f in ("mpref.c", "mpref_core.inc", "mpref_dk.inc")]

# precision -> (components, component dtype)
PRECS = {
    "dd": (2, np.float64),
    "ddc": (2, np.float64),
    "td": (3, np.float64),
    "qd": (4, np.float64),
    "tdc": (3, np.float64),
    "qdc": (4, np.float64),
    "ds": (2, np.float32),
    "tf": (3, np.float32),
    "qf": (4, np.float32),
}
DK_PRECS = ("dd", "ddc", "td", "qd")

# per-polynomial solver status codes
DK_CAP, DK_CONVERGED, DK_STAGNATED, DK_TIMEOUT, DK_BREAKDOWN = 0, 1, 2, 3, 4

_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
_lock = threading.Lock()
_libs: dict = {}


def _lib_path(counting: bool) -> str:
    return os.path.join(LIBDIR, "libmpref_count.so" if counting else "libmpref.so")


def build(force: bool = False) -> None:
    """Compile libmpref.so and libmpref_count.so (the counting build) in-tree."""
    os.makedirs(LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SRC)
    for counting in (False, True):
        out = _lib_path(counting)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", *_CFLAGS, *(["-DMPREF_COUNT"] if counting else []),
               os.path.join(HERE, "mpref.c"), "-lm", "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def lib(counting: bool = False) -> ctypes.CDLL:
    with _lock:
        if counting not in _libs:
            build()
            L = ctypes.CDLL(_lib_path(counting))
            _declare(L)
            _libs[counting] = L
        return _libs[counting]


@contextlib.contextmanager
def mutant(replacements):
    """Temporarily route every call to a build of the oracle with source edits
    applied: `replacements` is a list of (file, old, new) string substitutions,
    each of which must match exactly once.  Used by the tests that plant
    mistakes in the oracle to show that its pins catch them."""
    with tempfile.TemporaryDirectory() as d:
        for f in ("mpref.c", "mpref_core.inc", "mpref_dk.inc"):
            shutil.copy(os.path.join(HERE, f), d)
        for f, old, new in replacements:
            path = os.path.join(d, f)
            src = open(path).read()
            if src.count(old) != 1:
                raise ValueError(f"mutation does not match exactly once in {f}: {old!r}")
            open(path, "w").write(src.replace(old, new))
        libs = {}
        for counting in (False, True):
            out = os.path.join(d, f"m{int(counting)}.so")
            subprocess.run(["gcc", *_CFLAGS, *(["-DMPREF_COUNT"] if counting else []),
                            os.path.join(d, "mpref.c"), "-lm", "-o", out], check=True)
            L = ctypes.CDLL(out)
            _declare(L)
            libs[counting] = L
        with _lock:
            saved = dict(_libs)
            _libs.clear()
            _libs.update(libs)
        try:
            yield
        finally:
            with _lock:
                _libs.clear()
                _libs.update(saved)


_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_vp = ctypes.c_void_p
_dbl = ctypes.c_double


def _declare(L):
    for s in PRECS:
        sig = {
            "add": [_i64, _vp, _i64, _vp, _i64, _vp, _i64],
            "mul": [_i64, _vp, _i64, _vp, _i64, _vp, _i64],
            "recip": [_i64, _vp, _i64, _vp, _i64],
            "axpy": [_i64, _vp, _vp, _i64, _vp, _i64],
            "dot": [_i64, _vp, _i64, _vp, _i64, _vp],
            "gemv": [_i64, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _i64],
            "gemm": [ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64,
                     _i64, _vp, _i64, _i64],
            "cgemm": [ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _vp, _vp, _i64, _i64, _vp, _vp,
                      _i64, _i64, _vp, _vp, _i64, _i64],
            "gemm_strassen": [_i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _i64],
            "polyeval": [_i64, _vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _i64],
            "polyeval_estrin": [_i64, _vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _i64],
            "polyeval_backward": [_i64, _vp, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                  _vp, _i64],
        }
        for op, args in sig.items():
            f = getattr(L, f"mpref_{op}_{s}")
            f.argtypes = args
            f.restype = None
    for s in DK_PRECS:
        f = getattr(L, f"mpref_poly_from_roots_{s}")
        f.argtypes = [_i64, _vp, _vp, _vp, _vp, _i64]
        f = getattr(L, f"mpref_aberth_{s}")
        f.argtypes = [_i64, _vp, _i64, _vp, _i64, _dbl]
        f = getattr(L, f"mpref_roots_{s}")
        f.argtypes = [_i64, _vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _dbl, _i32, _i32,
                      _i32, _dbl]
    for t, ct in (("d", ctypes.c_double), ("f", ctypes.c_float)):
        for op in ("two_sum", "quick_two_sum", "two_prod"):
            f = getattr(L, f"mpref_{op}_{t}")
            f.argtypes = [ct, ct, ctypes.POINTER(ct), ctypes.POINTER(ct)]
    L.mpref_dk_cos_sin.argtypes = [_dbl, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]
    L.mpref_dk_nthroot.argtypes = [_dbl, _i64]
    L.mpref_dk_nthroot.restype = _dbl
    L.mpref_count_get.argtypes = [_vp]


def _p(a):
    return a.ctypes.data_as(_vp) if a is not None else None


def _arr(x, prec):
    K, dt = PRECS[prec]
    a = np.ascontiguousarray(x, dtype=dt)
    assert a.shape[0] == K, f"{prec}: expected {K} components, got shape {a.shape}"
    return a


# ---------------------------------------------------------------------------
# EFT primitives (Algorithms 1-3) on scalars
# ---------------------------------------------------------------------------

def _eft(name, a, b, f32=False):
    ct = ctypes.c_float if f32 else ctypes.c_double
    s, e = ct(), ct()
    getattr(lib(), f"mpref_{name}_{'f' if f32 else 'd'}")(a, b, ctypes.byref(s), ctypes.byref(e))
    return s.value, e.value


def two_sum(a, b, f32=False):
    return _eft("two_sum", a, b, f32)


def quick_two_sum(a, b, f32=False):
    return _eft("quick_two_sum", a, b, f32)


def two_prod(a, b, f32=False):
    return _eft("two_prod", a, b, f32)


# ---------------------------------------------------------------------------
# elementwise and linear algebra
# ---------------------------------------------------------------------------

def add(prec, a, b, counting=False):
    a, b = _arr(a, prec), _arr(b, prec)
    c = np.empty_like(a)
    n = a[0].size
    getattr(lib(counting), f"mpref_add_{prec}")(n, _p(a), n, _p(b), n, _p(c), n)
    return c


def mul(prec, a, b, counting=False):
    a, b = _arr(a, prec), _arr(b, prec)
    c = np.empty_like(a)
    n = a[0].size
    getattr(lib(counting), f"mpref_mul_{prec}")(n, _p(a), n, _p(b), n, _p(c), n)
    return c


def recip(prec, a):
    a = _arr(a, prec)
    c = np.empty_like(a)
    n = a[0].size
    getattr(lib(), f"mpref_recip_{prec}")(n, _p(a), n, _p(c), n)
    return c


def op_counts(prec, op, a=None, b=None):
    """(add, sub, mul, fma) operation counts of one `op` ('add' or 'mul') in `prec`,
    summed over the elements of the K-arrays a and b (default: one element equal
    to 1).  The branch-free algorithms count the same on every input; the
    conventional ones (tdc, qdc) depend on their renormalisation's zero tests."""
    K, dt = PRECS[prec]
    a = np.ones((K, 1), dtype=dt) if a is None else a
    b = a if b is None else b
    L = lib(True)
    L.mpref_count_reset()
    (add if op == "add" else mul)(prec, a, b, counting=True)
    out = np.zeros(4, dtype=np.int64)
    L.mpref_count_get(_p(out))
    return tuple(int(v) for v in out)


def axpy(prec, alpha, x, y):
    """Returns alpha*x + y (y is not modified)."""
    K, dt = PRECS[prec]
    x = _arr(x, prec)
    y = _arr(y, prec).copy()
    al = np.ascontiguousarray(np.asarray(alpha, dtype=dt).reshape(K))
    n = x[0].size
    getattr(lib(), f"mpref_axpy_{prec}")(n, _p(al), _p(x), n, _p(y), n)
    return y


def dot(prec, x, y):
    K, dt = PRECS[prec]
    x, y = _arr(x, prec), _arr(y, prec)
    s = np.zeros(K, dtype=dt)
    n = x[0].size
    getattr(lib(), f"mpref_dot_{prec}")(n, _p(x), n, _p(y), n, _p(s))
    return s


def gemv(prec, A, x):
    """A: (K, m, n), x: (K, n) -> y: (K, m)."""
    A, x = _arr(A, prec), _arr(x, prec)
    K, m, n = A.shape
    y = np.zeros((K, m), dtype=A.dtype)
    getattr(lib(), f"mpref_gemv_{prec}")(m, n, _p(A), n, m * n, _p(x), n, _p(y), m)
    return y


def gemm(prec, A, B, opA=0, opB=0, rows=None):
    """C := op(A) op(B).  A is (K, m, k) for opA=0 or (K, k, m) for opA=1; likewise B.
    `rows` = (r0, r1) computes only rows r0..r1-1 of C (returned as (K, r1-r0, n))."""
    A, B = _arr(A, prec), _arr(B, prec)
    K = A.shape[0]
    m, k = (A.shape[1], A.shape[2]) if not opA else (A.shape[2], A.shape[1])
    k2, n = (B.shape[1], B.shape[2]) if not opB else (B.shape[2], B.shape[1])
    assert k == k2
    lda, ldb = A.shape[2], B.shape[2]
    r0, r1 = (0, m) if rows is None else rows
    C = np.zeros((K, r1 - r0, n), dtype=A.dtype)
    if r1 > r0:
        if opA:
            Ap = A.ctypes.data + r0 * A.itemsize
        else:
            Ap = A.ctypes.data + r0 * lda * A.itemsize
        getattr(lib(), f"mpref_gemm_{prec}")(opA, opB, r1 - r0, n, k, _vp(Ap), lda, A[0].size,
                                             _p(B), ldb, B[0].size, _p(C), n, C[0].size)
    return C


def gemm_strassen(prec, A, B, cutoff=32):
    """C := A B by Strassen's recursion (Section 3.1): classical fold below `cutoff`,
    quadrants zero-padded to ceil(size/2) where a dimension is odd."""
    A, B = _arr(A, prec), _arr(B, prec)
    K, m, k = A.shape
    k2, n = B.shape[1], B.shape[2]
    assert k == k2 and cutoff >= 2
    C = np.zeros((K, m, n), dtype=A.dtype)
    if m and n:
        getattr(lib(), f"mpref_gemm_strassen_{prec}")(m, n, k, _p(A), k, max(A[0].size, 1), _p(B), n,
                                                      max(B[0].size, 1), _p(C), n, C[0].size, cutoff)
    return C


def cgemm(prec, Ar, Ai, Br, Bi, opA=0, opB=0):
    """Complex C := op(A) op(B) by the 3M method (Eq. 3); returns (Re C, Im C)."""
    Ar, Ai, Br, Bi = (_arr(x, prec) for x in (Ar, Ai, Br, Bi))
    K = Ar.shape[0]
    m, k = (Ar.shape[1], Ar.shape[2]) if not opA else (Ar.shape[2], Ar.shape[1])
    k2, n = (Br.shape[1], Br.shape[2]) if not opB else (Br.shape[2], Br.shape[1])
    assert k == k2
    Cr = np.zeros((K, m, n), dtype=Ar.dtype)
    Ci = np.zeros_like(Cr)
    getattr(lib(), f"mpref_cgemm_{prec}")(opA, opB, m, n, k, _p(Ar), _p(Ai), Ar.shape[2],
                                          Ar[0].size, _p(Br), _p(Bi), Br.shape[2], Br[0].size,
                                          _p(Cr), _p(Ci), n, max(m * n, 1))
    return Cr, Ci


# ---------------------------------------------------------------------------
# polynomials
# ---------------------------------------------------------------------------

def polyeval(prec, coef_off, coef, npts, x_re, x_im=None):
    coef = _arr(coef, prec)
    off = np.ascontiguousarray(coef_off, dtype=np.int64)
    npoly = len(off) - 1
    x_re = _arr(x_re, prec)
    x_im = _arr(x_im, prec) if x_im is not None else None
    K = coef.shape[0]
    y_re = np.zeros((K, npoly * npts), dtype=coef.dtype)
    y_im = np.zeros_like(y_re) if x_im is not None else None
    getattr(lib(), f"mpref_polyeval_{prec}")(npoly, _p(off), _p(coef), coef.shape[1], npts,
                                             _p(x_re), _p(x_im), x_re.shape[1], _p(y_re),
                                             _p(y_im), y_re.shape[1])
    return (y_re, y_im) if x_im is not None else y_re


def polyeval_estrin(prec, coef_off, coef, npts, x_re, x_im=None):
    """Batched evaluation by Estrin's scheme (same layout and returns as polyeval)."""
    coef = _arr(coef, prec)
    off = np.ascontiguousarray(coef_off, dtype=np.int64)
    npoly = len(off) - 1
    x_re = _arr(x_re, prec)
    x_im = _arr(x_im, prec) if x_im is not None else None
    K = coef.shape[0]
    y_re = np.zeros((K, npoly * npts), dtype=coef.dtype)
    y_im = np.zeros_like(y_re) if x_im is not None else None
    getattr(lib(), f"mpref_polyeval_estrin_{prec}")(npoly, _p(off), _p(coef), coef.shape[1], npts,
                                                    _p(x_re), _p(x_im), x_re.shape[1], _p(y_re),
                                                    _p(y_im), y_re.shape[1])
    return (y_re, y_im) if x_im is not None else y_re


def polyeval_backward(prec, coef_off, coef, npts, x, dy, want_dcoef=True, want_dx=True):
    coef = _arr(coef, prec)
    off = np.ascontiguousarray(coef_off, dtype=np.int64)
    npoly = len(off) - 1
    x, dy = _arr(x, prec), _arr(dy, prec)
    dcoef = np.zeros_like(coef) if want_dcoef else None
    dx = np.zeros_like(x) if want_dx else None
    getattr(lib(), f"mpref_polyeval_backward_{prec}")(
        npoly, _p(off), _p(coef), coef.shape[1], npts, _p(x), x.shape[1], _p(dy), dy.shape[1],
        _p(dcoef), coef.shape[1], _p(dx), x.shape[1])
    return dcoef, dx


def poly_from_roots(prec, prob):
    """Coefficients (K, sum(n_p+1)) of the root-solving workload `prob` (inputs.DKProblem)."""
    K, dt = PRECS[prec]
    coef = np.zeros((K, int(prob.coef_off[-1])), dtype=dt)
    getattr(lib(), f"mpref_poly_from_roots_{prec}")(
        prob.npoly, _p(prob.coef_off), _p(prob.rootdata), _p(prob.delta), _p(coef), coef.shape[1])
    return coef


def aberth(prec, coef, radius=0.0):
    """Aberth starting values (Eq. 5) of one monic polynomial: coef (K, n+1) -> (2K, n).
    radius > 0 replaces Eq. 5's radius."""
    coef = _arr(coef, prec)
    K, n1 = coef.shape
    z = np.zeros((2 * K, n1 - 1), dtype=np.float64)
    getattr(lib(), f"mpref_aberth_{prec}")(n1 - 1, _p(coef), n1, _p(z), n1 - 1, float(radius))
    return z


def roots(prec, coef_off, coef, z0=None, tol=0.0, max_iter=0, stag_window=0, stag_min_iter=0,
          radius=0.0):
    """Durand-Kerner on every polynomial.  Returns (roots (2K, sum n_p), iters, status)."""
    coef = _arr(coef, prec)
    K = coef.shape[0]
    off = np.ascontiguousarray(coef_off, dtype=np.int64)
    npoly = len(off) - 1
    total = int(off[-1]) - npoly
    r = np.zeros((2 * K, max(total, 0)), dtype=np.float64)
    z0a = np.ascontiguousarray(z0, dtype=np.float64) if z0 is not None else None
    iters = np.zeros(npoly, dtype=np.int32)
    status = np.zeros(npoly, dtype=np.int32)
    getattr(lib(), f"mpref_roots_{prec}")(
        npoly, _p(off), _p(coef), coef.shape[1], _p(z0a), z0a.shape[1] if z0a is not None else 0,
        _p(r), max(total, 1), _p(iters), _p(status), float(tol), int(max_iter), int(stag_window),
        int(stag_min_iter), float(radius))
    return r, iters, status


def dk_cos_sin(theta):
    c, s = ctypes.c_double(), ctypes.c_double()
    lib().mpref_dk_cos_sin(theta, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def dk_nthroot(v, m):
    return lib().mpref_dk_nthroot(v, m)
