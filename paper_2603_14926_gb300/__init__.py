"""paper_2603_14926_gb300 -- branch-free multicomponent arithmetic on GB300.

Thin Python binding over libmpgpu.so (C ABI declared in include/mpgpu.h): every
function here only checks shapes, picks plane strides and the current CUDA
stream, and calls the library entry point of the same name.  All arithmetic
runs in the library's CUDA kernels; there is no fallback.  PyTorch provides the
device memory and streams.

Numbers are "K-arrays": torch tensors of shape (K, ...) on a CUDA device,
float64 for dd/ddc/td/qd/tdc/qdc and float32 for ds/tf/qf, each component plane
contiguous (component 0 leading).  Complex K-arrays have 2K planes.
"""

from __future__ import annotations

import ctypes
import os
import threading

PRECS = {"dd": (2, "float64"), "ddc": (2, "float64"), "td": (3, "float64"),
         "qd": (4, "float64"), "tdc": (3, "float64"), "qdc": (4, "float64"),
         "ds": (2, "float32"), "tf": (3, "float32"), "qf": (4, "float32")}
# conventional (renormalising) precisions: elementwise, BLAS-1, GEMV, GEMM and
# Strassen families only
CONVENTIONAL = ("tdc", "qdc")
DK_PRECS = ("dd", "ddc", "td", "qd")
# per-polynomial solver status codes (mp_roots_P)
DK_CAP, DK_CONVERGED, DK_STAGNATED, DK_TIMEOUT, DK_BREAKDOWN = 0, 1, 2, 3, 4
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "workspace too small",
          4: "watchdog expired", 5: "not supported"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmpgpu.so")
_lib = None
_lock = threading.Lock()


class MPError(RuntimeError):
    def __init__(self, fn, code, cuda=0):
        super().__init__(f"{fn}: {STATUS.get(code, code)}" + (f" (cudaError {cuda})" if cuda else ""))
        self.code = code


def build(force: bool = False) -> str:
    from . import buildlib as _b

    return _b.build(force=force)


_i64, _i32, _vp, _dbl, _int = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double, ctypes.c_int


class RootsOpts(ctypes.Structure):
    """mp_roots_opts (include/mpgpu.h)."""
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("stag_window", ctypes.c_int32), ("stag_min_iter", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("radius", ctypes.c_double),
                ("watchdog_cycles", ctypes.c_int64), ("max_degree", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("sort", ctypes.c_int32), ("engine", ctypes.c_int32)]


def _declare(L):
    for p in PRECS:
        sigs = {
            "add": [_i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp],
            "mul": [_i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp],
            "recip": [_i64, _vp, _i64, _vp, _i64, _vp],
            "axpy": [_i64, _vp, _vp, _i64, _vp, _i64, _vp],
            "dot": [_i64, _vp, _i64, _vp, _i64, _vp, _vp, ctypes.c_size_t, _vp],
            "gemv": [_i64, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp],
            "gemm": [_int, _int, _i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp, _i64,
                     _i64, _vp],
            "gemm_ex": [_int, _int, _i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp,
                        _i64, _i64, _int, _vp],
            "cgemm": [_int, _int, _i64, _i64, _i64, _vp, _vp, _i64, _i64, _vp, _vp, _i64, _i64,
                      _vp, _vp, _i64, _i64, _vp, ctypes.c_size_t, _vp],
            "gemm_strassen": [_i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64,
                              _i64, _vp, ctypes.c_size_t, _vp],
            "polyeval": [_i64, _vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _i64, _vp],
            "polyeval_estrin": [_i64, _vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _i64, _vp],
            "polyeval_backward": [_i64, _vp, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                  _vp, _i64, _vp, ctypes.c_size_t, _vp],
        }
        for name, args in sigs.items():
            f = getattr(L, f"mp_{name}_{p}", None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = _int
        getattr(L, f"mp_dot_workspace_{p}").argtypes = [_i64]
        getattr(L, f"mp_dot_workspace_{p}").restype = ctypes.c_size_t
        if p not in CONVENTIONAL:
            getattr(L, f"mp_polyeval_backward_workspace_{p}").argtypes = [_i64, _i64]
            getattr(L, f"mp_polyeval_backward_workspace_{p}").restype = ctypes.c_size_t
            getattr(L, f"mp_cgemm_workspace_{p}").argtypes = [_i64, _i64, _i64, _i64]
            getattr(L, f"mp_cgemm_workspace_{p}").restype = ctypes.c_size_t
        getattr(L, f"mp_gemm_strassen_workspace_{p}").argtypes = [_i64, _i64, _i64, _i64]
        getattr(L, f"mp_gemm_strassen_workspace_{p}").restype = ctypes.c_size_t
        getattr(L, f"mp_gemm_num_configs_{p}").restype = _int
        getattr(L, f"mp_gemm_tma_timeouts_{p}").argtypes = [ctypes.POINTER(ctypes.c_uint)]
        getattr(L, f"mp_gemm_tma_timeouts_{p}").restype = _int
        getattr(L, f"mp_gemm_hybrid_fallbacks_{p}").argtypes = [ctypes.POINTER(ctypes.c_uint)]
        getattr(L, f"mp_gemm_hybrid_fallbacks_{p}").restype = _int
        getattr(L, f"mp_gemm_config_name_{p}").argtypes = [_int]
        getattr(L, f"mp_gemm_config_name_{p}").restype = ctypes.c_char_p
    for p in DK_PRECS:
        f = getattr(L, f"mp_poly_from_roots_{p}", None)
        if f is None:
            continue
        f.argtypes = [_i64, _vp, _vp, _vp, _i32, _vp, _i64, _vp]
        f.restype = _int
        f = getattr(L, f"mp_roots_init_{p}")
        f.argtypes = [_i64, _vp, _vp, _i64, _dbl, _i32, _vp, _i64, _vp]
        f.restype = _int
        f = getattr(L, f"mp_roots_workspace_{p}")
        f.argtypes = [_i64]
        f.restype = ctypes.c_size_t
        f = getattr(L, f"mp_roots_workspace_deg_{p}")
        f.argtypes = [_i64, _i32]
        f.restype = ctypes.c_size_t
        getattr(L, f"mp_roots_max_degree_{p}").restype = _i32
        f = getattr(L, f"mp_roots_{p}")
        f.argtypes = [_i64, _vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _vp,
                      ctypes.POINTER(RootsOpts), _vp, ctypes.c_size_t, _vp]
        f.restype = _int
    L.mp_roots_hybrid_fallbacks.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
    L.mp_roots_hybrid_fallbacks.restype = _int
    L.mp_peak_run.argtypes = [_int, _i64, _int, _int, ctypes.POINTER(ctypes.c_float),
                              ctypes.POINTER(ctypes.c_double), _vp]
    L.mp_peak_run.restype = _int
    L.mp_status_str.restype = ctypes.c_char_p
    L.mp_version.restype = ctypes.c_char_p
    L.mp_last_cuda_error.restype = _int
    L.mp_sm_count.restype = _int


def load():
    """Load libmpgpu.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2603_14926_gb300.build() first")
            L = ctypes.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
        return _lib


def lib():
    return _lib if _lib is not None else load()


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _torch():
    import torch

    return torch


def _stream():
    return _torch().cuda.current_stream().cuda_stream


def _call(name, *args):
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        raise MPError(name, rc, lib().mp_last_cuda_error() if rc == 2 else 0)


def _dtype(prec):
    t = _torch()
    return t.float64 if PRECS[prec][1] == "float64" else t.float32


def _check(prec, x, name, ndim=None):
    t = _torch()
    K = PRECS[prec][0]
    if not isinstance(x, t.Tensor) or not x.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if x.dtype != _dtype(prec):
        raise TypeError(f"{name}: expected {_dtype(prec)} for {prec}, got {x.dtype}")
    if x.shape[0] != K:
        raise ValueError(f"{name}: expected {K} component planes, got shape {tuple(x.shape)}")
    if ndim is not None and x.dim() != ndim:
        raise ValueError(f"{name}: expected {ndim} dims, got {tuple(x.shape)}")
    if x.dim() >= 2 and x.shape[-1] > 1 and x.stride(-1) != 1:
        raise ValueError(f"{name}: the last dimension must be contiguous (unit stride)")
    if x.dim() == 2 and not x[0].is_contiguous():
        raise ValueError(f"{name}: each component plane must be contiguous")
    return x


def _ps(x):
    """Plane stride in elements."""
    return x.stride(0) if x.shape[0] > 1 else x[0].numel()


def _ptr(x):
    return None if x is None else x.data_ptr()


def empty(prec, *shape, device="cuda"):
    K = PRECS[prec][0]
    return _torch().empty((K, *shape), dtype=_dtype(prec), device=device)


def zeros(prec, *shape, device="cuda"):
    K = PRECS[prec][0]
    return _torch().zeros((K, *shape), dtype=_dtype(prec), device=device)


# ---------------------------------------------------------------------------
# elementwise, AXPY, dot, GEMV, GEMM
# ---------------------------------------------------------------------------

def _ew(name, prec, a, b=None, out=None):
    _check(prec, a, "a")
    if b is not None:
        _check(prec, b, "b")
        if b.shape != a.shape:
            raise ValueError("a and b differ in shape")
    out = empty(prec, *a.shape[1:], device=a.device) if out is None else _check(prec, out, "out")
    n = a[0].numel()
    if b is None:
        _call(f"mp_{name}_{prec}", n, _ptr(a), _ps(a), _ptr(out), _ps(out), _stream())
    else:
        _call(f"mp_{name}_{prec}", n, _ptr(a), _ps(a), _ptr(b), _ps(b), _ptr(out), _ps(out),
              _stream())
    return out


def add(prec, a, b, out=None):
    return _ew("add", prec, a, b, out)


def mul(prec, a, b, out=None):
    return _ew("mul", prec, a, b, out)


def recip(prec, a, out=None):
    return _ew("recip", prec, a, None, out)


def axpy(prec, alpha, x, y):
    """y := alpha * x + y in place; alpha is a sequence of K host numbers."""
    _check(prec, x, "x")
    _check(prec, y, "y")
    K = PRECS[prec][0]
    ct = ctypes.c_double if PRECS[prec][1] == "float64" else ctypes.c_float
    al = (ct * K)(*[float(v) for v in alpha])
    _call(f"mp_axpy_{prec}", x[0].numel(), ctypes.cast(al, _vp), _ptr(x), _ps(x), _ptr(y), _ps(y),
          _stream())
    return y


def dot_workspace(prec, n):
    return int(getattr(lib(), f"mp_dot_workspace_{prec}")(n))


def dot(prec, x, y, out=None, ws=None):
    _check(prec, x, "x")
    _check(prec, y, "y")
    t = _torch()
    n = x[0].numel()
    K = PRECS[prec][0]
    out = empty(prec, device=x.device) if out is None else out
    nb = dot_workspace(prec, n)
    if ws is None:
        ws = t.empty(nb, dtype=t.uint8, device=x.device)
    _call(f"mp_dot_{prec}", n, _ptr(x), _ps(x), _ptr(y), _ps(y), _ptr(out), _ptr(ws),
          ws.numel() * ws.element_size(), _stream())
    return out.reshape(K)


def gemv(prec, A, x, out=None):
    _check(prec, A, "A", 3)
    _check(prec, x, "x", 2)
    K, m, n = A.shape
    if A[0].stride(1) != 1:
        raise ValueError("A rows must be contiguous")
    out = empty(prec, m, device=A.device) if out is None else out
    _call(f"mp_gemv_{prec}", m, n, _ptr(A), A[0].stride(0), _ps(A), _ptr(x), _ps(x), _ptr(out),
          _ps(out), _stream())
    return out


def gemm_num_configs(prec):
    return int(getattr(lib(), f"mp_gemm_num_configs_{prec}")())


def gemm_tma_timeouts(prec):
    """How many TMA waits of the TMA-staged GEMM ran out (synchronizes; 0 normally)."""
    v = ctypes.c_uint()
    _call(f"mp_gemm_tma_timeouts_{prec}", ctypes.byref(v))
    return v.value


def gemm_hybrid_fallbacks(prec):
    """How many GEMM threads of this precision took the hybrid engine's FP64
    recomputation since the library was loaded (synchronizes)."""
    v = ctypes.c_uint()
    _call(f"mp_gemm_hybrid_fallbacks_{prec}", ctypes.byref(v))
    return v.value


def gemm_config_name(prec, c):
    return getattr(lib(), f"mp_gemm_config_name_{prec}")(c).decode()


def gemm(prec, A, B, opA=0, opB=0, out=None, config=None):
    """C := op(A) op(B).  A is (K, m, k) for opA=0 or (K, k, m) for opA=1; likewise B.
    config: a tile configuration index, -1 for the built-in choice, or None for the
    autotuner's cached choice for this shape (built-in when none is cached)."""
    _check(prec, A, "A", 3)
    _check(prec, B, "B", 3)
    m, k = (A.shape[1], A.shape[2]) if not opA else (A.shape[2], A.shape[1])
    k2, n = (B.shape[1], B.shape[2]) if not opB else (B.shape[2], B.shape[1])
    if k != k2:
        raise ValueError(f"inner dimensions differ: {k} vs {k2}")
    for X, nm in ((A, "A"), (B, "B")):
        if X[0].stride(1) != 1:
            raise ValueError(f"{nm} rows must be contiguous")
    out = empty(prec, m, n, device=A.device) if out is None else _check(prec, out, "out", 3)
    if config is None:
        from .tune import best_gemm_config

        config = best_gemm_config(prec, m, n, k)
    _call(f"mp_gemm_ex_{prec}", int(opA), int(opB), m, n, k, _ptr(A), A[0].stride(0), _ps(A),
          _ptr(B), B[0].stride(0), _ps(B), _ptr(out), out[0].stride(0), _ps(out), int(config),
          _stream())
    return out


def gemm_strassen_workspace(prec, m, n, k, cutoff=32):
    return int(getattr(lib(), f"mp_gemm_strassen_workspace_{prec}")(m, n, k, cutoff))


def gemm_strassen(prec, A, B, cutoff=32, out=None, ws=None):
    """Real C := A B by Strassen's recursion (classical GEMM below `cutoff`,
    zero-padded quadrants for odd sizes); A (K, m, k), B (K, k, n)."""
    t = _torch()
    _check(prec, A, "A", 3)
    _check(prec, B, "B", 3)
    m, k = A.shape[1], A.shape[2]
    k2, n = B.shape[1], B.shape[2]
    if k != k2:
        raise ValueError(f"inner dimensions differ: {k} vs {k2}")
    C = out if out is not None else empty(prec, m, n, device=A.device)
    nb = gemm_strassen_workspace(prec, m, n, k, cutoff)
    if ws is None:
        ws = t.empty(max(nb, 1), dtype=t.uint8, device=A.device)
    _call(f"mp_gemm_strassen_{prec}", m, n, k, _ptr(A), A[0].stride(0), _ps(A), _ptr(B), B[0].stride(0),
          _ps(B), _ptr(C), C[0].stride(0), _ps(C), int(cutoff), _ptr(ws), ws.numel(), _stream())
    return C


def cgemm(prec, Ar, Ai, Br, Bi, opA=0, opB=0, out=None, ws=None):
    """Complex C := op(A) op(B) by the 3M method; returns (Re C, Im C)."""
    t = _torch()
    for X, nm in ((Ar, "Ar"), (Ai, "Ai"), (Br, "Br"), (Bi, "Bi")):
        _check(prec, X, nm, 3)
    if Ai.shape != Ar.shape or Bi.shape != Br.shape or Ai.stride() != Ar.stride() or Bi.stride() != Br.stride():
        raise ValueError("real and imaginary parts must share shape and strides")
    m, k = (Ar.shape[1], Ar.shape[2]) if not opA else (Ar.shape[2], Ar.shape[1])
    k2, n = (Br.shape[1], Br.shape[2]) if not opB else (Br.shape[2], Br.shape[1])
    if k != k2:
        raise ValueError(f"inner dimensions differ: {k} vs {k2}")
    Cr, Ci = out if out is not None else (empty(prec, m, n, device=Ar.device),
                                          empty(prec, m, n, device=Ar.device))
    nb = int(getattr(lib(), f"mp_cgemm_workspace_{prec}")(m, n, _ps(Ar), _ps(Br)))
    if ws is None:
        ws = t.empty(max(nb, 1), dtype=t.uint8, device=Ar.device)
    _call(f"mp_cgemm_{prec}", int(opA), int(opB), m, n, k, _ptr(Ar), _ptr(Ai), Ar[0].stride(0), _ps(Ar),
          _ptr(Br), _ptr(Bi), Br[0].stride(0), _ps(Br), _ptr(Cr), _ptr(Ci), Cr[0].stride(0), _ps(Cr),
          _ptr(ws), ws.numel(), _stream())
    return Cr, Ci


# ---------------------------------------------------------------------------
# polynomials and roots
# ---------------------------------------------------------------------------

def polyeval(prec, coef_off, coef, npts, x_re, x_im=None, scheme="horner"):
    """Batched evaluation, Horner's rule (default) or Estrin's scheme
    (scheme="estrin"); coef_off is a CUDA int64 tensor (npoly+1)."""
    _check(prec, coef, "coef", 2)
    _check(prec, x_re, "x_re", 2)
    npoly = coef_off.numel() - 1
    y_re = empty(prec, npoly * npts, device=coef.device)
    y_im = None
    if x_im is not None:
        _check(prec, x_im, "x_im", 2)
        y_im = empty(prec, npoly * npts, device=coef.device)
    if scheme not in ("horner", "estrin"):
        raise ValueError(f"unknown scheme {scheme!r}")
    fn = f"mp_polyeval_{prec}" if scheme == "horner" else f"mp_polyeval_estrin_{prec}"
    _call(fn, npoly, _ptr(coef_off), _ptr(coef), _ps(coef), npts, _ptr(x_re),
          _ptr(x_im), _ps(x_re), _ptr(y_re), _ptr(y_im), _ps(y_re), _stream())
    return (y_re, y_im) if x_im is not None else y_re


def polyeval_backward_workspace(prec, npoly, npts):
    return int(getattr(lib(), f"mp_polyeval_backward_workspace_{prec}")(npoly, npts))


def polyeval_backward(prec, coef_off, coef, npts, x, dy, want_dcoef=True, want_dx=True, ws=None):
    """Adjoint of real-argument polyeval: returns (dcoef, dx) (None where not wanted).
    `ws` is accepted and unused: the adjoint needs no workspace."""
    t = _torch()
    _check(prec, coef, "coef", 2)
    _check(prec, x, "x", 2)
    _check(prec, dy, "dy", 2)
    npoly = coef_off.numel() - 1
    dcoef = empty(prec, coef.shape[1], device=coef.device) if want_dcoef else None
    dx = empty(prec, x.shape[1], device=coef.device) if want_dx else None
    nb = polyeval_backward_workspace(prec, npoly, npts) if want_dcoef else 0
    if ws is None and nb:
        ws = t.empty(nb, dtype=t.uint8, device=coef.device)
    _call(f"mp_polyeval_backward_{prec}", npoly, _ptr(coef_off), _ptr(coef), _ps(coef), npts,
          _ptr(x), _ps(x), _ptr(dy), _ps(dy), _ptr(dcoef), _ps(dcoef) if dcoef is not None else 0,
          _ptr(dx), _ps(dx) if dx is not None else 0, _ptr(ws),
          ws.numel() * ws.element_size() if ws is not None else 0, _stream())
    return dcoef, dx


def poly_from_roots(prec, coef_off, rootdata, delta, max_degree, total):
    """Coefficients (K, total) of the root-solving workload (see inputs.DKProblem);
    coef_off, rootdata and delta are CUDA tensors, max_degree and total host ints."""
    coef = empty(prec, total, device=rootdata.device)
    npoly = coef_off.numel() - 1
    _call(f"mp_poly_from_roots_{prec}", npoly, _ptr(coef_off), _ptr(rootdata), _ptr(delta),
          int(max_degree), _ptr(coef), _ps(coef), _stream())
    return coef


def roots_init(prec, coef_off, coef, max_degree, radius=0.0):
    _check(prec, coef, "coef", 2)
    K = PRECS[prec][0]
    npoly = coef_off.numel() - 1
    total = coef.shape[1] - npoly
    z = _torch().zeros((2 * K, max(total, 1)), dtype=coef.dtype, device=coef.device)
    _call(f"mp_roots_init_{prec}", npoly, _ptr(coef_off), _ptr(coef), _ps(coef), float(radius),
          int(max_degree), _ptr(z), z.stride(0), _stream())
    return z[:, :total]


def roots_workspace(prec, npoly, max_degree=None):
    """Workspace bytes of mp_roots_P for npoly polynomials (and, above the
    shared-memory bound, degrees up to max_degree)."""
    if max_degree is None:
        return int(getattr(lib(), f"mp_roots_workspace_{prec}")(npoly))
    return int(getattr(lib(), f"mp_roots_workspace_deg_{prec}")(npoly, int(max_degree)))


def roots_max_degree(prec):
    return int(getattr(lib(), f"mp_roots_max_degree_{prec}")())


def roots(prec, coef_off, coef, max_degree, z0=None, tol=0.0, max_iter=0, stag_window=0,
          stag_min_iter=0, mode=0, radius=0.0, watchdog_cycles=0, threads=0, blocks_per_sm=0,
          sort=0, out=None, ws=None, engine=0):
    """Durand-Kerner on every polynomial; returns (roots (2K, total), iters, status)."""
    t = _torch()
    _check(prec, coef, "coef", 2)
    K = PRECS[prec][0]
    npoly = coef_off.numel() - 1
    total = coef.shape[1] - npoly
    dev = coef.device
    r = t.zeros((2 * K, max(total, 1)), dtype=coef.dtype, device=dev) if out is None else out
    iters = t.zeros(npoly, dtype=t.int32, device=dev)
    status = t.zeros(npoly, dtype=t.int32, device=dev)
    nb = roots_workspace(prec, npoly, max_degree)
    if ws is None:
        ws = t.empty(max(nb, 1), dtype=t.uint8, device=dev)
    o = RootsOpts(tol, max_iter, stag_window, stag_min_iter, mode, radius, watchdog_cycles,
                  int(max_degree), threads, blocks_per_sm, sort, engine)
    _call(f"mp_roots_{prec}", npoly, _ptr(coef_off), _ptr(coef), _ps(coef), _ptr(z0),
          z0.stride(0) if z0 is not None else 0, _ptr(r), r.stride(0), _ptr(iters),
          _ptr(status), ctypes.byref(o), _ptr(ws), ws.numel(), _stream())
    return r[:, :total], iters, status


def roots_hybrid_fallbacks():
    """Root updates recomputed on the FP64 pipe since the library was loaded
    (the hybrid engine left its domain; synchronizes)."""
    v = ctypes.c_ulonglong()
    _call("mp_roots_hybrid_fallbacks", ctypes.byref(v))
    return v.value


class RootsGraph:
    """The persistent batched Durand-Kerner solve (work-queue reset, optional
    descending-degree order, one persistent launch) captured once in a CUDA graph
    and replayed.  Outputs live in preallocated tensors: .roots, .iters, .status.
    Options as for roots(); mode must be 0."""

    def __init__(self, prec, coef_off, coef, max_degree, z0=None, tol=0.0, max_iter=0,
                 stag_window=0, stag_min_iter=0, radius=0.0, watchdog_cycles=0, threads=0,
                 blocks_per_sm=0, sort=1, engine=0):
        t = _torch()
        _check(prec, coef, "coef", 2)
        K = PRECS[prec][0]
        self.prec, self.coef_off, self.coef, self.z0 = prec, coef_off, coef, z0
        self.npoly = coef_off.numel() - 1
        self.total = coef.shape[1] - self.npoly
        dev = coef.device
        self._r = t.zeros((2 * K, max(self.total, 1)), dtype=coef.dtype, device=dev)
        self.iters = t.zeros(self.npoly, dtype=t.int32, device=dev)
        self.status = t.zeros(self.npoly, dtype=t.int32, device=dev)
        self.ws = t.empty(max(roots_workspace(prec, self.npoly, max_degree), 1), dtype=t.uint8, device=dev)
        self.opts = RootsOpts(tol, max_iter, stag_window, stag_min_iter, 0, radius, watchdog_cycles,
                              int(max_degree), threads, blocks_per_sm, sort, engine)
        # one single-sweep launch outside capture loads the module and sets the
        # kernel's attributes; the captured launch then runs the full options
        warm = RootsOpts(tol, 1, stag_window, stag_min_iter, 0, radius, watchdog_cycles,
                         int(max_degree), threads, blocks_per_sm, sort, engine)
        self._launch(warm)
        t.cuda.synchronize()
        self.graph = t.cuda.CUDAGraph()
        with t.cuda.graph(self.graph):
            self._launch()
        t.cuda.synchronize()

    def _launch(self, opts=None):
        z0 = self.z0
        _call(f"mp_roots_{self.prec}", self.npoly, _ptr(self.coef_off), _ptr(self.coef),
              _ps(self.coef), _ptr(z0), z0.stride(0) if z0 is not None else 0, _ptr(self._r),
              self._r.stride(0), _ptr(self.iters), _ptr(self.status),
              ctypes.byref(opts if opts is not None else self.opts), _ptr(self.ws), self.ws.numel(),
              _stream())

    @property
    def roots(self):
        return self._r[:, :self.total]

    def replay(self):
        self.graph.replay()
        return self.roots, self.iters, self.status


def peak(kind, iters=4096, blocks=None, threads=256):
    """Pipe-peak microbenchmark: returns (lane instructions per second, ms)."""
    L = lib()
    blocks = blocks or L.mp_sm_count() * 8
    ms, ops = ctypes.c_float(), ctypes.c_double()
    _call("mp_peak_run", kind, iters, blocks, threads, ctypes.byref(ms), ctypes.byref(ops),
          _stream())
    return ops.value / (ms.value * 1e-3), ms.value
