"""mp_polyeval_backward_noalloc_qd: the QD Horner adjoint for callers that
cannot allocate device memory (a fixed pool that must not grow, a plugin whose
allocator belongs to its host, a real-time loop where an allocation could
stall).  Its scratch is a fixed array inside the library, so the caller passes
only inputs and outputs.

The test calls it through the C ABI twice in a row, on two different problems,
and checks each result bit for bit against mp_polyeval_backward_qd (the entry
point that takes a caller workspace) -- the tolerance the Horner adjoint's
parity tests use -- and the first result also against the CPU oracle's
adjoint.  It also checks the size limit.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_2603_14926_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_POINTS = 1 << 17  # MP_NOALLOC_MAX_POINTS in mpgpu.h


def _fn(mp):
    f = mp.lib().mp_polyeval_backward_noalloc_qd
    i64, vp = ctypes.c_int64, ctypes.c_void_p
    f.argtypes = [i64, vp, vp, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp]
    f.restype = ctypes.c_int
    return f


def _problem(seed, npoly, dmin, dmax, npts):
    rng = np.random.default_rng(seed)
    deg = rng.integers(dmin, dmax + 1, npoly)
    off = np.zeros(npoly + 1, dtype=np.int64)
    np.cumsum(deg + 1, out=off[1:])
    coef = inputs.mp_uniform(seed, int(off[-1]), 4, stream=inputs.STREAM_C)
    x = inputs.mp_uniform(seed + 1, npoly * npts, 4, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(seed + 2, npoly * npts, 4, stream=inputs.STREAM_Y)
    return off, coef, x, dy


def _noalloc(mp, off, coef, npts, x, dy):
    import torch

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    doff, dc, dxs, ddy = t(off), t(coef), t(x), t(dy)
    dcoef = torch.full_like(dc, float("nan"))
    dx = torch.full_like(dxs, float("nan"))
    rc = _fn(mp)(len(off) - 1, doff.data_ptr(), dc.data_ptr(), dc.stride(0), npts, dxs.data_ptr(),
                 dxs.stride(0), ddy.data_ptr(), ddy.stride(0), dcoef.data_ptr(), dcoef.stride(0),
                 dx.data_ptr(), dx.stride(0), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, mp.lib().mp_status_str(rc)
    torch.cuda.synchronize()
    return dcoef.cpu().numpy(), dx.cpu().numpy()


def _with_workspace(mp, off, coef, npts, x, dy):
    import torch

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    dc, dx = mp.polyeval_backward("qd", t(off), t(coef), npts, t(x), t(dy))
    torch.cuda.synchronize()
    return dc.cpu().numpy(), dx.cpu().numpy()


def _same(a, b):
    return a.shape == b.shape and np.array_equal(np.ascontiguousarray(a).view(np.uint64),
                                                 np.ascontiguousarray(b).view(np.uint64))


def test_noalloc_matches_workspace_entry_point_twice(mp, oracle):
    # call 1: 9 polynomials of degree 0..70 at 300 points (three 32-coefficient sweeps)
    # call 2: a different problem that fills the whole scratch (32 x 4096 points)
    for seed, npoly, dmin, dmax, npts in ((11, 9, 0, 70, 300), (12, 32, 20, 40, MAX_POINTS // 32)):
        off, coef, x, dy = _problem(seed, npoly, dmin, dmax, npts)
        got_c, got_x = _noalloc(mp, off, coef, npts, x, dy)
        want_c, want_x = _with_workspace(mp, off, coef, npts, x, dy)
        assert _same(got_c, want_c), seed
        assert _same(got_x, want_x), seed
        if seed == 11:  # and the first call against the CPU oracle's adjoint directly
            ref_c, ref_x = oracle.polyeval_backward("qd", off, coef, npts, x, dy)
            assert _same(got_c, ref_c) and _same(got_x, ref_x)


def test_noalloc_rejects_oversize_requests(mp):
    import torch

    npts = MAX_POINTS // 8 + 1
    off = torch.tensor([0, 3, 6, 9, 12, 15, 18, 21, 24], dtype=torch.int64, device="cuda")
    coef = torch.zeros((4, 24), dtype=torch.float64, device="cuda")
    x = torch.zeros((4, 8 * npts), dtype=torch.float64, device="cuda")
    dcoef = torch.zeros_like(coef)
    dx = torch.zeros_like(x)
    s = torch.cuda.current_stream().cuda_stream
    f = _fn(mp)
    rc = f(8, off.data_ptr(), coef.data_ptr(), 24, npts, x.data_ptr(), x.stride(0), x.data_ptr(),
           x.stride(0), dcoef.data_ptr(), 24, dx.data_ptr(), dx.stride(0), s)
    assert rc == 3  # MP_ENOMEM: 8 * npts points exceed the fixed scratch
    # without dcoef no scratch is used, so the limit does not apply
    rc = f(8, off.data_ptr(), coef.data_ptr(), 24, npts, x.data_ptr(), x.stride(0), x.data_ptr(),
           x.stride(0), None, 0, dx.data_ptr(), dx.stride(0), s)
    assert rc == 0
    torch.cuda.synchronize()
