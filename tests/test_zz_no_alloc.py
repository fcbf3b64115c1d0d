"""mp_roots_noalloc_qd: the QD batched root solver for callers that cannot
allocate device memory (a fixed pool that must not grow, a plugin whose
allocator belongs to its host, a real-time loop where an allocation could
stall).  Its workspace (the persistent queue's counter and the degree order) is
a fixed array inside the library, so the caller passes only inputs and outputs.

The test calls it through the C ABI twice in a row, on two different problems
(the second with the descending-degree order, so both parts of the array are
used, and the counter left by the first call must be cleared by the second),
and checks each result bit for bit against mp_roots_qd (the entry point that
takes a caller workspace) -- the tolerance the solver's parity tests use -- and
the first result also against the CPU oracle's solver.  It also checks the size
limits.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_2603_14926_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_POLYS = 1 << 14  # MP_NOALLOC_MAX_POLYS in mpgpu.h
RC_ENOMEM = 3        # MP_ENOMEM


def _fn(mp):
    f = mp.lib().mp_roots_noalloc_qd
    i64, vp = ctypes.c_int64, ctypes.c_void_p
    f.argtypes = [i64, vp, vp, i64, vp, i64, vp, i64, vp, vp, ctypes.POINTER(mp.RootsOpts), vp]
    f.restype = ctypes.c_int
    return f


def _opts(mp, max_degree, max_iter, sort):
    return mp.RootsOpts(0.0, max_iter, 0, 0, 0, 1.1, 0, max_degree, 0, 0, sort, 0)


def _noalloc(mp, off, coef, max_degree, max_iter, sort):
    import torch

    npoly = len(off) - 1
    total = coef.shape[1] - npoly
    doff = torch.from_numpy(off).cuda()
    dc = torch.from_numpy(np.ascontiguousarray(coef)).cuda()
    r = torch.full((8, total), float("nan"), dtype=torch.float64, device="cuda")
    it = torch.full((npoly,), -1, dtype=torch.int32, device="cuda")
    st = torch.full((npoly,), -1, dtype=torch.int32, device="cuda")
    o = _opts(mp, max_degree, max_iter, sort)
    rc = _fn(mp)(npoly, doff.data_ptr(), dc.data_ptr(), dc.stride(0), None, 0, r.data_ptr(), r.stride(0),
                 it.data_ptr(), st.data_ptr(), ctypes.byref(o), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, mp.lib().mp_status_str(rc)
    torch.cuda.synchronize()
    return r.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def _with_workspace(mp, off, coef, max_degree, max_iter, sort):
    import torch

    r, it, st = mp.roots("qd", torch.from_numpy(off).cuda(),
                         torch.from_numpy(np.ascontiguousarray(coef)).cuda(), max_degree,
                         radius=1.1, max_iter=max_iter, sort=sort)
    torch.cuda.synchronize()
    return r.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def _same(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    return a.shape == b.shape and a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_noalloc_matches_workspace_entry_point_twice(mp, oracle):
    # call 1: 24 polynomials of degree 5..60, natural order
    # call 2: a different problem of 300 polynomials, descending-degree order
    for seed, npoly, dmin, dmax, max_iter, sort in ((21, 24, 5, 60, 40, 0), (22, 300, 3, 30, 25, 1)):
        prob = inputs.dk_problem(seed, npoly, dmin, dmax)
        coef = oracle.poly_from_roots("qd", prob)
        got = _noalloc(mp, prob.coef_off, coef, dmax, max_iter, sort)
        want = _with_workspace(mp, prob.coef_off, coef, dmax, max_iter, sort)
        for g, w in zip(got, want):
            assert _same(g, w), seed
        if seed == 21:  # and the first call against the CPU oracle's solver directly
            wr, wit, wst = oracle.roots("qd", prob.coef_off, coef, radius=1.1, max_iter=max_iter)
            assert _same(got[0], wr)
            assert np.array_equal(got[1], wit) and np.array_equal(got[2], wst)


def test_noalloc_rejects_oversize_requests(mp):
    import torch

    f = _fn(mp)
    s = torch.cuda.current_stream().cuda_stream
    npoly = MAX_POLYS + 1
    off = torch.arange(0, 3 * (npoly + 1), 3, dtype=torch.int64, device="cuda")  # degree 2 each
    coef = torch.zeros((4, 3 * npoly), dtype=torch.float64, device="cuda")
    coef[0, 0::3] = -0.25  # x^2 - 1/4
    coef[0, 2::3] = 1.0
    r = torch.zeros((8, 2 * npoly), dtype=torch.float64, device="cuda")
    it = torch.full((npoly,), -7, dtype=torch.int32, device="cuda")
    st = torch.full((npoly,), -7, dtype=torch.int32, device="cuda")
    o = _opts(mp, 2, 5, 0)
    args = (off.data_ptr(), coef.data_ptr(), coef.stride(0), None, 0, r.data_ptr(), r.stride(0),
            it.data_ptr(), st.data_ptr(), ctypes.byref(o), s)
    assert f(npoly, *args) == RC_ENOMEM  # more polynomials than the fixed array orders
    # above the shared-memory degree bound the solver would need per-block slots
    big = _opts(mp, mp.roots_max_degree("qd") + 1, 5, 0)
    assert f(4, *args[:-2], ctypes.byref(big), s) == RC_ENOMEM
    torch.cuda.synchronize()
    assert (it == -7).all() and (st == -7).all()  # nothing was enqueued
    # at the limit it runs
    assert f(MAX_POLYS, *args) == 0
    torch.cuda.synchronize()
    assert (it[:MAX_POLYS] >= 1).all() and (it[MAX_POLYS:] == -7).all()
