"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/mpgpu.h declares; host-only paths (workspace sizes, argument errors)
answer without a GPU."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpgpu.h")


def declared_functions():
    """Function names declared by the header after macro expansion."""
    out = subprocess.run(["gcc", "-E", "-P", "-x", "c", HEADER], capture_output=True, text=True,
                         check=True).stdout
    return sorted(set(re.findall(r"\b(mp_[A-Za-z0-9_]+)\s*\(", out)))


def test_header_is_plain_c():
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c", HEADER],
                   check=True)


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc to build")
def test_library_exports_every_declared_symbol():
    from paper_2603_14926_gb300 import buildlib as build

    lib = build.build()
    L = ctypes.CDLL(lib)
    names = declared_functions()
    assert len(names) > 80
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2603_14926_gb300 as mpg

    monkeypatch.setattr(mpg, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(mpg, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        mpg.load()


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc to build")
def test_strassen_host_side_contract():
    """The Strassen entry point's host-side contract, checked with no GPU (neither
    call reaches CUDA): the workspace is three 256-byte-aligned buffers per
    recursion level (ceil halves until a size drops below the cutoff), and bad
    arguments are rejected before anything is enqueued."""
    from paper_2603_14926_gb300 import buildlib as build

    L = ctypes.CDLL(build.build())
    i64 = ctypes.c_int64
    ws = L.mp_gemm_strassen_workspace_qd
    ws.restype, ws.argtypes = ctypes.c_size_t, [i64, i64, i64, i64]

    def levels(m, n, k, cut, elem=32):
        total = 0
        while m >= cut and n >= cut and k >= cut:
            hm, hn, hk = (m + 1) // 2, (n + 1) // 2, (k + 1) // 2
            total += sum(-(-elem * x // 256) * 256 for x in (hm * hk, hk * hn, hm * hn))
            m, n, k = hm, hn, hk
        return total

    for m, n, k, cut in ((64, 64, 64, 32), (65, 65, 65, 32), (100, 77, 90, 16), (8, 8, 8, 2), (31, 31, 31, 32),
                         (4096, 4096, 4096, 2048), (1, 5, 7, 2)):
        assert ws(m, n, k, cut) == levels(m, n, k, cut), (m, n, k, cut)
    assert ws(40, 40, 40, 41) == 0 and ws(-1, 4, 4, 2) == 0
    f = L.mp_gemm_strassen_qd
    f.restype = ctypes.c_int
    f.argtypes = [i64, i64, i64, ctypes.c_void_p, i64, i64, ctypes.c_void_p, i64, i64, ctypes.c_void_p, i64, i64,
                  i64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    MP_OK, MP_EINVAL = 0, 1
    assert f(4, 4, 4, None, 4, 16, None, 4, 16, None, 4, 16, 1, None, 0, None) == MP_EINVAL   # cutoff < 2
    assert f(-1, 4, 4, None, 4, 16, None, 4, 16, None, 4, 16, 2, None, 0, None) == MP_EINVAL  # m < 0
    assert f(4, 4, 4, None, 4, 16, None, 4, 16, None, 4, 16, 2, None, 0, None) == MP_EINVAL   # no C
    assert f(0, 4, 4, None, 4, 16, None, 4, 16, None, 4, 16, 2, None, 0, None) == MP_OK       # empty C
