"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/mpgpu.h declares (no GPU needed: nothing is called)."""

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
