"""Build libmpgpu.so in-tree for sm_103a (nvcc, one -gencode, parallel units).

    python -m paper_2603_14926_gb300.buildlib [--force] [--jobs N]

Objects go to paper_2603_14926_gb300/lib/obj, the library to
paper_2603_14926_gb300/lib/libmpgpu.so (both git-ignored).  The CUDA runtime
is linked statically, so the library needs only the driver at run time.
"""

from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libmpgpu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fno-fast-math", f"-I{INCLUDE}", f"-I{CSRC}"]
GEMM_PRECS = ("dd", "ddc", "td", "qd", "tdc", "qdc", "ds", "tf", "qf")


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmpgpu.so")
    return exe


def units():
    """(object name, source, extra flags) for every translation unit."""
    out = [("k_blas1.o", "k_blas1.cu", [])]
    for p in GEMM_PRECS:
        out.append((f"k_gemm_{p}.o", "k_gemm.cu", [f"-DMPGPU_GEMM_PREC={p}"]))
    for extra in ("k_poly.cu", "k_roots.cu", "k_cgemm.cu", "k_strassen.cu"):
        if os.path.exists(os.path.join(CSRC, extra)):
            out.append((extra.replace(".cu", ".o"), extra, []))
    return out


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "mpgpu.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    newest = _deps_mtime()
    exe = nvcc()
    todo = []
    for obj, src, extra in units():
        o = os.path.join(OBJDIR, obj)
        if force or not os.path.exists(o) or os.path.getmtime(o) < newest:
            todo.append((o, [exe, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", o]))

    def run(item):
        o, cmd = item
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(o)}:\n{r.stdout}\n{r.stderr}")
        return o

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(run, todo))
    objs = [os.path.join(OBJDIR, obj) for obj, _, _ in units()]
    if force or todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, objs)):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args(argv)
    print(build(a.force, a.jobs, a.verbose))


if __name__ == "__main__":
    sys.exit(main())
