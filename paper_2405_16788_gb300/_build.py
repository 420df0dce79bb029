"""Compile the CUDA library libdipole.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library next to this file.  Nothing here needs a GPU.  build(checked=True)
makes the checked build, libdipole_checked.so (-DDIPOLE_CHECKED: the traversals
test the indexes they read before using them and report DIPOLE_EBOUNDS); load it
by setting DIPOLE_LIBRARY to its path before importing the binding.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libdipole.so")
OUT_CHECKED = os.path.join(HERE, "libdipole_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["capi.cu", "sort.cu", "tree_build.cu", "refit.cu", "traverse.cu", "traverse_grad.cu"]
HEADERS = ["common.cuh", "kernels.cuh", "tree.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              *ARCH]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdipole")
    return p


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(HERE, "..", "include", "dipole.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libdipole.so (or libdipole_checked.so) if it is missing or older
    than its sources."""
    out = OUT_CHECKED if checked else OUT
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_input():
        return out
    bdir = BUILD_DIR + ("_checked" if checked else "")
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (["-DDIPOLE_CHECKED"] if checked else [])

    def one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", *ARCH, *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=False))
