"""Build of the CUDA library (libsphmesh.so) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library next to this file (``_lib/libsphmesh.so``). No torch extension
machinery: the library exports a plain C ABI (include/sphmesh.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libsphmesh.so")
SOURCES = ["sph_api.cu", "sph_cells.cu", "sph_colors.cu", "sph_init.cu", "sph_noalloc.cu", "sph_step_2d.cu",
           "sph_step_3d.cu", "sph_adjoint_2d.cu", "sph_adjoint_3d.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsphmesh")
    return p


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                   "-I" + os.path.join(ROOT, "include"), "-I" + CSRC] + list(extra)


def _stale(objs_src):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for f in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    if os.path.getmtime(os.path.join(ROOT, "include", "sphmesh.h")) > t:
        return True
    return False


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(os.path.join(OUT_DIR, "obj"), exist_ok=True)
    if not force and not _stale(SOURCES):
        return LIB
    cc = nvcc()

    def one(src):
        obj = os.path.join(OUT_DIR, "obj", src.replace(".cu", ".o"))
        cmd = [cc] + flags(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
