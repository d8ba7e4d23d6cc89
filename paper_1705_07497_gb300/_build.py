"""Compiles libct.so (CUDA, sm_103a) in-tree with nvcc.

Each ``csrc/*.cu`` translation unit is compiled in parallel to an object in
``_build/``; the objects are linked into ``_lib/libct.so`` with the CUDA
runtime linked statically.  Nothing here runs a GPU: nvcc cross-compiles.
"""

import concurrent.futures as cf
import fcntl
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libct.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3",
    "-lineinfo",
    "-std=c++17",
    "-Xcompiler",
    "-fPIC,-O2",
    "-I" + INC,
    "-I" + SRC,
]


def nvcc():
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        path = os.path.join(cand, "bin", "nvcc") if cand else ""
        if path and os.path.exists(path):
            return path
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found (set CUDA_HOME)")
    return found


def _sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(os.path.join(INC, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra):
    obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src, __file__] + _headers()):
        tmp = obj + ".tmp%d" % os.getpid()
        cmd = [nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", tmp]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, res.stdout, res.stderr))
        os.replace(tmp, obj)
    return obj


def build(force=False, verbose=False, extra=()):
    """Builds libct.so if any source or header is newer; returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with open(os.path.join(OBJ, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if force:
            for o in glob.glob(os.path.join(OBJ, "*.o")):
                os.remove(o)
        srcs = _sources()
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
            objs = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
        if _stale(LIB, objs):
            tmp = LIB + ".tmp%d" % os.getpid()
            cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode != 0:
                raise RuntimeError("link failed:\n%s%s" % (res.stdout, res.stderr))
            os.replace(tmp, LIB)
        if verbose:
            print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
