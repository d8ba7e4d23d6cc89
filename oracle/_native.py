"""Builds and loads the oracle's C parts (``siddon.c``, ``spmv.c``) with gcc.

Test infrastructure only (see the package docstring).
"""

import ctypes
import fcntl
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_siddon.so")
_SPMV_SRC = os.path.join(_HERE, "spmv.c")
_SPMV_LIB = os.path.join(_OUT_DIR, "liboracle_spmv.so")

_lib = None
_spmv = None


def build(force=False):
    """Compiles ``siddon.c`` into ``_build/liboracle_siddon.so`` (plain gcc)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    with open(os.path.join(_OUT_DIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
        if force or not fresh:
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            )
            os.replace(tmp, _LIB)
        fresh = os.path.exists(_SPMV_LIB) and os.path.getmtime(_SPMV_LIB) >= os.path.getmtime(_SPMV_SRC)
        if force or not fresh:
            tmp = _SPMV_LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                 "-o", tmp, _SPMV_SRC]
            )
            os.replace(tmp, _SPMV_LIB)
    return _LIB


def spmv_lib():
    """The threaded CSR product of ``spmv.c``."""
    global _spmv
    if _spmv is None:
        build()
        L = ctypes.CDLL(_SPMV_LIB)
        L.oracle_csr_matvec.restype = None
        L.oracle_csr_matvec.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        _spmv = L
    return _spmv


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.oracle_siddon_count.restype = ctypes.c_int64
        L.oracle_siddon_count.argtypes = [ctypes.c_int] * 4 + [i64p]
        L.oracle_siddon_fill.restype = ctypes.c_int
        L.oracle_siddon_fill.argtypes = [ctypes.c_int] * 4 + [
            i64p,
            ctypes.POINTER(ctypes.c_int32),
            ctypes.POINTER(ctypes.c_double),
        ]
        L.oracle_directions.restype = None
        L.oracle_directions.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 2
        L.oracle_siddon_rows.restype = ctypes.c_int64
        L.oracle_siddon_rows.argtypes = [ctypes.c_int] * 4 + [ctypes.c_int64, i64p, i64p, i64p,
                                                              ctypes.POINTER(ctypes.c_int32),
                                                              ctypes.POINTER(ctypes.c_double)]
        L.oracle_num_kept.restype = ctypes.c_int
        L.oracle_num_kept.argtypes = [ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib
