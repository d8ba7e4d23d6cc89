"""CPU checks of the C ABI: the library builds, loads, exports every symbol
that include/ct.h declares, and rejects invalid arguments before touching a
GPU."""

import ctypes
import os
import re

import pytest

from paper_1705_07497_gb300 import _build, ct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ct.lib()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "ct.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ct_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_symbols():
    assert _declared_symbols() == sorted(ct.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(ct.LIB_PATH)
    for name in _declared_symbols():
        assert hasattr(raw, name), name


def test_status_strings(lib):
    assert ct.status_string(ct.CT_OK) == "ok"
    assert "breakdown" in ct.status_string(ct.CT_ERR_BREAKDOWN).lower()
    assert ct.status_string(12345) == "unknown status"


@pytest.mark.parametrize(
    "geom",
    [(0, 90, 3, 91), (64, 0, 3, 91), (64, 90, 0, 91), (64, 90, 3, 0), (-1, 1, 1, 1), (50000, 4, 1, 8)],
)
def test_invalid_geometry_is_rejected_without_a_gpu(lib, geom):
    g = ct.Geometry(*geom)
    h = ctypes.c_void_p()
    rc = lib.ct_build_matrix(ctypes.byref(g), 0, ctypes.byref(h))
    assert rc == ct.CT_ERR_ARG
    assert h.value is None
    assert lib.ct_last_error().decode() != ""


def test_null_and_flag_errors(lib):
    h = ctypes.c_void_p()
    assert lib.ct_build_matrix(None, 0, ctypes.byref(h)) == ct.CT_ERR_ARG
    g = ct.Geometry(8, 8, 1, 12)
    assert lib.ct_build_matrix(ctypes.byref(g), 0, None) == ct.CT_ERR_ARG
    assert lib.ct_build_matrix(ctypes.byref(g), 0x100, ctypes.byref(h)) == ct.CT_ERR_ARG
    assert lib.ct_build_matrix(ctypes.byref(g), ct.CT_KEEP_FP32_COPY, ctypes.byref(h)) == ct.CT_ERR_ARG
    assert lib.ct_matrix_info(None, None, None, None) == ct.CT_ERR_ARG
    lib.ct_destroy_matrix(None)  # no-op


def test_binding_refuses_wrong_dtypes(lib):
    import numpy as np

    with pytest.raises(TypeError):
        ct._vec(np.zeros(4, dtype=np.float64))
    with pytest.raises(TypeError):
        ct._vec([1.0, 2.0])


def test_ragged_argument_errors(lib):
    p = ct.SbParams(1.0, 1.0, 3, 3, 0.0, 0, 0, 0)
    arr = (ctypes.c_void_p * 1)()
    assert lib.ct_split_bregman_ragged(0, arr, arr, arr, ctypes.byref(p), None, None) == ct.CT_ERR_ARG
    assert lib.ct_split_bregman_ragged(1, None, arr, arr, ctypes.byref(p), None, None) == ct.CT_ERR_ARG
    assert lib.ct_split_bregman_ragged(1, arr, arr, arr, None, None, None) == ct.CT_ERR_ARG
    bad = ct.SbParams(1.0, 0.0, 3, 3, 0.0, 0, 0, 0)  # lambda must be positive
    assert lib.ct_split_bregman_ragged(1, arr, arr, arr, ctypes.byref(bad), None, None) == ct.CT_ERR_ARG
    with pytest.raises(ValueError):
        ct.ct_split_bregman_ragged([None], p, [], [])


def test_spmm_unroll_argument_errors(lib):
    v = ctypes.c_int32()
    assert lib.ct_set_spmm_unroll(None, 4, 4) == ct.CT_ERR_ARG
    assert lib.ct_get_spmm_unroll(None, 4, ctypes.byref(v)) == ct.CT_ERR_ARG


def test_chambolle_pock_argument_errors(lib):
    p = ct.CpParams(1.0, 0.3, 0.3, 1.0, 3, 3)
    assert lib.ct_chambolle_pock(None, ctypes.byref(p), None, None, 1, None, None) == ct.CT_ERR_ARG


@pytest.mark.parametrize(
    "geom,params,code",
    [
        ((48, 40, 1, 68), (6, 0.0, 0), ct.CT_ERR_UNSUPPORTED),  # N not a power of two
        ((8, 40, 1, 12), (2, 0.0, 0), ct.CT_ERR_UNSUPPORTED),   # N below 16
        ((32, 40, 1, 46), (0, 0.0, 0), ct.CT_ERR_ARG),          # m_sp below 1
        ((32, 40, 1, 46), (13, 0.0, 0), ct.CT_ERR_ARG),         # m_sp above 12
        ((32, 40, 1, 46), (6, -1.0, 0), ct.CT_ERR_ARG),         # negative tau
        ((32, 40, 1, 46), (6, 0.0, 7), ct.CT_ERR_ARG),          # unknown mode
        ((32, 0, 1, 46), (6, 0.0, 0), ct.CT_ERR_ARG),           # bad geometry
    ],
)
def test_fourier_argument_errors_without_a_gpu(lib, geom, params, code):
    """ct_build_fourier validates sizes and parameters before any CUDA call."""
    g = ct.Geometry(*geom)
    p = ct.FourierParams(*params)
    h = ctypes.c_void_p()
    assert lib.ct_build_fourier(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)) == code
    assert h.value is None
    assert lib.ct_build_fourier(ctypes.byref(g), None, ctypes.byref(h)) == ct.CT_ERR_ARG
    assert lib.ct_fourier_forward(None, None, None, None) == ct.CT_ERR_ARG


_STRUCTS = [
    ("ct_geometry", "Geometry"),
    ("ct_cg_params", "CgParams"),
    ("ct_cg_stats", "CgStats"),
    ("ct_sb_params", "SbParams"),
    ("ct_sb_stats", "SbStats"),
    ("ct_cp_params", "CpParams"),
    ("ct_fourier_params", "FourierParams"),
    ("ct_tuning", "Tuning"),
]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the struct of the same name in include/ct.h."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ct.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS:
        lines.append('    printf("%s size %%zu\\n", sizeof(%s));' % (pyname, cname))
        for fname, _ in getattr(ct, pyname)._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (pyname, fname, cname, cf))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        pyname, what, value = line.split()
        cls = getattr(ct, pyname)
        want = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert int(value) == want, (pyname, what, int(value), want)
        seen += 1
    assert seen == sum(1 + len(getattr(ct, p)._fields_) for _, p in _STRUCTS)


def test_binding_argument_counts_match_the_prototypes(lib):
    """Each function the binding declares takes as many arguments as its
    prototype in include/ct.h."""
    text = open(os.path.join(ROOT, "include", "ct.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = dict(re.findall(r"\b(ct_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text))
    checked = 0
    for name, params in protos.items():
        argtypes = getattr(lib, name).argtypes
        if argtypes is None:
            continue
        n = 0 if params.strip() in ("", "void") else params.count(",") + 1
        assert len(argtypes) == n, (name, len(argtypes), n)
        checked += 1
    assert checked >= len(protos) - 1
