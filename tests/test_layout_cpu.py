"""The library's tiled image layout (csrc/layout.cuh), compiled as plain C++
on the host: internal index and pixel coordinates are inverse maps, the
pixels fill the padded range exactly once, every 16 x 16 tile is one run of
256 indices and every 4 x 4 micro-tile one run of 16 (one 128-byte line of
double-float values)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#define __host__
#define __device__
#include <cstdio>
#include <vector>
#include "layout.cuh"
using namespace ct;
int main() {
    const int sizes[] = {1, 15, 16, 17, 33, 64, 100};
    for (int n : sizes) {
        const int tn = tiles_per_side(n);
        const int64_t np = padded_pixels(n);
        if (np != (int64_t)tn * tn * 256) { std::printf("FAIL padded %d\n", n); return 1; }
        std::vector<int> hits((size_t)np, 0);
        for (int i = 0; i < tn * 16; ++i)
            for (int j = 0; j < tn * 16; ++j) {
                const int64_t t = tiled_index(i, j, tn);
                if (t < 0 || t >= np) { std::printf("FAIL range %d %d %d\n", n, i, j); return 1; }
                ++hits[(size_t)t];
                int a, b;
                tiled_coords(t, tn, a, b);
                if (a != i || b != j) { std::printf("FAIL inverse %d %d %d\n", n, i, j); return 1; }
                if ((t >> 8) != (int64_t)(i / 16) * tn + j / 16) { std::printf("FAIL tile %d\n", n); return 1; }
                const int64_t micro0 = tiled_index(i & ~3, j & ~3, tn);
                if ((t & ~(int64_t)15) != micro0 || (micro0 & 15) != 0) { std::printf("FAIL micro %d\n", n); return 1; }
            }
        for (int64_t t = 0; t < np; ++t)
            if (hits[(size_t)t] != 1) { std::printf("FAIL bijection %d\n", n); return 1; }
    }
    std::printf("ok\n");
    return 0;
}
"""


def test_tiled_layout_is_a_bijection_with_tile_and_line_runs(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "layout_check.cpp"
    src.write_text(SRC)
    exe = tmp_path / "layout_check"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1705_07497_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
