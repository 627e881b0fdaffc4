"""The kernels' in-register DFT butterflies (radix 2, 3, 4, 5, 7, 8, 16, 32,
both signs),
compiled for the host from the same header the sm_103a kernels include and
checked against the direct DFT in double: no GPU needed.  A wrong rotation
constant or a dropped term in a butterfly shows up here before any kernel
runs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1407_6915_gb300", "csrc")

HARNESS = r'''
#include "engine.cuh"
#include <cmath>
#include <cstdio>
using namespace fftseg;
template <int R, int S> double err() {
    float2 v[32]; double xr[32], xi[32];
    unsigned st = 12345u + R * 7u + (S > 0);
    for (int i = 0; i < R; ++i) {
        st = st * 1103515245u + 12345u; xr[i] = (st >> 8) / 16777216.0 - 0.5;
        st = st * 1103515245u + 12345u; xi[i] = (st >> 8) / 16777216.0 - 0.5;
        v[i] = make_float2((float)xr[i], (float)xi[i]);
        xr[i] = v[i].x; xi[i] = v[i].y;
    }
    dft<R, S>(v);
    double num = 0, den = 0;
    for (int k = 0; k < R; ++k) {
        double ar = 0, ai = 0;
        for (int j = 0; j < R; ++j) {
            const double ph = S * 2.0 * M_PI * (double)((j * k) % R) / R;
            ar += xr[j] * cos(ph) - xi[j] * sin(ph);
            ai += xr[j] * sin(ph) + xi[j] * cos(ph);
        }
        num += (v[k].x - ar) * (v[k].x - ar) + (v[k].y - ai) * (v[k].y - ai);
        den += ar * ar + ai * ai;
    }
    return sqrt(num / den);
}
int main() {
    printf("%d %.3e\n", 2, err<2, -1> () > err<2, 1>() ? err<2, -1>() : err<2, 1>());
    printf("%d %.3e\n", 4, err<4, -1> () > err<4, 1>() ? err<4, -1>() : err<4, 1>());
    printf("%d %.3e\n", 8, err<8, -1> () > err<8, 1>() ? err<8, -1>() : err<8, 1>());
    printf("%d %.3e\n", 16, err<16, -1>() > err<16, 1>() ? err<16, -1>() : err<16, 1>());
    printf("%d %.3e\n", 32, err<32, -1>() > err<32, 1>() ? err<32, -1>() : err<32, 1>());
    printf("%d %.3e\n", 3, err<3, -1> () > err<3, 1>() ? err<3, -1>() : err<3, 1>());
    printf("%d %.3e\n", 5, err<5, -1> () > err<5, 1>() ? err<5, -1>() : err<5, 1>());
    printf("%d %.3e\n", 7, err<7, -1> () > err<7, 1>() ? err<7, -1>() : err<7, 1>());
    return 0;
}
'''


def test_register_butterflies_match_the_direct_dft(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "bfly.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "bfly"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    errs = {int(a): float(b) for a, b in (line.split() for line in out if line.strip())}
    assert set(errs) == {2, 3, 4, 5, 7, 8, 16, 32}
    for r, e in errs.items():
        # float32 butterflies: a few units in the last place of the largest output
        assert e < 4e-7 * max(1, r.bit_length()), (r, e)
