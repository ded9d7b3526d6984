"""The location -> (aisle, depth) division by 2L is done on the device as a
multiply-high and a shift whose constants the host computes once per layout
(``geo_set_div`` in the library's internal header; the invariant-divisor method
of Granlund and Montgomery, 1994).  This test compiles that host routine in a
small C++ harness and checks the quotient against plain integer division for
every slots-per-side value the library accepts (L = 1 .. 65,535), at every
quotient boundary near zero and near 2^31 and at seeded random locations: a
wrong rounding of the multiplier or an off-by-one shift fails at the top of the
range, where the error term is largest."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2110_13693_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include "wh_internal.h"

static uint32_t quot(const wh::Geo& g, uint32_t x) {
    return (uint32_t)(((uint64_t)x * g.div_m) >> 32) >> g.div_s;   // __umulhi(x, m) >> s
}

int main() {
    uint64_t state = 0x9E3779B97F4A7C15ull, checked = 0;
    for (int L = 1; L <= 65535; ++L) {
        wh::Geo g{};
        g.L = L;
        wh::geo_set_div(g);
        const uint32_t d = 2u * (uint32_t)L, top = 0x7FFFFFFFu;
        uint32_t xs[40];
        int n = 0;
        for (uint32_t k = 0; k < 8; ++k) {           // the first quotient boundaries
            xs[n++] = k * d;
            xs[n++] = k * d + d - 1;
        }
        const uint32_t kt = top / d;                 // the last boundaries below 2^31
        for (uint32_t k = kt - 4; k <= kt; ++k) {
            xs[n++] = k * d;
            xs[n++] = k * d - 1;
            if ((uint64_t)k * d + d - 1 <= top) xs[n++] = k * d + d - 1;
        }
        xs[n++] = top;
        for (int r = 0; r < 5; ++r) {                // seeded random locations (xorshift64*)
            state ^= state >> 12; state ^= state << 25; state ^= state >> 27;
            xs[n++] = (uint32_t)((state * 2685821657736338717ull) >> 33);
        }
        for (int i = 0; i < n; ++i) {
            if (xs[i] > top) continue;
            ++checked;
            if (quot(g, xs[i]) != xs[i] / d) {
                std::printf("MISMATCH L=%d x=%u got=%u want=%u\n", L, xs[i], quot(g, xs[i]), xs[i] / d);
                return 1;
            }
        }
    }
    std::printf("OK %llu\n", (unsigned long long)checked);
    return 0;
}
"""


def test_location_division_exact(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isfile(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "div.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "div"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("OK")
    assert int(out.stdout.split()[1]) > 65535 * 30
