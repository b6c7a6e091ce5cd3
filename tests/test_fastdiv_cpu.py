"""The invariant-divisor division of the site-index kernels (csrc/fastdiv.h),
checked on the CPU against the hardware integer division.

The header is plain C++ for a host compiler; this test compiles a small driver
with g++ and compares floor(n / d) for every n below 2^20 and for random and
extreme 32-bit n, over the divisors a lattice can give (X/2, Y, Z up to a few
hundred) and over powers of two and large divisors.
"""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
HDR = ROOT / "paper_2212_06635_gb300" / "csrc" / "fastdiv.h"

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include "fastdiv.h"
using namespace tmk;
static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint32_t rnd() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return (uint32_t)(s >> 16); }
static int check(uint32_t d) {
    const FastDiv f = make_fastdiv(d);
    for (uint32_t n = 0; n < (1u << 20); ++n)
        if (fdiv(n, f) != n / d) { std::printf("FAIL d=%u n=%u\n", d, n); return 1; }
    for (int k = 0; k < 200000; ++k) {
        const uint32_t n = rnd();
        if (fdiv(n, f) != n / d) { std::printf("FAIL d=%u n=%u\n", d, n); return 1; }
    }
    const uint32_t edge[] = {0xffffffffu, 0xfffffffeu, 0x80000000u, 0x7fffffffu, d, d - 1, d + 1, 2 * d - 1};
    for (uint32_t n : edge)
        if (fdiv(n, f) != n / d) { std::printf("FAIL d=%u n=%u\n", d, n); return 1; }
    return 0;
}
int main() {
    int bad = 0;
    for (uint32_t d = 1; d <= 300; ++d) bad |= check(d);
    for (int l = 0; l < 32; ++l) { bad |= check(1u << l); bad |= check((1u << l) + 1); if (l > 1) bad |= check((1u << l) - 1); }
    const uint32_t big[] = {1000003u, 65537u, 0x7fffffffu, 0x80000001u, 0xfffffffeu, 0xffffffffu};
    for (uint32_t d : big) bad |= check(d);
    if (!bad) std::printf("OK\n");
    return bad;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_fastdiv_matches_integer_division(tmp_path):
    src = tmp_path / "fd.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "fd"
    subprocess.run(["g++", "-O2", "-std=c++17", f"-I{HDR.parent}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout
