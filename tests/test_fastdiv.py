"""Host logic: the invariant-divisor division of cell indices (Granlund & Montgomery,
Theorem 4.2) equals integer division for every grid extent the library accepts, checked by a
small C++ program built with the host compiler."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cstdint>
#include "rhi_fastdiv.h"
using namespace rhi;
static uint64_t state = 88172645463325252ULL;
static uint32_t next31() { state ^= state << 13; state ^= state >> 7; state ^= state << 17;
                           return (uint32_t)(state >> 33); }
int main() {
    long long bad = 0, checked = 0;
    unsigned ds[] = {1, 2, 3, 5, 7, 9, 10, 11, 13, 16, 24, 31, 32, 33, 63, 64, 65, 100, 127, 128,
                     129, 255, 256, 257, 1000, 1023, 1024, 1025, 4096, 65535, 65536, 65537,
                     16384, 16129, 66049, 1u << 20, (1u << 20) + 1, 1u << 30, (1u << 31) - 1,
                     1u << 31};
    for (unsigned d : ds) {
        FastDiv f = make_fastdiv(d);
        for (int t = 0; t < 200000; ++t) {
            uint32_t n = next31();
            if (t < 64) n = (uint32_t)(((1ULL << 31) - 1) - t);      // the top of the range
            if (t >= 64 && t < 128) n = (uint32_t)(t - 64);
            if (t >= 128 && t < 192) n = (uint32_t)((unsigned long long)d * (t - 128) - 1 + (t == 128));
            if (n >= (1u << 31)) continue;
            ++checked;
            if (fdiv(n, f) != n / d) { if (bad < 5) printf("d=%u n=%u got %u\n", d, n, fdiv(n, f)); ++bad; }
        }
    }
    for (unsigned d = 1; d <= 4096; ++d) {                          // every small extent
        FastDiv f = make_fastdiv(d);
        for (int t = 0; t < 500; ++t) {
            uint32_t n = next31();
            ++checked;
            if (fdiv(n, f) != n / d) ++bad;
        }
    }
    printf("checked %lld bad %lld\n", checked, bad);
    return bad != 0;
}
'''


def test_fastdiv_equals_integer_division(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "fd.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fd"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_0901_1110_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "bad 0" in out.stdout
