"""The magic-number division of csrc/fastdiv.cuh (Granlund-Montgomery), built
as host code, against exact integer division for every divisor up to 4096,
large divisors, and numerators at both ends of [0, 2^31)."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <cstdio>
#include <cstdint>
#include "fastdiv.cuh"
int main() {
    using namespace mc;
    long long bad = 0, checked = 0;
    auto check = [&](uint32_t d) {
        const FastDiv f = make_fastdiv(d);
        auto one = [&](uint32_t n) {
            uint32_t q, r;
            fast_divmod(n, f, q, r);
            if (q != n / d || r != n % d) { if (bad < 5) printf("d=%u n=%u q=%u\n", d, n, q); ++bad; }
            ++checked;
        };
        for (uint32_t n = 0; n < 70000; ++n) one(n);
        for (uint32_t n = 0x7FFFFFFFu - 70000; n < 0x7FFFFFFFu; ++n) one(n);
        one(0x7FFFFFFFu);
        uint64_t x = 0x9E3779B97F4A7C15ull * d;
        for (int i = 0; i < 20000; ++i) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; one((uint32_t)(x & 0x7FFFFFFFu)); }
        for (uint32_t k = 1; k < 64; ++k) { uint64_t n = (uint64_t)d * k * 997; if (n < 0x80000000ull) { one((uint32_t)n); one((uint32_t)n - 1); } }
    };
    for (uint32_t d = 1; d <= 4096; ++d) check(d);
    const uint32_t big[] = {65535u, 65536u, 65537u, 1000003u, 16777215u, 16777216u, 0x40000001u, 0x7FFFFFFFu, 0x80000000u};
    for (uint32_t d : big) check(d);
    printf("%lld %lld\n", checked, bad);
    return bad != 0;
}
"""


def test_fast_division_is_exact():
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.cpp")
        open(c, "w").write(SRC)
        exe = os.path.join(d, "t")
        subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_0903_3053_gb300", "csrc"), c, "-o",
                        exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout
        checked, bad = map(int, r.stdout.split()[-2:])
        assert bad == 0 and checked > 4096 * 160000
