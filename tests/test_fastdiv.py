"""The kernels' division by invariant divisors (csrc/fastdiv.h, the method of
Granlund and Montgomery, PLDI 1994, Sec. 4) against C's '/': every divisor up
to 4096 with every dividend below 70,000 and the largest ones, then random
divisors and dividends over the whole range the kernels use (0 <= n < 2^31).
The header is compiled for the host with g++; the device build computes the
high product with __umulhi and shares the rest of the code."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2310_17274_gb300", "csrc")

HARNESS = r"""
#include "fastdiv.h"
#include <cstdio>
#include <random>
using namespace crgb;
int main() {
  long long bad = 0;
  for (int d = 1; d <= 4096; ++d) {
    const FastDiv f = make_fastdiv(d);
    for (int n = 0; n < 70000; ++n) bad += fdiv(n, f) != n / d;
    for (int n : {2147483647, 2147483646, 2147483647 - d, 1 << 30}) bad += fdiv(n, f) != n / d;
  }
  std::mt19937_64 g(7);
  for (int it = 0; it < 1000000; ++it) {
    const int d = 1 + (int)(g() % ((it & 1) ? 100000ull : 2147483647ull));
    const int n = (int)(g() % 2147483648ull);
    bad += fdiv(n, make_fastdiv(d)) != n / d;
  }
  // a divisor below 1 is taken as 1
  bad += fdiv(12345, make_fastdiv(0)) != 12345;
  std::printf("%lld\n", bad);
  return bad != 0;
}
"""


def test_fastdiv_matches_integer_division(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    src = tmp_path / "fd.cc"
    src.write_text(HARNESS)
    exe = tmp_path / "fd"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "0", r.stdout + r.stderr
