"""Host check of the integer widening FP32 -> FP64 (csrc/fp_widen.h) that the operator
passes use for the precision form's FP32 vectors: it must equal the IEEE conversion bit for
bit on every class (normal, subnormal, signed zero, infinity) and give a NaN for a NaN.
The header is plain C++ outside nvcc; it is compiled here with g++ and run over every
exponent with a spread of fractions, the extreme fractions and every subnormal position."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_04384_gb300", "csrc")

PROG = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include "fp_widen.h"
int main() {
  long long bad = 0, n = 0;
  auto check = [&](unsigned u) {
    float f; std::memcpy(&f, &u, 4);
    double a = iga::widen_f32(f), b = (double)f;
    ++n;
    if (std::isnan(f)) { if (!std::isnan(a) || std::signbit(a) != std::signbit(f)) ++bad; return; }
    if (std::memcmp(&a, &b, 8) != 0) ++bad;
  };
  for (unsigned s = 0; s < 2; ++s)
    for (unsigned e = 0; e < 256; ++e) {
      for (unsigned f = 0; f < (1u << 23); f += 997) check((s << 31) | (e << 23) | f);
      for (unsigned f : {0u, 1u, 2u, 3u, 0x7fffffu, 0x400000u, 0x3fffffu})
        check((s << 31) | (e << 23) | f);
      for (int t = 0; t < 23; ++t) check((s << 31) | (e << 23) | (1u << t));
    }
  std::printf("%lld %lld\n", n, bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_widening_is_exact(tmp_path):
    src = tmp_path / "w.cpp"
    src.write_text(PROG)
    exe = tmp_path / "w"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    n, bad = map(int, r.stdout.split())
    assert n > 4_000_000 and bad == 0, r.stdout
