"""Host check of the integer-operation FP64 conversions (csrc/fp_bits.cuh)
that the data preparation and the one-pass start use instead of the
conversion instructions: widen_f32 must equal the IEEE 754 binary32 ->
binary64 conversion on every one of the 2^32 inputs, narrow_f64 the
round-to-nearest-even binary64 -> binary32 conversion on random bit
patterns, on doubles across the float exponent range with exact ties, near
ties and carries into the exponent, and at the range ends, and finite_bits
must equal isfinite.  The functions are host-and-device code; this test
builds a host program around them with nvcc (no GPU needed).  The GPU side
is pinned bit for bit through a one-row Gram in tests/test_gpu_parity.py."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_09382_gb300", "csrc")

PROGRAM = r"""
#include "fp_bits.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
using concord::widen_f32; using concord::narrow_f64; using concord::finite_bits;
static bool same_f(float a, float b) {
  if (std::isnan(a) || std::isnan(b)) return std::isnan(a) && std::isnan(b);
  return std::memcmp(&a, &b, 4) == 0;
}
static bool same_d(double a, double b) {
  if (std::isnan(a) || std::isnan(b)) return std::isnan(a) && std::isnan(b);
  return std::memcmp(&a, &b, 8) == 0;
}
int main() {
  unsigned long long bad = 0;
  for (unsigned long long x = 0; x <= 0xffffffffull; ++x) {
    const unsigned u = (unsigned)x;
    float f;
    std::memcpy(&f, &u, 4);
    if (!same_d(widen_f32(f), (double)f)) ++bad;
  }
  if (bad) { printf("widen %llu\n", bad); return 1; }
  std::mt19937_64 g(7);
  auto check = [&](unsigned long long u) {
    double d;
    std::memcpy(&d, &u, 8);
    if (!same_f(narrow_f64(d), (float)d)) ++bad;
    if (finite_bits(d) != (bool)std::isfinite(d)) ++bad;
  };
  for (int i = 0; i < 20000000; ++i) check(g());
  for (int i = 0; i < 20000000; ++i) {
    unsigned long long u = g();
    const unsigned long long e = 880 + g() % 290;  // the float exponent range and past it
    u = (u & 0x800fffffffffffffull) | (e << 52);
    switch (g() % 4) {
      case 1: u = (u & ~0x1fffffffull) | 0x10000000ull; break;                 // exact tie
      case 2: u = (u & ~0x1fffffffull) | (0x10000000ull + g() % 3 - 1); break;  // near tie
      case 3: u = (u & ~0x1fffffffull) | 0x1fffffffull; break;                 // carry
      default: break;
    }
    check(u);
  }
  const double ends[] = {3.4028234663852886e38, 3.4028235677973366e38, 1.1754943508222875e-38,
                         1.1754942106924411e-38, 0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN};
  for (double d : ends)
    for (double v : {d, std::nextafter(d, 0.0), std::nextafter(d, 1e300), -d}) {
      unsigned long long u;
      std::memcpy(&u, &v, 8);
      check(u);
    }
  if (bad) { printf("narrow / finite %llu\n", bad); return 1; }
  printf("ok\n");
  return 0;
}
"""


def test_integer_fp64_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "fpbits.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fpbits"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                        "-I" + CSRC, "-o", str(exe), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
