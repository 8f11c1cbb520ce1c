"""The fixed-point coordinate of the float32 path, floor(w 2^32 / L) mod 2^32,
computed with integer arithmetic (device_common.cuh): its host instantiation,
compiled with nvcc, against the exact floor from a 128-bit product of the two
significands on millions of positions, box edges of the workloads and edge cases
(0, the largest double below L, tiny w)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_07693_gb300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "device_common.cuh"

// exact floor(w * 2^32 / L) through the exact rational product of the doubles
// w = mw 2^ew and 2^32 / L = f 2^x (f 53-bit), with __int128 arithmetic
static unsigned long long exact(double w, double inv_unit) {
  if (w == 0.0) return 0;
  int ew, ei;
  const double fw = std::frexp(w, &ew), fi = std::frexp(inv_unit, &ei);
  const unsigned __int128 mw = (unsigned __int128)std::ldexp(fw, 53), mi = (unsigned __int128)std::ldexp(fi, 53);
  const int sh = 106 - ew - ei;          // w inv_unit = mw mi 2^(ew + ei - 106)
  const unsigned __int128 p = mw * mi;
  if (sh >= 128) return 0;
  return (unsigned long long)((sh >= 0) ? (p >> sh) : (p << -sh));
}

int main() {
  std::mt19937_64 rng(7);
  long bad = 0, n = 0;
  for (double L : {28.7, 143.5, 68.88, 459.2, 318.86, 573.999, 16.5, 2000.0}) {
    const double inv = 4294967296.0 / L;
    int x = 0;
    const double f = std::frexp(inv, &x);
    const unsigned long long M = (unsigned long long)std::ldexp(f, 64);
    const int s = x - 64;
    std::uniform_real_distribution<double> U(0.0, L);
    for (int k = 0; k < 1000000; ++k) {
      double w = U(rng);
      if (k == 0) w = 0.0;
      if (k == 1) w = std::nextafter(L, 0.0);
      if (k == 2) w = 1e-300;
      if (k == 3) w = 1e-9;
      if (k == 4) w = 0.5 * L;
      const unsigned got = apip::fixed_coord(w, M, s);
      const unsigned want = (unsigned)(exact(w, inv) & 0xffffffffull);
      ++n;
      if (got != want) { if (++bad < 5) std::printf("L=%.17g w=%.17g got=%u want=%u\n", L, w, got, want); }
    }
  }
  std::printf("checked %ld mismatches %ld\n", n, bad);
  return bad != 0;
}
"""


def test_integer_fixed_coordinate_is_the_exact_floor(tmp_path):
    if not os.path.exists(NVCC) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    src = tmp_path / "fixed.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fixed"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "mismatches 0" in r.stdout
