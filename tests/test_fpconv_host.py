"""The exact integer binary32 <-> binary64 conversions of fpconv.cuh, compiled for the host
with the system C++ compiler, against the host's IEEE conversions (round to nearest even):
every binary32 exponent and sign with a sweep of fractions (all edge fractions included)
widened, and binary64 values across the binary32 subnormal / normal / overflow range with
forced round-to-nearest-even ties rounded.  The device build of the same functions is
checked against the GPU's conversion instructions by kpsb_conversion_check."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2410_00233_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include "fpconv.cuh"
using namespace kpsb;
static unsigned long long bits64(double d) { unsigned long long b; std::memcpy(&b, &d, 8); return b; }
static unsigned bits32(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static double from64(unsigned long long b) { double d; std::memcpy(&d, &b, 8); return d; }
static float from32(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static unsigned long long mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
int main() {
  unsigned long long bad = 0, n = 0;
  static const unsigned edge[6] = {0u, 1u, 2u, 0x7fffffu, 0x400000u, 0x3fffffu};
  // widening: every sign and exponent, fractions 0, 1, 2, the top values and a stride
  for (unsigned se = 0; se < 512; ++se)
    for (unsigned k = 0; k < 8192 + 6; ++k) {
      const unsigned m = k < 8192 ? (k * 1021u) & 0x7fffffu : edge[k - 8192];
      const float f = from32((se << 23) | m);
      const double a = f2d_bits(f), b = (double)f;
      bad += !(bits64(a) == bits64(b) || (std::isnan(a) && std::isnan(b)));
      ++n;
    }
  // rounding: binary64 values around and inside the binary32 range, ties forced
  for (unsigned long long i = 0; i < (1ull << 22); ++i) {
    const unsigned long long h = mix(i + 1), h2 = mix(h);
    unsigned long long ex;
    switch (h2 & 15u) {
      case 0: ex = 0; break;
      case 1: ex = 0x7ff; break;
      case 2: ex = (h2 >> 8) & 0x7ff; break;
      default: ex = 896 - 30 + ((h2 >> 8) % 300); break;
    }
    unsigned long long fr = h & 0xfffffffffffffull;
    switch ((h2 >> 4) & 3u) {
      case 0: fr = (fr & ~0x1fffffffull) | 0x10000000ull; break;
      case 1: fr = (fr & ~0x1fffffffull) | 0x0fffffffull; break;
      case 2: fr = (fr & ~0x1fffffffull) | 0x10000001ull; break;
      default: break;
    }
    if (ex == 0x7ff && ((h2 >> 6) & 1u)) fr = 0;
    const double d = from64((h & 0x8000000000000000ull) | (ex << 52) | fr);
    const float a = d2f_rn_bits(d), b = (float)d;
    bad += !(bits32(a) == bits32(b) || (std::isnan(a) && std::isnan(b)));
    ++n;
  }
  std::printf("checked %llu mismatches %llu\n", n, bad);
  return bad != 0;
}
"""


def _cuda_include():
    for root in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if root and os.path.exists(os.path.join(root, "include", "cuda_runtime.h")):
            return os.path.join(root, "include")
    nv = shutil.which("nvcc")
    if nv:
        inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_integer_conversions_match_host_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    src = tmp_path / "fpconv_check.cpp"
    exe = tmp_path / "fpconv_check"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
