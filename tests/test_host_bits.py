"""Doubles assembled from bit patterns with integer operations
(paper_2104_10231_gb300/csrc/fbits.h: the per-atom output kernels use them in
place of the FP64-rate conversion instructions) against the host's own
round-to-nearest-even conversions: 64-bit unsigned integers near every power
of two, exact ties, the largest values and random ones; floats of every
exponent, signed zeros, subnormals, infinities and NaN."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2104_10231_gb300", "csrc")

DRIVER = r"""
#include "fbits.h"
#include <cmath>
#include <cstdio>
#include <random>
using relres::bits_of_double;
static long bad_u = 0, bad_f = 0, n_u = 0, n_f = 0;
static void check_u(uint64_t u) {
  ++n_u;
  if (bits_of_double(relres::double_of_u64(u)) != bits_of_double(static_cast<double>(u))) {
    if (bad_u < 5) std::printf("u64 %llu\n", static_cast<unsigned long long>(u));
    ++bad_u;
  }
}
static void check_f(uint32_t b) {
  float f;
  std::memcpy(&f, &b, sizeof f);
  ++n_f;
  const double a = relres::double_of_float(f), r = static_cast<double>(f);
  const bool same = std::isnan(r) ? std::isnan(a) : bits_of_double(a) == bits_of_double(r);
  if (!same) {
    if (bad_f < 5) std::printf("float bits %08x\n", b);
    ++bad_f;
  }
}
int main() {
  std::mt19937_64 rng(2104);
  for (int s = 0; s < 64; ++s)
    for (long long d = -1100; d <= 1100; ++d) check_u((1ull << s) + static_cast<uint64_t>(d));
  for (int k = 0; k < 200000; ++k) {
    const int lz = static_cast<int>(rng() % 11);
    const uint64_t top = (rng() | (1ull << 63)) >> lz;  // leading one at bit 63 - lz
    const uint64_t rest = 0x400ull >> lz;               // exactly half of the rounded-away part
    const uint64_t keep = ~((0x800ull >> lz) - 1ull);
    check_u((top & keep) | rest);                          // a tie
    check_u((top & keep) | (rest ? rest - 1ull : 0ull));   // just below
    check_u((top & keep) | (rest + 1ull));                 // just above
  }
  for (int k = 0; k < 3000000; ++k) check_u(rng() >> (rng() % 64));
  check_u(~0ull);
  check_u(~0ull - 1ull);
  for (uint32_t e = 0; e < 256; ++e)
    for (int k = 0; k < 4000; ++k) {
      const uint32_t sign = static_cast<uint32_t>(rng() & 1u) << 31;
      const uint32_t frac = k < 2 ? static_cast<uint32_t>(k) : static_cast<uint32_t>(rng() & 0x7fffffu);
      check_f(sign | (e << 23) | frac);
    }
  std::printf("%ld %ld %ld %ld\n", n_u, bad_u, n_f, bad_f);
  return (bad_u || bad_f) ? 1 : 0;
}
"""


def test_integer_built_doubles_match_the_host_conversions(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    src = tmp_path / "bits_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "bits_driver"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    print(r.stdout)
    n_u, bad_u, n_f, bad_f = (int(x) for x in r.stdout.split()[-4:])
    assert r.returncode == 0 and bad_u == 0 and bad_f == 0, r.stdout
    assert n_u > 3_500_000 and n_f == 256 * 4000
