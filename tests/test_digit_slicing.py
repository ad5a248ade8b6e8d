"""Host-side checks (no GPU) of the digit slicing that feeds the FP64-accurate
tensor-core GEMM: the header ``csrc/lc_digits.cuh`` is host and device code,
so a small host program compiled with nvcc runs the kernels' own arithmetic
on the CPU.

For digit widths beta = 6, 7 and S = 9, 8 slices it checks, on random values
spanning 2^-60 .. 2^60 and on edge cases (row maxima, powers of two, exact
rounding halves, zeros, subnormals, the fixed exponent used for unit rows):

* the row exponent e puts the row's largest entry in [1/8, 1/2) after
  scaling by 2^-e;
* oz_fixed(x, beta S - e) is x 2^(beta S - e) rounded to the nearest integer
  (error at most 1/2, computed in long double);
* every digit is an integer of magnitude <= 2^(beta-1) held exactly in BF16,
  and the digits rebuild that integer exactly (Horner in base 2^beta) -- the
  property a dropped carry of the top digit breaks;
* the paired form (two entries per call, BF16 pairs) gives the same digits;
* the exactness bound of one FP32 chain: K_max 2^(2 beta - 2) = 2^24.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2506_01120_gb300", "csrc")

HARNESS = r"""
#include "lc_digits.cuh"
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
using namespace lc;

static long long checks = 0, fails = 0;

static void fail(const char* what, double x, double rowmax, int beta) {
  if (fails < 20) printf("FAIL %s x=%.17g rowmax=%.17g beta=%d\n", what, x, rowmax, beta);
  ++fails;
}

static void digits_of(double x, int e, int S, int beta, long long* out) {
  __nv_bfloat16 d[16];
  oz_digits(x, e, S, beta, d, 1);
  for (int s = 0; s < S; ++s) {
    const float f = __bfloat162float(d[s]);
    out[s] = (long long)f;
    if ((float)out[s] != f) fail("digit not an integer", x, 0, beta);
  }
}

static void check_value(double x, int e, double rowmax, int beta, int S) {
  ++checks;
  long long d[16];
  digits_of(x, e, S, beta, d);
  const long long Y = oz_fixed(x, beta * S - e);
  long long rec = 0;
  for (int s = 0; s < S; ++s) {
    if (llabs(d[s]) > (1LL << (beta - 1))) fail("digit out of range", x, rowmax, beta);
    rec = rec * (1LL << beta) + d[s];
  }
  if (rec != Y) fail("digits do not rebuild the integer", x, rowmax, beta);
  if (std::fpclassify(x) == FP_NORMAL) {
    const long double t = (long double)x * ldexpl(1.0L, beta * S - e);
    if (fabsl(t - (long double)Y) > 0.5L) fail("rounding off by more than 1/2", x, rowmax, beta);
  } else if (Y != 0) {
    fail("zero or subnormal gives a nonzero integer", x, rowmax, beta);
  }
  // the paired form, second entry -x
  __nv_bfloat162 p[16];
  oz_digits2(x, -x, e, S, beta, p, 1);
  long long dn[16];
  digits_of(-x, e, S, beta, dn);
  for (int s = 0; s < S; ++s) {
    const float2 f = __bfloat1622float2(p[s]);
    if ((long long)f.x != d[s] || (long long)f.y != dn[s]) fail("paired digits differ", x, rowmax, beta);
  }
}

static int row_exp_of(double rowmax, int beta) {
  const int e = oz_row_exp(oz_bits(std::fabs(rowmax)));
  if (std::fpclassify(rowmax) == FP_NORMAL) {
    const long double r = fabsl((long double)rowmax) * ldexpl(1.0L, -e);
    if (!(r < 0.5L && r >= 0.125L)) fail("row exponent", rowmax, rowmax, beta);
  } else if (e != 0) {
    fail("row exponent of a zero or subnormal row", rowmax, rowmax, beta);
  }
  return e;
}

int main() {
  std::mt19937_64 rng(20250601);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> k(-60, 60);
  const int betas[2] = {6, 7}, slices[2] = {9, 8};
  for (int b = 0; b < 2; ++b) {
    const int beta = betas[b], S = slices[b];
    if (((1LL << (26 - 2 * beta)) << (2 * beta - 2)) != (1LL << 24)) fail("chain bound", 0, 0, beta);
    for (int r = 0; r < 4000; ++r) {
      const double rowmax = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), k(rng)) * (r & 1 ? -1.0 : 1.0);
      const int e = row_exp_of(rowmax, beta);
      check_value(rowmax, e, rowmax, beta, S);
      check_value(-rowmax, e, rowmax, beta, S);
      for (int i = 0; i < 40; ++i) check_value(rowmax * u(rng), e, rowmax, beta, S);
      check_value(rowmax * 1e-20, e, rowmax, beta, S);
      // an exact rounding half: (n + 1/2) 2^(e - beta S)
      const double half = std::ldexp((double)(rng() % 1000) + 0.5, e - beta * S);
      if (std::fabs(half) <= std::fabs(rowmax)) check_value(half, e, rowmax, beta, S);
    }
    for (int p = -40; p <= 40; ++p) {   // powers of two as row maxima
      const double rowmax = std::ldexp(1.0, p);
      const int e = row_exp_of(rowmax, beta);
      check_value(rowmax, e, rowmax, beta, S);
      check_value(-rowmax / 3.0, e, rowmax, beta, S);
    }
    // zero and subnormal rows and entries
    check_value(0.0, row_exp_of(0.0, beta), 0.0, beta, S);
    check_value(-0.0, 0, 0.0, beta, S);
    const double sub = std::ldexp(1.0, -1060);
    check_value(sub, row_exp_of(sub, beta), sub, beta, S);
    // unit rows with the fixed exponent 1: |v| <= 1, also one ulp above
    for (int i = 0; i < 20000; ++i) check_value(u(rng), 1, 1.0, beta, S);
    check_value(1.0, 1, 1.0, beta, S);
    check_value(-1.0, 1, 1.0, beta, S);
    check_value(std::nextafter(1.0, 2.0), 1, 1.0, beta, S);
  }
  printf("checks %lld fails %lld\n", checks, fails);
  return fails ? 1 : 0;
}
"""


def test_digit_slicing_host_arithmetic(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "digits.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "digits"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout
    last = out.stdout.strip().splitlines()[-1].split()
    assert last[0] == "checks" and int(last[1]) > 300000 and last[3] == "0"
