"""The multiply-shift division that the sweep, residual and factor kernels use for their index maps
(Granlund and Montgomery, PLDI 1994), checked on the host against integer division: the library's
own header is compiled into a host program with nvcc and run here, so no GPU is needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_1111_4363_gb300", "csrc", "la_internal.cuh")

PROGRAM = r"""
#include <stdio.h>
#include "la_internal.cuh"
using la::FastDiv;
using la::fdiv;
using la::make_fastdiv;

static unsigned long long state = 0x9E3779B97F4A7C15ull;
static unsigned rnd31() {                       // splitmix64, top 31 bits
  unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (unsigned)((z ^ (z >> 31)) >> 33);
}

static long long fails = 0;
static void check(int x, const FastDiv& f) {
  if (fdiv(x, f) != x / f.d) {
    if (fails < 10) printf("x=%d d=%d got %d want %d\n", x, f.d, fdiv(x, f), x / f.d);
    ++fails;
  }
}
static void check_divisor(int d, int dense) {
  unsigned l = 0;
  while ((1u << l) < (unsigned)d) ++l;
  if ((1ull << (31 + l)) / (unsigned long long)d + 1ull >= (1ull << 32)) {
    printf("multiplier overflows for d=%d\n", d);
    ++fails;
  }
  const FastDiv f = make_fastdiv(d);
  for (int x = 0; x < dense; ++x) check(x, f);
  for (int k = 0; k < 64; ++k) {                 // the top of the range and around multiples of d
    check(0x7fffffff - k, f);
    const long long q = (0x7fffffffll / d) - k;
    if (q >= 0)
      for (int e = -1; e <= 1; ++e) {
        const long long x = q * d + e;
        if (x >= 0 && x <= 0x7fffffff) check((int)x, f);
      }
  }
  for (int k = 0; k < 256; ++k) check((int)rnd31(), f);
}

int main() {
  for (int d = 1; d <= 4096; ++d) check_divisor(d, d <= 1024 ? 1 << 16 : 1 << 12);
  for (int b = 12; b < 31; ++b)                  // powers of two and their neighbours
    for (int e = -1; e <= 1; ++e) check_divisor((1 << b) + e, 1 << 10);
  check_divisor(0x7fffffff, 1 << 10);
  for (int k = 0; k < 20000; ++k) {
    const int d = 1 + (int)(rnd31() % 0x7ffffffeu);
    check_divisor(d, 64);
  }
  printf("fails %lld\n", fails);
  return fails != 0;
}
"""


def test_multiply_shift_division_is_exact(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "fastdiv_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fastdiv_check"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().endswith("fails 0")
