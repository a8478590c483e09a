"""Index maps of the sweep kernels, checked on the host: the library's own header is compiled into a
host program with nvcc and run here, so no GPU is needed.

- The multiply-shift division the sweep, residual and factor kernels use for their index maps
  (Granlund and Montgomery, PLDI 1994) against integer division.
- The colour classes the sweeps launch (2 colours per axis, the j-th CTA of a colour -> subvolume)
  and the subvolume boxes: every subvolume in exactly one colour, the boxes tile the grid, and two
  subvolumes of one colour are more than 2 points apart on some axis, so their unknowns share no
  entry of the radius-2 normal operator (exact parallel block Gauss-Seidel, Sec. II).
- The block band the library gives the finest-level factors, against the restatement that
  test_oracle_band.py pins on the oracle's own Cholesky factors."""
import os
import shutil
import subprocess

import pytest

from tests.test_oracle_band import band_blocks

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_1111_4363_gb300", "csrc", "la_internal.cuh")

PROGRAM = r"""
#include <stdio.h>
#include <vector>
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

// every subvolume in one colour, boxes tile the grid, same-colour boxes more than 2 points apart
static void check_colouring(int dim, int nx, int ny, int nz, int sx, int sy, int sz) {
  la::LevelGeom L = {};
  L.dim = dim;
  const int n[3] = {nx, ny, nz}, s[3] = {sx, sy, sz};
  L.np = 1;
  L.nsub = 1;
  for (int a = 0; a < 3; ++a) {
    L.n[a] = a < dim ? n[a] : 1;
    L.sub[a] = a < dim ? s[a] : 1;
    L.nb[a] = (L.n[a] + L.sub[a] - 1) / L.sub[a];
    L.np *= L.n[a];
    L.nsub *= L.nb[a];
  }
  std::vector<int> seen(L.nsub, 0), cover(L.np, 0);
  for (int colour = 0; colour < 8; ++colour) {
    const int cnt = la::colour_count(L, colour);
    if (colour >= (1 << dim) && cnt != 0) {
      printf("colour %d of a %dD level has %d subvolumes\n", colour, dim, cnt);
      ++fails;
    }
    std::vector<int> o(3 * cnt), e(3 * cnt);
    for (int j = 0; j < cnt; ++j) {
      const int b = la::colour_subvol(L, colour, j);
      if (b < 0 || b >= L.nsub) {
        printf("subvolume %d out of range\n", b);
        ++fails;
        return;
      }
      ++seen[b];
      la::subvol_box(L, b, &o[3 * j], &e[3 * j]);
      for (int a = 0; a < 3; ++a) {
        const int bb = a == 0 ? b % L.nb[0] : a == 1 ? (b / L.nb[0]) % L.nb[1] : b / (L.nb[0] * L.nb[1]);
        if ((bb & 1) != ((colour >> a) & 1) || e[3 * j + a] < 1) {
          printf("subvolume %d: axis %d parity or extent\n", b, a);
          ++fails;
        }
      }
      for (int z = 0; z < e[3 * j + 2]; ++z)
        for (int y = 0; y < e[3 * j + 1]; ++y)
          for (int x = 0; x < e[3 * j]; ++x)
            ++cover[((o[3 * j + 2] + z) * L.n[1] + o[3 * j + 1] + y) * L.n[0] + o[3 * j] + x];
    }
    for (int j = 0; j < (L.nsub <= 40000 ? cnt : 0); ++j)   // pairs: levels up to 40,000 subvolumes
      for (int k = j + 1; k < cnt; ++k) {
        bool apart = false;                       // gap > 2 points on some axis
        for (int a = 0; a < 3; ++a) {
          const int lo = o[3 * j + a] < o[3 * k + a] ? j : k, hi = lo == j ? k : j;
          if (o[3 * hi + a] - (o[3 * lo + a] + e[3 * lo + a] - 1) > 2) apart = true;
        }
        if (!apart) {
          if (fails < 10) printf("%dD %dx%dx%d sub %dx%dx%d colour %d: subvolumes %d and %d couple\n", dim, nx, ny,
                                 nz, sx, sy, sz, colour, j, k);
          ++fails;
        }
      }
  }
  for (int b = 0; b < L.nsub; ++b)
    if (seen[b] != 1) {
      printf("subvolume %d in %d colours\n", b, seen[b]);
      ++fails;
    }
  for (int p = 0; p < L.np; ++p)
    if (cover[p] != 1) {
      printf("point %d covered %d times\n", p, cover[p]);
      ++fails;
      return;
    }
}

int main() {
  // the workloads' levels (256^2 with 4 x 4 then 2 x 2 subvolumes, 128^3 and 8x8x6 with 2 x 2 x 2,
  // 64 points with 8, the ragged 30 x 22 parity grid) and ragged extents of every kind
  check_colouring(1, 64, 1, 1, 8, 1, 1);
  for (int n = 256; n >= 32; n /= 2) check_colouring(2, n, n, 1, n == 256 ? 4 : 2, n == 256 ? 4 : 2, 1);
  check_colouring(2, 30, 22, 1, 4, 4, 1);
  check_colouring(2, 15, 11, 1, 2, 2, 1);
  for (int n = 128; n >= 16; n /= 2) check_colouring(3, n, n, n, 2, 2, 2);
  check_colouring(3, 8, 8, 6, 2, 2, 2);
  for (int nx = 2; nx <= 19; ++nx)
    for (int ny = 2; ny <= 13; ny += 3)
      for (int sx = 2; sx <= 5; ++sx)
        for (int sy = 2; sy <= 4; ++sy) {
          check_colouring(2, nx, ny, 1, sx, sy, 1);
          check_colouring(3, nx, ny, 7, sx, sy, 3);
        }
  for (int d = 1; d <= 4096; ++d) check_divisor(d, d <= 1024 ? 1 << 16 : 1 << 12);
  for (int b = 12; b < 31; ++b)                  // powers of two and their neighbours
    for (int e = -1; e <= 1; ++e) check_divisor((1 << b) + e, 1 << 10);
  check_divisor(0x7fffffff, 1 << 10);
  for (int k = 0; k < 20000; ++k) {
    const int d = 1 + (int)(rnd31() % 0x7ffffffeu);
    check_divisor(d, 64);
  }
  // block band of the finest-level factors: one line per case, compared with the Python restatement
  for (int dim = 1; dim <= 3; ++dim)
    for (int sx = 1; sx <= 8; ++sx)
      for (int sy = 1; sy <= (dim > 1 ? 8 : 1); ++sy)
        for (int sz = 1; sz <= (dim > 2 ? 4 : 1); ++sz)
          for (int K = 1; K <= 8; ++K) {
            const int sub[3] = {sx, sy, sz}, n = sx * sy * sz * K;
            if (n > 256) continue;
            const int nblk = (n + LA_BLK - 1) / LA_BLK;
            printf("band %d %d %d %d %d %d %d\n", dim, sx, sy, sz, K, nblk, la::fine_band_blocks(dim, sub, K, nblk));
          }
  printf("fails %lld\n", fails);
  return fails != 0;
}
"""


def test_index_maps_on_the_host(tmp_path):
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
    bands = [tuple(int(v) for v in line.split()[1:]) for line in out.stdout.splitlines()
             if line.startswith("band ")]
    assert len(bands) > 300
    seen = {}
    for dim, sx, sy, sz, K, nblk, band in bands:
        want = min(max(band_blocks(dim, (sx, sy, sz), K, nblk), 1), nblk - 1)
        assert band == want, (dim, sx, sy, sz, K, nblk, band, want)
        seen[(dim, sx, sy, sz, K)] = band
    # the finest levels the wide factorisation runs on: 4 x 4 x 4 and 8 x 8 points with K = 4
    assert seen[(3, 4, 4, 4, 4)] == 8 and seen[(2, 8, 8, 1, 4)] == 4
