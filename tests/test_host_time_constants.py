"""The CUDA path's host-side time-basis constants (S0: the closed forms of Sec. IV and the Gauss rule
the per-step field matrices use) against the oracle, on the CPU: the library's own header is compiled
into a host program with nvcc and its output compared with the oracle's quadrature.

- Ub, Qb, Ub0 (closed forms on the library side, Gauss-Legendre quadrature in the oracle) and the end
  values b_n(+1), for K = 1..8 and two steps.
- The residual-norm weight Wt: Ub^{-1} (default), Ub, identity.
- The K + 8-node Gauss rule and the b_m at its nodes, and the 48-node rule of the plane-wave maps,
  against numpy's Gauss-Legendre rule and the oracle's b functions."""
import os
import shutil
import subprocess

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import timebasis as tb

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_1111_4363_gb300", "csrc", "la_internal.cuh")

PROGRAM = r"""
#include <stdio.h>
#include "la_internal.cuh"

static void row(const char* tag, int K, double dt, int weight, const double* v, int n) {
  printf("%s %d %.17g %d", tag, K, dt, weight);
  for (int i = 0; i < n; ++i) printf(" %.17g", v[i]);
  printf("\n");
}

int main() {
  const double dts[2] = {0.05, 0.7};
  for (int K = 1; K <= LA_KMAX; ++K)
    for (int d = 0; d < 2; ++d)
      for (int weight = 0; weight < 3; ++weight) {
        la::TimeMats t;
        if (!la::fill_time_constants(K, dts[d], weight, t)) {
          printf("failed %d\n", K);
          return 1;
        }
        row("Ub", K, dts[d], weight, t.Ub, K * K);
        row("Qb", K, dts[d], weight, t.Qb, K * K);
        row("Ub0", K, dts[d], weight, t.Ub0, K);
        row("endv", K, dts[d], weight, t.endv, K);
        row("Wt", K, dts[d], weight, t.Wt, K * K);
        row("tau", K, dts[d], weight, t.tau, t.nq);
        row("wq", K, dts[d], weight, t.wq, t.nq);
        row("bq", K, dts[d], weight, t.bq, t.nq * LA_KMAX);
      }
  double x[48], w[48];
  la::gauss_legendre(48, x, w);
  row("x48", 0, 0.0, 0, x, 48);
  row("w48", 0, 0.0, 0, w, 48);
  return 0;
}
"""


@pytest.fixture(scope="module")
def constants(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("time_constants")
    src, exe = d / "time_constants.cu", d / "time_constants"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    table = {}
    for line in out.stdout.splitlines():
        f = line.split()
        table[(f[0], int(f[1]), float(f[2]), int(f[3]))] = np.array([float(v) for v in f[4:]])
    return table


@pytest.mark.parametrize("K", range(1, 9))
@pytest.mark.parametrize("dt", [0.05, 0.7])
def test_static_time_matrices_match_the_oracle(constants, K, dt):
    Ub, Qb, Ub0 = tb.static_matrices(K, dt)
    for weight in range(3):
        got = lambda tag: constants[(tag, K, dt, weight)]
        np.testing.assert_allclose(got("Ub").reshape(K, K), Ub, rtol=0, atol=1e-14 * max(1.0, K * dt))
        np.testing.assert_allclose(got("Qb").reshape(K, K), Qb, rtol=0, atol=1e-13)
        np.testing.assert_allclose(got("Ub0"), Ub0, rtol=0, atol=1e-15)
        np.testing.assert_array_equal(got("endv"), tb.end_values(K))
        Wt = got("Wt").reshape(K, K)
        want = {0: np.linalg.inv(Ub), 1: Ub, 2: np.eye(K)}[weight]
        np.testing.assert_allclose(Wt, want, rtol=1e-10, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("K", range(1, 9))
def test_gauss_rule_and_basis_at_its_nodes(constants, K):
    nq = K + 8
    tau = constants[("tau", K, 0.05, 0)]
    wq = constants[("wq", K, 0.05, 0)]
    x, w = npleg.leggauss(nq)
    order = np.argsort(tau)
    np.testing.assert_allclose(tau[order], x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(wq[order], w, rtol=0, atol=1e-15)
    bq = constants[("bq", K, 0.05, 0)].reshape(nq, -1)[:, :K]
    b, _ = tb.b_functions(K, tau)
    np.testing.assert_allclose(bq, b.T, rtol=0, atol=1e-13)


def test_48_node_rule_of_the_plane_wave_maps(constants):
    x, w = constants[("x48", 0, 0.0, 0)], constants[("w48", 0, 0.0, 0)]
    xr, wr = npleg.leggauss(48)
    order = np.argsort(x)
    # two independent routes to the rule (Newton on P_48 here, numpy's own): rounding of a few ulps
    np.testing.assert_allclose(x[order], xr, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w[order], wr, rtol=0, atol=1e-14)
    assert abs(np.sum(w) - 2.0) < 1e-14
