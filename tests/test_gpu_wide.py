"""Finest-level subvolumes of more than 128 unknowns (up to 4 x 4 x 4 points x K = 4 = 256, the 3D
workload's subvolume, Sec. II's larger relaxation volumes), factorised in global memory, against the
oracle (GB300 required): single colour passes (exact block minimisation), fixed V-cycle schedules with
2 x 2 x 2 Galerkin subvolumes, ragged tails, 2D 8 x 8 blocks, the padded size 192, mixed precision
and converged steps against the direct solve."""
import dataclasses

import numpy as np
import pytest

from oracle import multigrid, relax, system
from oracle.propagate import numpy_coarse_nu, numpy_coarse_sub, numpy_sub
from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, oracle_system, rel_l2

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def h3(n, sub=(4, 4, 4), K=4, levels=1, **kw):
    w = wl.hydrogen_3d(n=8, nsteps=8, ncomp=4, sub=4)
    return dataclasses.replace(w, n=n, sub=sub, nt=K, levels=levels, coarse_sub=(2, 2, 2), **kw)


def s2(n, sub=(8, 8, 1), K=4, levels=1, **kw):
    w = wl.softcore_2d(n=16, levels=1)
    return dataclasses.replace(w, n=n, sub=sub, nt=K, levels=levels, coarse_sub=(2, 2, 1), **kw)


CASES = {
    "3d_4x4x4_K4": lambda: h3((8, 8, 8)),                       # 256 unknowns, two blocks per axis
    "3d_4x4x4_K3_ragged": lambda: h3((8, 8, 6), K=3),           # 192 unknowns, z tail of 2
    "3d_4x4x2_K8": lambda: h3((8, 8, 4), sub=(4, 4, 2), K=8),   # 256 unknowns, K = 8
    "2d_8x8_K4": lambda: s2((16, 24, 1)),                       # 256 unknowns, 2D
    "2d_8x4_K6_ragged": lambda: s2((20, 12, 1), sub=(8, 4, 1), K=6),   # 192 unknowns, x tail of 4
}


@pytest.mark.parametrize("weight", ["dual", "identity"])
@pytest.mark.parametrize("name", list(CASES))
def test_wide_single_colour_pass(name, weight):
    w = dataclasses.replace(CASES[name](), weight=weight)
    ctx = gpu_context(w)
    psi0 = wl.initial_state(w).ravel()
    t0 = 0.35
    prob, M, f, W = oracle_system(w, psi0, t0)
    G = (M.conj().T @ W @ M).tocsr()
    g = M.conj().T @ (W @ f)
    R = relax.BlockRelaxation(G, prob.shape, numpy_sub(w), prob.K)
    c0 = wl.random_state(M.shape[1], 5) * 0.05
    for colour in range(1 << w.dim):
        ref = c0.copy()
        R.colour_pass(ref, g, colour)
        got = c0.copy()
        ctx.relax_colour(psi0, t0, colour, got)
        assert rel_l2(got - c0, ref - c0) < 1e-10, colour
        assert rel_l2(got, ref) < TOL64, colour


def fixed_cycles(w, ncycles, t0=0.2, precision=0):
    psi0 = wl.initial_state(w).ravel()
    prob, M, f, W = oracle_system(w, psi0, t0)
    c_ref, hist, _, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, numpy_sub(w), w.levels, w.nu1, w.nu2,
                                             w.coarse_sweeps, ncycles=ncycles, coarse_sub=numpy_coarse_sub(w),
                                             coarse_nu=numpy_coarse_nu(w))
    ctx = gpu_context(w, precision=precision)
    c = np.zeros(M.shape[1], dtype=np.complex128)
    st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, t0, c, ncycles=ncycles)
    assert cycles == ncycles
    return c, c_ref, N, hist[-1]


@pytest.mark.parametrize("name,n,levels", [("8^3, 2 levels", (8, 8, 8), 2), ("16^3, 3 levels", (16, 16, 16), 3),
                                           ("16x8x12, 2 levels", (16, 8, 12), 2)])
def test_wide_fixed_schedule_v_cycles(name, n, levels):
    """Two V(1,2) cycles with a (1,0) Galerkin cycle, 4x4x4 finest subvolumes and 2x2x2 Galerkin ones
    (the 3D workload's schedule), from c = 0, against the oracle's multigrid."""
    w = h3(n, levels=levels, nu2=2, coarse_nu=(1, 0))
    c, c_ref, N, N_ref = fixed_cycles(w, 2)
    assert rel_l2(c, c_ref) < TOL64
    assert N == pytest.approx(N_ref, rel=1e-9)


def test_wide_ragged_3d_grid():
    """10x6x7 points with 4x4x4 subvolumes: tails of 2, 2 and 3 points (16 to 64 points per block)."""
    w = h3((10, 6, 7))
    c, c_ref, _, _ = fixed_cycles(w, 2)
    assert rel_l2(c, c_ref) < TOL64


@pytest.mark.parametrize("name", ["3d_4x4x4_K4", "2d_8x8_K4"])
def test_wide_converged_step_matches_direct_solve(name):
    w = dataclasses.replace(CASES[name](), levels=2)
    psi0 = wl.initial_state(w).ravel()
    prob, M, f, W = oracle_system(w, psi0, 0.0)
    cd = system.direct_solve(M, f)
    for precision in (0, 1):
        ctx = gpu_context(w, precision=precision, tol=1e-24 if precision == 0 else 1e-22, max_cycles=80)
        c = np.zeros(M.shape[1], dtype=np.complex128)
        st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, 0.0, c)
        assert rel <= (1e-24 if precision == 0 else 1e-22), (precision, rel)
        assert rel_l2(c, cd) < 1e-9, precision


def test_wide_mixed_precision_cycles_contract_like_fp64():
    """The complex64 wide factors precondition the FP64-refined iteration as well as the FP64 ones:
    after the same number of cycles N/N(0) agrees within a factor of two."""
    w = h3((16, 16, 16), levels=3, nu2=2, coarse_nu=(1, 0))
    psi0 = wl.initial_state(w).ravel()
    rels = []
    for precision in (0, 1):
        ctx = gpu_context(w, precision=precision)
        c = np.zeros(w.nunknowns, dtype=np.complex128)
        st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, 0.2, c, ncycles=3)
        rels.append(rel)
    assert rels[1] <= 2 * rels[0] + 1e-20, rels
