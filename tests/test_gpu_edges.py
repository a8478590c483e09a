"""Edge and degenerate cases of the CUDA path against the oracle (GB300 required): every size class
of the time basis (K = 1, 2, 5, 8, including the largest subvolume of 128 unknowns), odd K in mixed
precision (per-point complex64 kernels instead of the TMA-staged ones), a grid that is one
subvolume, no laser field, a ragged 3D grid, zero steps, a zero initial state, a different grid
spacing on every axis and the laser coupled along y or z."""
import dataclasses

import numpy as np
import pytest

from oracle import multigrid, system
from oracle.propagate import numpy_coarse_nu, numpy_coarse_sub, numpy_sub
from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, oracle_system, rel_l2, small_3d

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def fixed_cycles(w, ncycles, t0=0.2):
    """ncycles cycles from c = 0 on the GPU and in the oracle with the identical schedule."""
    psi0 = wl.initial_state(w).ravel()
    prob, M, f, W = oracle_system(w, psi0, t0)
    c_ref, hist, _, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, numpy_sub(w), w.levels, w.nu1, w.nu2,
                                             w.coarse_sweeps, ncycles=ncycles, coarse_sub=numpy_coarse_sub(w),
                                             coarse_nu=numpy_coarse_nu(w))
    ctx = gpu_context(w)
    c = np.zeros(M.shape[1], dtype=np.complex128)
    st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, t0, c, ncycles=ncycles)
    return c, c_ref, N, hist[-1]


@pytest.mark.parametrize("K", [1, 2, 5, 8])
def test_every_time_basis_size(K):
    """4x4 subvolumes with K time functions: 16 (K=1) to 128 (K=8) unknowns per subvolume."""
    w = dataclasses.replace(wl.softcore_2d(n=16, levels=2), nt=K)
    c, c_ref, N, N_ref = fixed_cycles(w, 2)
    assert rel_l2(c, c_ref) < TOL64
    assert N == pytest.approx(N_ref, rel=1e-9)


def test_largest_subvolume():
    """8x4 points x 4 time functions = 128 unknowns, the largest one-CTA factorisation."""
    w = dataclasses.replace(wl.softcore_2d(n=32, levels=2), nt=4, sub=(8, 4, 1))
    c, c_ref, _, _ = fixed_cycles(w, 2)
    assert rel_l2(c, c_ref) < TOL64


@pytest.mark.parametrize("K", [3, 5])
def test_mixed_precision_with_odd_K(K):
    """Odd K has no tensor map (16-byte TMA rule), so the complex64 V-cycle takes the per-point
    kernels; refined to 1e-22 it reaches the FP64 direct solution."""
    w = dataclasses.replace(wl.softcore_2d(n=16, levels=2), nt=K)
    psi0 = wl.initial_state(w).ravel()
    prob, M, f, W = oracle_system(w, psi0, 0.0)
    cd = system.direct_solve(M, f)
    ctx = gpu_context(w, precision=1, tol=1e-22, max_cycles=80)
    c = np.zeros(M.shape[1], dtype=np.complex128)
    st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, 0.0, c)
    assert rel <= 1e-22
    assert rel_l2(c, cd) < 1e-9


def test_grid_of_one_subvolume():
    """4x4 grid, 4x4 subvolume, one level: only colour 0 has a subvolume."""
    w = dataclasses.replace(wl.softcore_2d(n=16, levels=1), n=(4, 4, 1))
    c, c_ref, _, _ = fixed_cycles(w, 3)
    assert rel_l2(c, c_ref) < TOL64


def test_no_laser_field():
    w = dataclasses.replace(wl.softcore_2d(n=16, levels=2), pulse=None)
    c, c_ref, _, _ = fixed_cycles(w, 2)
    assert rel_l2(c, c_ref) < TOL64


def test_ragged_3d_grid():
    """10x6x7 points with 4x2x2 subvolumes: tails of 2 and 1 points, one level."""
    w = dataclasses.replace(small_3d(levels=1), n=(10, 6, 7), sub=(4, 2, 2))
    c, c_ref, _, _ = fixed_cycles(w, 2)
    assert rel_l2(c, c_ref) < TOL64


def test_zero_steps_leave_the_state_unchanged():
    w = wl.softcore_2d(n=16, levels=2)
    ctx = gpu_context(w)
    psi0 = wl.initial_state(w).ravel()
    psi = psi0.copy()
    ctx.step(psi, 0, 0.0)
    assert np.array_equal(psi, psi0)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_initial_state_stays_zero(precision):
    """psi0 = 0: f = 0, N(0) = 0, no cycle runs and the state stays exactly zero."""
    w = dataclasses.replace(wl.softcore_2d(n=16, levels=2), trial=3)
    ctx = gpu_context(w, precision=precision)
    psi = np.zeros(w.npoints, dtype=np.complex128)
    st, stats = ctx.step(psi, 3, 0.0, stats=True)
    assert np.count_nonzero(psi) == 0
    assert all(s[0] == 0 and s[3] == 0.0 for s in stats)


ANISOTROPIC = {
    # a different spacing, and extent, on every axis: the per-axis kinetic weights of the fine stencil,
    # of the footprint residual, of the wide factorisation's (H, H^2) table and of the Galerkin levels
    "2d_4x4_K6": lambda: dataclasses.replace(wl.softcore_2d(n=16, levels=2), n=(16, 12, 1), h=(0.2, 0.35, 1.0)),
    "3d_2x2x2_K4": lambda: dataclasses.replace(small_3d(), h=(0.3, 0.45, 0.25)),
    "3d_4x4x4_K4_wide": lambda: dataclasses.replace(wl.hydrogen_3d(n=8, nsteps=4, ncomp=4, sub=4), n=(16, 8, 8),
                                                    h=(0.3, 0.45, 0.25), levels=2),
}


@pytest.mark.parametrize("name", list(ANISOTROPIC))
def test_anisotropic_spacing(name):
    c, c_ref, N, N_ref = fixed_cycles(ANISOTROPIC[name](), 2)
    assert rel_l2(c, c_ref) < TOL64
    assert N == pytest.approx(N_ref, rel=1e-9)


def strong_pulse(axis):
    """Two components, one enveloped, strong enough at t0 = 0.2 that the coupling axis shows."""
    return wl.Pulse(amp=[0.3, -0.2], omega=[1.1, 0.7], t_center=[0.25, 0.1], sigma=[0.5, 0.0], axis=axis)


LASER_AXES = {
    # the dipole coupling along y and z: the laser coordinate of the residual stencils, of the
    # footprint sweeps, of the one-CTA and wide factorisations and of the Galerkin construction
    "2d_y": lambda: dataclasses.replace(ANISOTROPIC["2d_4x4_K6"](), pulse=strong_pulse(1)),
    "3d_y": lambda: dataclasses.replace(ANISOTROPIC["3d_2x2x2_K4"](), pulse=strong_pulse(1)),
    "3d_z_wide": lambda: dataclasses.replace(ANISOTROPIC["3d_4x4x4_K4_wide"](), pulse=strong_pulse(2)),
}


@pytest.mark.parametrize("name", list(LASER_AXES))
def test_laser_axis(name):
    c, c_ref, N, N_ref = fixed_cycles(LASER_AXES[name](), 2)
    assert rel_l2(c, c_ref) < TOL64
    assert N == pytest.approx(N_ref, rel=1e-9)


@pytest.mark.parametrize("name", list(LASER_AXES))
def test_mixed_precision_contracts_like_fp64_on_every_axis(name):
    """The complex64 kernels (TMA-staged stencils, float factors and sweeps, float Galerkin levels) on
    the anisotropic grids with the laser along y or z: a wrong spacing or coupling axis there would
    leave only the FP64 refinement right and slow the contraction far below the FP64 path's, so
    after the same two cycles N/N(0) agrees with it within a factor of two."""
    w = LASER_AXES[name]()
    psi0 = wl.initial_state(w).ravel()
    rels = []
    for precision in (0, 1):
        ctx = gpu_context(w, precision=precision)
        c = np.zeros(w.nunknowns, dtype=np.complex128)
        st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, 0.2, c, ncycles=2)
        rels.append(rel)
    assert rels[0] < 1e-6
    assert rels[1] <= 2 * rels[0] + 1e-20, rels
