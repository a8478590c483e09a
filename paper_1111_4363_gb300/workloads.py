"""Seeded synthetic inputs for the least-action propagator.

This module is shared by the CUDA path, the tests, the benchmark and the CPU
oracle.  It holds only problem *definitions* (grid placement, potential
samples, initial wavefunctions, laser-pulse parameters, relaxation schedule);
none of the least-action arithmetic (time matrices, action residual, local
solves, transfers) lives here.

Grid placement (a reading: the paper does not fix it): on each axis the points
are x_k = (k - (n-1)/2) h, k = 0..n-1, with homogeneous Dirichlet walls one
spacing beyond the outermost points.  Mass m = 1 (atomic units).

Arrays use numpy C order with x fastest: shape (n_z, n_y, n_x) truncated to
``dim`` axes, so the flat point index is p = (z*n_y + y)*n_x + x.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


@dataclasses.dataclass
class Pulse:
    """Laser field E(t) = sum_k amp_k * env_k(t) * sin(omega_k t), coupled as E(t) * x_axis.

    env_k(t) = exp(-((t - t_center_k)/sigma_k)^2) when sigma_k > 0, else 1.
    """
    amp: List[float]
    omega: List[float]
    t_center: List[float]
    sigma: List[float]
    axis: int = 0

    @property
    def ncomp(self) -> int:
        return len(self.amp)


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    n: Tuple[int, int, int]          # points per axis, (n_x, n_y, n_z); unused axes are 1
    h: Tuple[float, float, float]    # spacing per axis
    nt: int                          # K: free Legendre time functions per point
    dt: float
    sub: Tuple[int, int, int]        # subvolume extent in points per axis (finest level)
    levels: int                      # multigrid levels (1 = single-level relaxation)
    nu1: int = 1
    nu2: int = 1
    coarse_sweeps: int = 2
    max_cycles: int = 60
    tol: float = 1e-10               # relative action N(c)/N(0)
    weight: str = "dual"             # residual-norm weight: "dual" | "literal" | "identity"
    nsteps: int = 1
    potential: str = "harmonic"      # "harmonic" | "softcore" | "zero"
    softcore_a: float = 1.0          # V = -1/sqrt(r^2 + a)
    pulse: Optional[Pulse] = None
    psi_kind: str = "gaussian"       # "displaced_noisy" | "gaussian"
    seed: int = 0
    coarse_sub: Optional[Tuple[int, int, int]] = None   # subvolume extent on Galerkin levels (None: sub)
    trial: int = 0                 # la_step trial iterate: 0 = zero, 1..3 = extrapolation from 1..3 steps
    coarse_nu: Optional[Tuple[int, int]] = None   # (nu1, nu2) on Galerkin levels above the coarsest (None: nu1, nu2)
    local_form: str = "lsq"        # subvolume problem: "lsq" (least squares) | "square" (Dirichlet form, red-black)
    factor_group: int = 0          # CTA packing of the small-subvolume factorisations: 0 by size, 1 one per CTA

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape, slowest axis first."""
        return tuple(self.n[a] for a in reversed(range(self.dim)))

    @property
    def npoints(self) -> int:
        return int(np.prod(self.shape))

    @property
    def nunknowns(self) -> int:
        return self.npoints * self.nt


def axis_coordinates(n: int, h: float) -> np.ndarray:
    """x_k = (k - (n-1)/2) h."""
    return (np.arange(n, dtype=np.float64) - 0.5 * (n - 1)) * h


def coordinate_arrays(w: Workload) -> List[np.ndarray]:
    """Per-axis coordinate arrays broadcast to the full grid, index a = 0 is x."""
    axes = [axis_coordinates(w.n[a], w.h[a]) for a in range(w.dim)]
    # numpy meshgrid with 'ij' on reversed axes gives arrays of shape w.shape
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    return list(reversed(grids))


def potential(w: Workload) -> np.ndarray:
    """Static potential V0 sampled at the grid points, float64 array of shape w.shape."""
    xs = coordinate_arrays(w)
    r2 = sum(x * x for x in xs)
    if w.potential == "harmonic":
        return 0.5 * r2
    if w.potential == "softcore":
        return -1.0 / np.sqrt(r2 + w.softcore_a)
    if w.potential == "zero":
        return np.zeros(w.shape)
    raise ValueError(w.potential)


def laser_coordinate(w: Workload) -> np.ndarray:
    """The dipole coordinate x_axis at every point (the spatial factor of E(t) x)."""
    axis = w.pulse.axis if w.pulse is not None else 0
    return coordinate_arrays(w)[axis]


def initial_state(w: Workload) -> np.ndarray:
    """Seeded initial wavefunction psi0, complex128 array of shape w.shape."""
    rng = np.random.default_rng(w.seed)
    xs = coordinate_arrays(w)
    if w.psi_kind == "displaced_noisy":
        # pi^{-1/4} exp(-(x-1)^2/2) + 1e-3 (N(0,1) + i N(0,1)), no renormalisation
        g = math.pi ** (-0.25) * np.exp(-0.5 * (xs[0] - 1.0) ** 2)
        noise = rng.standard_normal(w.shape) + 1j * rng.standard_normal(w.shape)
        return (g + 1e-3 * noise).astype(np.complex128)
    if w.psi_kind == "gaussian":
        r0 = rng.uniform(-2.0, 2.0, size=w.dim)
        k0 = rng.uniform(-0.5, 0.5, size=w.dim)
        arg = sum(-0.5 * (xs[a] - r0[a]) ** 2 + 1j * k0[a] * xs[a] for a in range(w.dim))
        psi = np.exp(arg)
        vol = float(np.prod(w.h[: w.dim]))
        psi /= math.sqrt(float(np.sum(np.abs(psi) ** 2)) * vol)
        return psi.astype(np.complex128)
    if w.psi_kind == "centred":
        arg = sum(-0.5 * xs[a] ** 2 for a in range(w.dim))
        psi = np.exp(arg).astype(np.complex128)
        vol = float(np.prod(w.h[: w.dim]))
        psi /= math.sqrt(float(np.sum(np.abs(psi) ** 2)) * vol)
        return psi
    raise ValueError(w.psi_kind)


def random_state(shape, seed: int) -> np.ndarray:
    """Seeded complex normal array (test inputs such as trial coefficients)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


# ----------------------------------------------------------------------------------------
# The five synthetic workloads.  Unspecified parameters (dt for 2D/3D, envelopes, initial
# states) are readings; they are listed with their reasons in the design notes.
# ----------------------------------------------------------------------------------------

def harmonic_1d() -> Workload:
    """1D, 64 points on [-8, 8], V = x^2/2, K = 4, dt = 0.05, 8-point subvolumes, 2 colours, no multigrid."""
    return Workload(name="1d_harmonic_64", dim=1, n=(64, 1, 1), h=(16.0 / 65.0, 1.0, 1.0), nt=4, dt=0.05,
                    sub=(8, 1, 1), levels=1, nu1=1, nu2=0, coarse_sweeps=0, max_cycles=400, tol=1e-12,
                    nsteps=20, potential="harmonic", psi_kind="displaced_noisy", seed=0)


def softcore_2d(n: int = 256, levels: int = 4, nsteps: int = 200) -> Workload:
    """2D, n x n points, h = 0.2, soft-core Coulomb -1/sqrt(r^2+1), laser 0.05 sin(0.057 t) x, K = 6."""
    return Workload(name=f"2d_softcore_{n}x{n}_K6", dim=2, n=(n, n, 1), h=(0.2, 0.2, 1.0), nt=6, dt=0.05,
                    sub=(4, 4, 1), levels=levels, nu1=1, nu2=1, coarse_sweeps=1, max_cycles=60, tol=1e-10,
                    nsteps=nsteps, potential="softcore", softcore_a=1.0,
                    pulse=Pulse(amp=[0.05], omega=[0.057], t_center=[0.0], sigma=[0.0], axis=0),
                    psi_kind="gaussian", seed=0, coarse_sub=(2, 2, 1))


def batched_2d(index: int) -> Workload:
    """One member of the batched family: seeded n in {64, 80, ..., 256}, E0 ~ U[0.01, 0.1], a ~ U[0.5, 2], K = 4."""
    rng = np.random.default_rng(index)
    n = int(rng.choice(np.arange(64, 257, 16)))
    e0 = float(rng.uniform(0.01, 0.1))
    a = float(rng.uniform(0.5, 2.0))
    return Workload(name=f"2d_batched_{index}", dim=2, n=(n, n, 1), h=(0.2, 0.2, 1.0), nt=4, dt=0.05,
                    sub=(4, 4, 1), levels=4, nu1=1, nu2=1, coarse_sweeps=2, max_cycles=60, tol=1e-10,
                    nsteps=100, potential="softcore", softcore_a=a,
                    pulse=Pulse(amp=[e0], omega=[0.057], t_center=[0.0], sigma=[0.0], axis=0),
                    psi_kind="gaussian", seed=index)


def hydrogen_3d(n: int = 128, nsteps: int = 400, ncomp: int = 32, sub: int = 4) -> Workload:
    """3D, n^3 points, h = 0.3, V = -1/sqrt(r^2+0.64), 32-component Gaussian-enveloped pulse on x, K = 4;
    sub^3-point finest subvolumes (4^3 x 4 = 256 unknowns), 2^3-point subvolumes on the Galerkin levels."""
    rng = np.random.default_rng(0)
    T = nsteps * 0.05
    amp = list(rng.normal(0.0, 0.02, size=ncomp))
    tc = list(np.linspace(0.0, T, ncomp))
    sig = [T / ncomp] * ncomp
    om = [0.057] * ncomp
    return Workload(name=f"3d_hydrogen_{n}^3_K4", dim=3, n=(n, n, n), h=(0.3, 0.3, 0.3), nt=4, dt=0.05,
                    sub=(sub, sub, sub), levels=4, nu1=1, nu2=1, coarse_sweeps=2, max_cycles=60, tol=1e-10,
                    nsteps=nsteps, potential="softcore", softcore_a=0.64,
                    pulse=Pulse(amp=amp, omega=om, t_center=tc, sigma=sig, axis=0),
                    psi_kind="centred", seed=0, coarse_sub=(2, 2, 2))
