"""Pins for the oracle's discrete adjoint: central finite differences of the forward map."""

import numpy as np
import pytest

from oracle import adjoint, system
from paper_1111_4363_gb300 import workloads as wl


def small_pulsed(n=10, dim=1, ncomp=3, nsteps=5):
    if dim == 1:
        w = wl.harmonic_1d()
        w.n = (n, 1, 1)
        w.h = (0.5, 1.0, 1.0)
    else:
        w = wl.softcore_2d(n=n, levels=1)
    w.nt = 3
    rng = np.random.default_rng(7)
    T = nsteps * w.dt
    w.pulse = wl.Pulse(amp=list(rng.normal(0, 0.3, ncomp)), omega=[2.0] * ncomp,
                       t_center=list(np.linspace(0, T, ncomp)), sigma=[T / 2] * ncomp, axis=0)
    return w


@pytest.mark.parametrize("dim", [1, 2])
def test_amplitude_gradient_matches_finite_differences(dim):
    w = small_pulsed(n=10 if dim == 1 else 6, dim=dim)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    g, _ = adjoint.gradients(prob, psi0, nsteps=5)
    g_fd = adjoint.finite_difference_gradient(prob, psi0, nsteps=5, eps=1e-5)
    np.testing.assert_allclose(g, g_fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(g_fd)))


def test_initial_state_gradient_matches_finite_differences():
    w = small_pulsed(n=10)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    _, lam0 = adjoint.gradients(prob, psi0, nsteps=4)
    rng = np.random.default_rng(1)
    d = rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)
    eps = 1e-6
    Jp = system.dipole(prob, adjoint.forward(prob, psi0 + eps * d, 4)[0][-1])
    Jm = system.dipole(prob, adjoint.forward(prob, psi0 - eps * d, 4)[0][-1])
    fd = (Jp - Jm) / (2 * eps)
    # dJ = 2 Re(lambda_0^dagger dpsi)
    assert fd == pytest.approx(2 * np.real(np.vdot(lam0, d)), rel=1e-7)
