"""la_backward (discrete adjoint on the forward factors) vs the oracle adjoint and finite differences."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint, system
from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def pulsed(kind: str, axis: int = 0) -> wl.Workload:
    rng = np.random.default_rng(11)
    if kind == "1d":
        w = wl.harmonic_1d()
        w = dataclasses.replace(w, levels=1)
    elif kind == "2d":
        w = wl.softcore_2d(n=16, levels=2)
        w = dataclasses.replace(w, nt=4)
    elif kind == "3d":
        w = wl.hydrogen_3d(n=8, nsteps=5, ncomp=3, sub=2)
        w = dataclasses.replace(w, levels=2)
    else:   # wide 4 x 4 x 4 subvolumes on a grid whose axes differ in extent and spacing
        w = wl.hydrogen_3d(n=8, nsteps=5, ncomp=3, sub=4)
        w = dataclasses.replace(w, n=(16, 8, 8), h=(0.3, 0.45, 0.25), levels=2)
    T = 5 * w.dt
    pulse = wl.Pulse(amp=list(rng.normal(0.0, 0.4, 3)), omega=[1.3, 2.1, 0.7], t_center=[0.0, T / 2, T],
                     sigma=[T / 2, T / 3, 0.0], axis=axis)
    return dataclasses.replace(w, pulse=pulse)


def run_forward(w, precision, psi0, nsteps, ckpt):
    ctx = gpu_context(w, precision=precision, tol=1e-22, max_cycles=80, ckpt_every=ckpt)
    psi = psi0.copy()
    ctx.step(psi, nsteps, 0.0)
    return ctx, psi


@pytest.mark.parametrize("kind,precision,trial,axis", [("1d", 0, 0, 0), ("2d", 0, 0, 0), ("2d", 1, 0, 0),
                                                      ("3d", 0, 0, 0), ("2d", 0, 3, 0), ("3d", 1, 3, 0),
                                                      ("2d", 0, 0, 1), ("3d_wide", 0, 0, 2)])
def test_backward_matches_oracle_adjoint(kind, precision, trial, axis):
    """The last two: the laser (and the dipole objective) along y, and along z on anisotropic wide
    subvolumes (cases where the coupling axis changes the gradient by 5-15%)."""
    w = dataclasses.replace(pulsed(kind, axis), trial=trial)
    nsteps, ckpt = 5, 2          # segments of 2, 2, 1 steps
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    ctx, psiT = run_forward(w, precision, psi0, nsteps, ckpt)
    _, dJ = adjoint.dipole_objective(prob, psiT)
    dpsi0 = np.zeros_like(psi0)
    g = ctx.backward(dJ, w.pulse.ncomp, dpsi0)
    g_ref, lam_ref = adjoint.gradients(prob, psi0, nsteps)
    assert rel_l2(g, g_ref) < 1e-8, (g, g_ref)
    assert rel_l2(dpsi0, lam_ref) < 1e-8


def test_backward_matches_finite_differences_of_the_gpu_forward():
    w = pulsed("2d")
    nsteps = 4
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    ctx, psiT = run_forward(w, 0, psi0, nsteps, 3)
    _, dJ = adjoint.dipole_objective(prob, psiT)
    g = ctx.backward(dJ, w.pulse.ncomp)
    eps = 1e-4
    fd = np.zeros(w.pulse.ncomp)
    for j in range(w.pulse.ncomp):
        vals = []
        for sgn in (1, -1):
            amp = list(w.pulse.amp)
            amp[j] += sgn * eps
            w2 = dataclasses.replace(w, pulse=dataclasses.replace(w.pulse, amp=amp))
            _, pT = run_forward(w2, 0, psi0, nsteps, 0)
            vals.append(system.dipole(prob, pT))
        fd[j] = (vals[0] - vals[1]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(fd)))


def test_backward_requires_a_recorded_forward():
    from paper_1111_4363_gb300 import binding as B
    w = pulsed("1d")
    ctx = gpu_context(w)
    with pytest.raises(B.LeastActionError) as e:
        ctx.backward(np.zeros(w.npoints, dtype=np.complex128), w.pulse.ncomp)
    assert e.value.status == B.LA_ESTATE


def test_autograd_function_gradients():
    """Gradients through torch.autograd (dipole objective written in torch) equal the oracle's."""
    import torch
    from paper_1111_4363_gb300 import autograd as A
    w = pulsed("2d")
    nsteps = 3
    prob = system.Problem.from_workload(w)
    psi0_np = wl.initial_state(w).ravel()
    ctx = gpu_context(w, tol=1e-22, max_cycles=80, ckpt_every=2)
    V0 = torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda")
    amp = torch.tensor(w.pulse.amp, dtype=torch.float64, requires_grad=True)
    psi0 = torch.from_numpy(psi0_np.copy()).cuda().requires_grad_(True)
    psiT = A.propagate(ctx, V0, w.pulse, amp, psi0, nsteps)
    x = torch.from_numpy(prob.xlaser).cuda()
    J = prob.vol * (x * psiT.abs() ** 2).sum()
    J.backward()
    g_ref, lam_ref = adjoint.gradients(prob, psi0_np, nsteps)
    assert rel_l2(amp.grad.numpy(), g_ref) < 1e-8
    assert rel_l2(psi0.grad.cpu().numpy(), 2 * lam_ref) < 1e-8


@pytest.mark.parametrize("kind,precision", [("2d", 0), ("3d", 1)])
def test_factor_cache_gives_identical_gradients(kind, precision):
    """cache_factors reuses the recomputed segment's factors in the adjoint relaxation: same numbers."""
    w = dataclasses.replace(pulsed(kind), trial=3)
    nsteps, ckpt = 5, 2
    psi0 = wl.initial_state(w).ravel()
    prob = system.Problem.from_workload(w)
    out = []
    for cache in (0, 1):
        ctx = gpu_context(w, precision=precision, ckpt_every=ckpt, cache_factors=cache)
        psi = psi0.copy()
        ctx.step(psi, nsteps, 0.0)
        _, dJ = adjoint.dipole_objective(prob, psi)
        dpsi0 = np.zeros_like(psi0)
        out.append((ctx.backward(dJ, w.pulse.ncomp, dpsi0), dpsi0))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
