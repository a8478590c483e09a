"""Shared test helpers: build oracle problems and CUDA contexts for the same seeded workload."""
import dataclasses

import numpy as np

from oracle import system
from oracle.propagate import numpy_sub
from paper_1111_4363_gb300 import workloads as wl


def variant(w: wl.Workload, **kw) -> wl.Workload:
    return dataclasses.replace(w, **kw)


def ragged_2d(levels=2) -> wl.Workload:
    """30 x 22 points with 4 x 4 subvolumes: ragged last subvolume on both axes, on every level."""
    w = wl.softcore_2d(n=32, levels=levels)
    return variant(w, name="2d_ragged_30x22", n=(30, 22, 1))


def small_3d(levels=2) -> wl.Workload:
    w = wl.hydrogen_3d(n=8, nsteps=4, ncomp=4, sub=2)
    return variant(w, n=(8, 8, 6), levels=levels)


def oracle_system(w: wl.Workload, psi0, t0):
    prob = system.Problem.from_workload(w)
    M, f, W = system.assemble(prob, t0, psi0.ravel(), w.weight)
    return prob, M, f, W


def rel_l2(a, b) -> float:
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_context(w: wl.Workload, precision=0, **overrides):
    import torch
    from paper_1111_4363_gb300 import binding as B
    cfg = B.config_from_workload(w, precision=precision, **overrides)
    ctx = B.Context(cfg)
    V0 = torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda")
    ctx.set_hamiltonian(V0, w.pulse)
    return ctx


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


# extrapolation of the next step's coefficients from the last 1, 2, 3 converged ones (newest first)
TRIAL_WEIGHTS = {1: [1.0], 2: [2.0, -1.0], 3: [3.0, -3.0, 1.0]}


def oracle_trial_propagation(w, psi0, nsteps, trial, ncycles, t0=0.0):
    """nsteps steps of exactly ncycles V-cycles each (oracle), every step started from the
    extrapolated trial (or c = 0 where the trial's action is not below N(0))."""
    from oracle import multigrid, system
    from oracle.propagate import numpy_coarse_nu, numpy_coarse_sub, numpy_sub
    prob = system.Problem.from_workload(w)
    psi = psi0.astype(np.complex128).copy()
    hist = []
    for s in range(nsteps):
        M, f, W = system.assemble(prob, t0 + s * w.dt, psi, w.weight)
        c0 = None
        if trial > 0 and hist:
            q = min(len(hist), trial)
            cand = sum(a * h for a, h in zip(TRIAL_WEIGHTS[q], hist[::-1][:q]))
            if system.action_norm(system.residual(M, f, cand), W) < system.action_norm(f, W):
                c0 = cand
        c, _, _, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, numpy_sub(w), w.levels, w.nu1, w.nu2,
                                          w.coarse_sweeps, ncycles=ncycles, c0=c0, coarse_sub=numpy_coarse_sub(w),
                                          coarse_nu=numpy_coarse_nu(w))
        hist.append(c)
        psi = system.advance(psi, c, prob.K)
    return psi
