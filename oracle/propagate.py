"""Time stepping with the least-action propagator (oracle; test infrastructure only).

Each step minimises the action over [t0, t0+dt] with phi(t0) = psi(t0) (Sec. I);
the end value phi(t0+dt) is the next step's initial condition.
"""
from __future__ import annotations

import numpy as np

from paper_1111_4363_gb300 import workloads as wl
from . import multigrid, system


def numpy_sub(w: wl.Workload):
    return tuple(w.sub[a] for a in reversed(range(w.dim)))


def numpy_coarse_sub(w: wl.Workload):
    return None if w.coarse_sub is None else tuple(w.coarse_sub[a] for a in reversed(range(w.dim)))


def numpy_coarse_nu(w: wl.Workload):
    return None if getattr(w, "coarse_nu", None) is None else tuple(w.coarse_nu)


def step_direct(prob: system.Problem, psi0: np.ndarray, t0: float):
    M, f, W = system.assemble(prob, t0, psi0)
    c = system.direct_solve(M, f)
    return system.advance(psi0, c, prob.K), c


def step_relax(prob: system.Problem, w: wl.Workload, psi0: np.ndarray, t0: float, ncycles=None, tol=None):
    M, f, W = system.assemble(prob, t0, psi0, w.weight)
    c, hist, cyc, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, numpy_sub(w), w.levels, w.nu1, w.nu2,
                                           w.coarse_sweeps, ncycles=ncycles,
                                           tol=w.tol if tol is None else tol, max_cycles=w.max_cycles,
                                           coarse_sub=numpy_coarse_sub(w), coarse_nu=numpy_coarse_nu(w))
    return system.advance(psi0, c, prob.K), c, hist, cyc


def propagate(w: wl.Workload, nsteps: int | None = None, method: str = "direct", psi0=None, t0: float = 0.0):
    """Propagate ``nsteps`` steps; returns (psi, list of per-step cycle counts)."""
    prob = system.Problem.from_workload(w)
    psi = (wl.initial_state(w).ravel() if psi0 is None else np.asarray(psi0).ravel()).astype(np.complex128)
    n = w.nsteps if nsteps is None else nsteps
    cycles = []
    for k in range(n):
        t = t0 + k * w.dt
        if method == "direct":
            psi, _ = step_direct(prob, psi, t)
        else:
            psi, _, _, cyc = step_relax(prob, w, psi, t)
            cycles.append(cyc)
    return psi, cycles
