"""Discrete adjoint of a least-action propagation (oracle; test infrastructure only).

Forward (Sec. I): each step solves M_k c_k = f_k with f_k = F_k psi_k, F_k psi =
h^d [ Ub0 (x) (H psi) + Eb0(t_k) (x) (x psi) ], and advances psi_{k+1} = psi_k + B c_k,
(B c)_p = sum_n b_n(1) c_pn.  Both M_k and F_k depend on the pulse amplitudes a_j
through Eb(t_k) = sum_j a_j Eb^(j)(t_k) and Eb0(t_k) = sum_j a_j Eb0^(j)(t_k).

For a real objective J(psi_T) with lambda_T = dJ/dpsi_T^* (conjugate Wirtinger derivative):
    mu_k      = M_k^{-dagger} B^T lambda_{k+1}                  (adjoint solve)
    lambda_k  = lambda_{k+1} + F_k^T mu_k                        (F_k is real)
    dJ/da_j   = sum_k 2 Re mu_k^dagger ( dF_k/da_j psi_k - dM_k/da_j c_k )
              = sum_k 2 h^d Re sum_p x_p mu_k,p^dagger ( Eb0^(j) psi_k,p + Eb^(j) c_k,p )
and dJ/dpsi_0^* = lambda_0.  The exact solves make this the gradient of the discrete map.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import system, timebasis as tb


def forward(prob: system.Problem, psi0: np.ndarray, nsteps: int, t0: float = 0.0):
    """Direct-solve propagation; returns the states psi_0..psi_n and coefficients c_0..c_{n-1}."""
    psis, cs = [np.asarray(psi0, dtype=np.complex128).ravel().copy()], []
    for k in range(nsteps):
        M, f, _ = system.assemble(prob, t0 + k * prob.dt, psis[-1])
        c = system.direct_solve(M, f)
        cs.append(c)
        psis.append(system.advance(psis[-1], c, prob.K))
    return psis, cs


def dipole_objective(prob: system.Problem, psi: np.ndarray):
    """J = h^d sum_p x_p |psi_p|^2 and dJ/dpsi^* = h^d x psi."""
    return system.dipole(prob, psi), prob.vol * prob.xlaser * psi


def gradients(prob: system.Problem, psi0: np.ndarray, nsteps: int, t0: float = 0.0, lam_T=None):
    """(dJ/da_j for every pulse component, dJ/dpsi_0^*) for the dipole objective (or a given lambda_T)."""
    psis, cs = forward(prob, psi0, nsteps, t0)
    if lam_T is None:
        _, lam_T = dipole_objective(prob, psis[-1])
    lam = np.asarray(lam_T, dtype=np.complex128).copy()
    K, v, x = prob.K, prob.vol, prob.xlaser
    Ub, _, Ub0 = tb.static_matrices(K, prob.dt)
    Hs = system.hamiltonian_operator(prob)
    endv = tb.end_values(K)
    ncomp = prob.pulse.ncomp if prob.pulse is not None else 0
    grad = np.zeros(ncomp)
    for k in reversed(range(nsteps)):
        t = t0 + k * prob.dt
        M, f, _ = system.assemble(prob, t, psis[k])
        y = np.kron(lam, endv)                               # B^T lambda
        mu = spla.splu(M.conj().T.tocsc()).solve(y)
        Mu = mu.reshape(-1, K)
        C = cs[k].reshape(-1, K)
        for j in range(ncomp):
            field = lambda tt, j=j: tb.pulse_component_field(prob.pulse, j, tt)
            Ebj, Eb0j = tb.field_matrices(K, prob.dt, t, field)
            w = np.outer(psis[k], Eb0j) + C @ Ebj.T           # (Eb0^(j) psi + Eb^(j) c)_p,m
            grad[j] += 2.0 * v * np.real(np.sum(x[:, None] * np.conj(Mu) * w))
        Eb, Eb0 = tb.field_matrices(K, prob.dt, t, prob.field)
        lam = lam + v * (Hs @ (Mu @ Ub0) + x * (Mu @ Eb0))  # F_k^T mu
    return grad, lam


def finite_difference_gradient(prob: system.Problem, psi0, nsteps: int, eps: float = 1e-5, t0: float = 0.0):
    """Central differences of the dipole objective with respect to each pulse amplitude."""
    import copy
    g = np.zeros(prob.pulse.ncomp)
    for j in range(prob.pulse.ncomp):
        vals = []
        for sgn in (+1, -1):
            p2 = copy.deepcopy(prob)
            p2.pulse.amp = list(prob.pulse.amp)
            p2.pulse.amp[j] += sgn * eps
            psis, _ = forward(p2, psi0, nsteps, t0)
            vals.append(system.dipole(p2, psis[-1]))
        g[j] = (vals[0] - vals[1]) / (2 * eps)
    return g
