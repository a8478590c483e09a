"""Legendre time basis and per-step time matrices (oracle; test infrastructure only).

Each time step [t0, t0+dt] is mapped to tau in [-1, 1], t = t0 + (tau+1) dt/2.
The time functions are Legendre polynomials P_0..P_K (Sec. IV uses Legendre
polynomials, whose overlaps are 2 delta_nm/(2n+1)).

Initial condition (Sec. I, Lagrange-multiplier paragraph): phi(x, t0) = psi0
fixes C_0 = psi0 - sum_{n>=1} (-1)^n C_n.  The free trial functions are then
b_n = P_n - (-1)^n P_0, n = 1..K, which vanish at t0, and eliminating the
multipliers leaves the stationarity rows tested against the same b_m.

Matrices (m, n = 1..K; m indexes the test function, n the trial function):
  Ub[m,n]  = (dt/2) int b_m b_n dtau             (U of Sec. I in the b basis)
  Qb[m,n]  =        int b_m (d b_n/dtau) dtau    (Q of Sec. I; dt cancels between d/dt and dt)
  Ub0[m]   = (dt/2) int b_m P_0 dtau             (coupling of the psi0 P_0 part)
  Eb[m,n]  = (dt/2) int b_m b_n E(t(tau)) dtau   (time part of V_ijnm for the dipole term)
  Eb0[m]   = (dt/2) int b_m P_0 E(t(tau)) dtau
All are computed here by Gauss-Legendre quadrature (the plain definition of the
integrals); the tests compare them with the paper's closed forms.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def legendre_P(nmax: int, tau: np.ndarray) -> np.ndarray:
    """Rows n = 0..nmax of P_n(tau)."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.empty((nmax + 1,) + tau.shape)
    for n in range(nmax + 1):
        coef = np.zeros(n + 1)
        coef[n] = 1.0
        out[n] = npleg.legval(tau, coef)
    return out


def legendre_dP(nmax: int, tau: np.ndarray) -> np.ndarray:
    """Rows n = 0..nmax of dP_n/dtau."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.empty((nmax + 1,) + tau.shape)
    for n in range(nmax + 1):
        coef = np.zeros(n + 1)
        coef[n] = 1.0
        out[n] = npleg.legval(tau, npleg.legder(coef)) if n > 0 else 0.0
    return out


def b_functions(K: int, tau: np.ndarray):
    """b_n(tau) and b_n'(tau) for n = 1..K (row n-1)."""
    P = legendre_P(K, tau)
    dP = legendre_dP(K, tau)
    sign = np.array([(-1.0) ** n for n in range(1, K + 1)])
    b = P[1:] - sign[:, None] * P[0][None, :]
    db = dP[1:]
    return b, db


def pulse_field(pulse, t: np.ndarray) -> np.ndarray:
    """E(t) = sum_k amp_k env_k(t) sin(omega_k t); env = exp(-((t-tc)/sigma)^2) for sigma > 0, else 1."""
    t = np.asarray(t, dtype=np.float64)
    e = np.zeros_like(t)
    if pulse is None:
        return e
    for a, w, tc, s in zip(pulse.amp, pulse.omega, pulse.t_center, pulse.sigma):
        env = np.exp(-((t - tc) / s) ** 2) if s > 0 else 1.0
        e = e + a * env * np.sin(w * t)
    return e


def pulse_component_field(pulse, k: int, t: np.ndarray) -> np.ndarray:
    """Field of component k with unit amplitude (the derivative of E(t) w.r.t. amp_k)."""
    t = np.asarray(t, dtype=np.float64)
    w, tc, s = pulse.omega[k], pulse.t_center[k], pulse.sigma[k]
    env = np.exp(-((t - tc) / s) ** 2) if s > 0 else 1.0
    return env * np.sin(w * t)


def static_matrices(K: int, dt: float, nquad: int | None = None):
    """(Ub, Qb, Ub0) of the b basis by Gauss-Legendre quadrature."""
    q = nquad if nquad is not None else K + 8
    tau, wq = npleg.leggauss(q)
    b, db = b_functions(K, tau)
    Ub = 0.5 * dt * (b * wq) @ b.T
    Qb = (b * wq) @ db.T
    Ub0 = 0.5 * dt * (b * wq) @ np.ones_like(tau)
    return Ub, Qb, Ub0


def field_matrices(K: int, dt: float, t0: float, field, nquad: int | None = None):
    """(Eb, Eb0) for a scalar field function field(t), by Gauss-Legendre quadrature with K+8 nodes."""
    q = nquad if nquad is not None else K + 8
    tau, wq = npleg.leggauss(q)
    b, _ = b_functions(K, tau)
    t = t0 + 0.5 * (tau + 1.0) * dt
    e = field(t)
    Eb = 0.5 * dt * (b * (wq * e)) @ b.T
    Eb0 = 0.5 * dt * (b * (wq * e)) @ np.ones_like(tau)
    return Eb, Eb0


def end_values(K: int) -> np.ndarray:
    """b_n(tau = +1) = 1 - (-1)^n: the weights that give phi(t0+dt) from the free coefficients."""
    return np.array([1.0 - (-1.0) ** n for n in range(1, K + 1)])
