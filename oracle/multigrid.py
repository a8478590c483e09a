"""Multigrid V-cycle for the least-action normal equations (oracle; test infrastructure only).

Sec. III: with an interpolation I from a coarse to a fine level and the
projection P = I^T, the coarse problem of A x = b is (P A P^T)(P x) = P b, and a
fine-level correction is delta x ~ I (P A P^T)^{-1} P r (Eqs. residual_rough,
correction_fine); recursion over levels gives the V-cycle.

Readings: A is the Hermitian normal matrix G = M^dagger W M (so the coarse
correction minimises the residual norm N over the coarse space), I is
cell-centred 2:1 linear interpolation per axis with zero Dirichlet ghosts
(weights 3/4, 1/4), acting on space only (the K time functions are kept), and
the coarsest level is relaxed ``coarse_sweeps`` times instead of a direct
factorisation.  Cycle shape V(nu1, nu2) on the finest level; the Galerkin levels
above the coarsest use (nu1, nu2) too, or ``coarse_nu`` = (nu1c, nu2c) when
given.  A single level means nu1 + nu2 sweeps per cycle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import relax, system


def interpolation_1d(nc: int) -> sp.csr_matrix:
    """Fine (2 nc) x coarse (nc): fine 2J <- 3/4 c_J + 1/4 c_{J-1}, fine 2J+1 <- 3/4 c_J + 1/4 c_{J+1}."""
    rows, cols, vals = [], [], []
    for J in range(nc):
        for fi, nb in ((2 * J, J - 1), (2 * J + 1, J + 1)):
            rows.append(fi); cols.append(J); vals.append(0.75)
            if 0 <= nb < nc:
                rows.append(fi); cols.append(nb); vals.append(0.25)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc, nc))


def interpolation(coarse_shape, K: int) -> sp.csr_matrix:
    """Tensor-product spatial interpolation, identity on the K time functions."""
    mats = [interpolation_1d(n) for n in coarse_shape]
    I = mats[0]
    for m in mats[1:]:
        I = sp.kron(I, m, format="csr")
    return sp.kron(I, sp.identity(K), format="csr")


class Hierarchy:
    """Levels 0 (finest) .. L-1, each with its Galerkin operator and block relaxation."""

    def __init__(self, G0, shape0, K, sub, levels, nu1=1, nu2=1, coarse_sweeps=2, coarse_sub=None, coarse_nu=None):
        self.K, self.L = K, levels
        self.nu1, self.nu2, self.coarse_sweeps = nu1, nu2, coarse_sweeps
        self.coarse_nu = (nu1, nu2) if coarse_nu is None else tuple(coarse_nu)
        self.shapes = [tuple(shape0)]
        self.G = [G0.tocsr()]
        self.I = []                    # I[l]: level l+1 -> level l
        for l in range(1, levels):
            fine = self.shapes[-1]
            if any(n % 2 for n in fine):
                raise ValueError("every level must have an even number of points per axis")
            coarse = tuple(n // 2 for n in fine)
            Il = interpolation(coarse, K)
            self.I.append(Il)
            self.G.append((Il.T @ self.G[-1] @ Il).tocsr())
            self.shapes.append(coarse)
        # the finest level uses ``sub``; Galerkin levels use ``coarse_sub`` when given
        subs = [sub] + [coarse_sub if coarse_sub is not None else sub] * (levels - 1)
        self.relax = [relax.BlockRelaxation(G, s, sb, K) for G, s, sb in zip(self.G, self.shapes, subs)]

    def vcycle(self, l, x, g, after_colour=None):
        """Improve x for G_l x = g by one V(nu1, nu2) cycle rooted at level l."""
        hook = after_colour if l == 0 else None
        if self.L == 1:
            for _ in range(self.nu1 + self.nu2):
                self.relax[0].sweep(x, g, hook)
            return
        if l == self.L - 1:
            for _ in range(self.coarse_sweeps):
                self.relax[l].sweep(x, g)
            return
        nu1, nu2 = (self.nu1, self.nu2) if l == 0 else self.coarse_nu
        for _ in range(nu1):
            self.relax[l].sweep(x, g, hook)
        s = g - self.G[l] @ x
        gc = self.I[l].T @ s
        xc = np.zeros_like(gc)
        self.vcycle(l + 1, xc, gc)
        x += self.I[l] @ xc
        if after_colour is not None and l == 0:
            after_colour(-1)           # -1 marks "after the coarse-grid correction"
        for _ in range(nu2):
            self.relax[l].sweep(x, g, hook)


def solve_step(M, f, W, shape, K, sub, levels, nu1, nu2, coarse_sweeps, ncycles=None, tol=None,
               max_cycles=200, after_colour=None, c0=None, coarse_sub=None, coarse_nu=None):
    """Relax from c0 (default 0) by V-cycles; returns (c, history of N, cycles run).

    Exactly ``ncycles`` cycles when given, else until N(c)/N(0) <= tol or ``max_cycles``.
    """
    G0 = (M.conj().T @ W @ M).tocsr()
    g0 = M.conj().T @ (W @ f)
    hier = Hierarchy(G0, shape, K, sub, levels, nu1, nu2, coarse_sweeps, coarse_sub, coarse_nu)
    c = np.zeros(M.shape[1], dtype=np.complex128) if c0 is None else c0.astype(np.complex128).copy()
    N0 = system.action_norm(f, W)
    hist = [system.action_norm(system.residual(M, f, c), W)]
    cyc = 0
    while True:
        if ncycles is not None and cyc >= ncycles:
            break
        if ncycles is None and (hist[-1] <= tol * N0 or cyc >= max_cycles):
            break
        hier.vcycle(0, c, g0, after_colour)
        cyc += 1
        hist.append(system.action_norm(system.residual(M, f, c), W))
    return c, hist, cyc, hier
