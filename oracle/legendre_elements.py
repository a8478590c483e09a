"""The paper's Legendre-element intergrid transfers (Sec. IV; oracle, test infrastructure only).

An element [-1, 1] with Legendre basis P_0..P_n is split into a left child
[-1, 0] and a right child [0, 1], each with its own Legendre basis in a local
coordinate y' in [-1, 1] (parent coordinate y = (y' -+ 1)/2).

  I^(L)[i, j] = int_{-1}^{1} P_i((y'-1)/2) P_j(y') dy'   (and (y'+1)/2 for the right child)

are the overlaps of each parent function with the child functions; dividing by
the child norms 2/(2j+1) gives the child expansion coefficients, so the parent
function P_i equals sum_j E^(s)[j, i] P_j on child s exactly.  The projection
back to the parent is the overlap-weighted transpose, normalised so that
projecting an interpolated function returns it (the paper's
(P^(L) + P^(R)) (I^(L) + I^(R)) = identity):
    P = (E^T O_f E)^{-1} E^T O_f,  E = [E^(L); E^(R)],  O_f = diag(O, O).
The garbled denominator of the paper's P formula is read as this normalisation.

Also the element kinetic matrix by quadrature (Eq. Tmatelt's first line):
    T[i, j] = 1/(2m) [ -P_i P_j' |_{-1}^{1} + int P_i' P_j' ].
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg

from .timebasis import legendre_P, legendre_dP


def overlap(nmax: int) -> np.ndarray:
    """O[n, n] = int P_n^2 = 2/(2n+1), computed by quadrature."""
    y, w = npleg.leggauss(nmax + 4)
    P = legendre_P(nmax, y)
    return (P * w) @ P.T


def child_overlaps(nmax: int):
    """(I_L, I_R): I_s[i, j] = int P_i(parent coordinate of y') P_j(y') dy'."""
    y, w = npleg.leggauss(nmax + 4)
    Pc = legendre_P(nmax, y)
    IL = (legendre_P(nmax, 0.5 * (y - 1.0)) * w) @ Pc.T
    IR = (legendre_P(nmax, 0.5 * (y + 1.0)) * w) @ Pc.T
    return IL, IR


def interpolation(nmax: int) -> np.ndarray:
    """E (2(n+1) x (n+1)): child coefficients (left block, then right block) of each parent function."""
    IL, IR = child_overlaps(nmax)
    norms = np.diag(overlap(nmax))
    return np.vstack([(IL / norms[None, :]).T, (IR / norms[None, :]).T])


def projection(nmax: int) -> np.ndarray:
    """P = (E^T O_f E)^{-1} E^T O_f."""
    E = interpolation(nmax)
    O = overlap(nmax)
    Of = np.block([[O, np.zeros_like(O)], [np.zeros_like(O), O]])
    return np.linalg.solve(E.T @ Of @ E, E.T @ Of)


def kinetic(nmax: int, mass: float = 1.0) -> np.ndarray:
    """T[i, j] = 1/(2m) [ -P_i(y) P_j'(y) |_{-1}^{1} + int P_i' P_j' ] by quadrature."""
    y, w = npleg.leggauss(nmax + 4)
    dP = legendre_dP(nmax, y)
    ends = np.array([-1.0, 1.0])
    Pe = legendre_P(nmax, ends)
    dPe = legendre_dP(nmax, ends)
    boundary = np.outer(Pe[:, 1], dPe[:, 1]) - np.outer(Pe[:, 0], dPe[:, 0])
    return (-boundary + (dP * w) @ dP.T) / (2.0 * mass)
