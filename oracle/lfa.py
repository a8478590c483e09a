"""Convergence maps of one relaxation step in the paper's Legendre-element basis (Sec. IV and
Sec. V, the plane-wave experiment; oracle, test infrastructure only).

One element is the box y, tau in [-1, 1] with Legendre functions P_i(y) (i < Nx) and P_n(tau)
(n < Nt); coefficients C[i, n] are stored at i*Nt + n.  The dimensionless least-action rows
(Eq. leastaction_dimensionless), row = test (j, m), column = trial (i, n):
    A[(j,m),(i,n)] = i O[j,i] Qt[m,n] - 2 kappa K[j,i] U[m,n] - nu O[j,i] U[m,n]
with O, U the Legendre overlaps, Qt[m, n] = int P_m P_n' (derivative on the trial function) and
K[j, i] = int P_j (-1/2 P_i'') (kinetic element, test j, trial i; the closed form of
Eq. Tmatelt as printed).  Residual r = -A C (Eq. actionresidual), norm N = r^H (O x U) r
(Eq. residnorm as printed), action S = C^H A C.

A relaxation over a volume of elements solves the correction problem (Eq. leastaction_correction)
with delta = 0 at t0 in every element (Eq. ic_correction), on the volume's outer boundary
(Eqs. bc1_correction, bc2_correction) and continuity across its inner element boundaries.  The
constraints enter through Lagrange multipliers: A delta + B^T lambda = r, B delta = 0.  Its delta
part is delta = Z (Z^T A Z)^{-1} Z^T r with Z an orthonormal basis of the null space of B, which
stays well defined where constraints repeat (the initial-time and boundary conditions meet at the
two bottom corners of an element, so an element's Nx + 2 Nt conditions have rank Nx + 2 Nt - 2).

Methods (Sec. V): "one" relaxes one element; "two" relaxes two elements [-1, 0], [0, 1] at once;
"transfer" takes the two-element residual to the parent element (Eq. residual_rough: r_c = P r,
A_c = P A I), relaxes there, interpolates the correction back (Eq. correction_fine) and then relaxes
each child element separately.  Both children use the listed (kappa, nu) in their own coordinates.

Trial function f = exp(i (k x + w t)) on x, t in [-1, 1]: one element takes the L2 projection; two
elements take the L2 projection constrained to be continuous at x = 0 (Eq. continuityprojection,
read in the L2 metric of the element bases).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg

from . import legendre_elements as le
from .timebasis import legendre_P, legendre_dP

KAPPA_NU = [(0.0, 0.0), (0.1, 0.0), (1.0, 0.0), (10.0, 0.0), (0.0, 1.0), (0.0, -1.0), (1.0, 1.0), (1.0, -1.0)]


def element_matrices(nx: int, nt: int):
    """O (nx x nx), U (nt x nt), Qt (nt x nt), K (nx x nx) by Gauss-Legendre quadrature."""
    y, w = npleg.leggauss(max(nx, nt) + 4)
    Px, Pt = legendre_P(nx - 1, y), legendre_P(nt - 1, y)
    O = (Px * w) @ Px.T
    U = (Pt * w) @ Pt.T
    Qt = (Pt * w) @ legendre_dP(nt - 1, y).T          # [m, n] = int P_m P_n'
    K = le.kinetic(nx - 1)                             # [j, i] = int P_j (-1/2 P_i'')
    return O, U, Qt, K


def element_operator(nx, nt, kappa, nu):
    O, U, Qt, K = element_matrices(nx, nt)
    return 1j * np.kron(O, Qt) - 2.0 * kappa * np.kron(K, U) - nu * np.kron(O, U)


def weight(nx, nt, nel):
    O, U, _, _ = element_matrices(nx, nt)
    return np.kron(np.eye(nel), np.kron(O, U))


def constraints(nx, nt, nel, left=True, right=True, initial=True, continuity=True):
    """Rows of B for nel elements side by side (element e holds x-coordinates left to right)."""
    n = nx * nt
    rows = []
    sgn_i = (-1.0) ** np.arange(nx)
    sgn_n = (-1.0) ** np.arange(nt)
    for e in range(nel if initial else 0):
        for i in range(nx):                            # value at tau = -1
            r = np.zeros(nel * n)
            r[e * n + i * nt: e * n + (i + 1) * nt] = sgn_n
            rows.append(r)
    for m in range(nt):
        if left:                                       # value at the left end of element 0
            r = np.zeros(nel * n)
            r[m: n: nt] = sgn_i
            rows.append(r)
        if right:                                      # value at the right end of the last element
            r = np.zeros(nel * n)
            r[(nel - 1) * n + m: nel * n: nt] = 1.0
            rows.append(r)
        for e in range(nel - 1 if continuity else 0):  # right end of e equals left end of e + 1
            r = np.zeros(nel * n)
            r[e * n + m: (e + 1) * n: nt] = 1.0
            r[(e + 1) * n + m: (e + 2) * n: nt] = -sgn_i
            rows.append(r)
    return np.array(rows).reshape(-1, nel * n)


def null_space(B, tol=1e-12):
    if B.shape[0] == 0:
        return np.eye(B.shape[1])
    _, s, vh = np.linalg.svd(B)
    rank = int(np.sum(s > tol * s[0]))
    return vh[rank:].conj().T


def constrained_solve(A, B, r, solver="null"):
    """delta with A delta + B^T lambda = r, B delta = 0.  solver "null": on the null space of B;
    "bordered": least squares (minimum norm) on the bordered system [A B^T; B 0], a second
    backward-stable route used to gauge how much rounding the problem itself amplifies."""
    if solver == "null":
        Z = null_space(B)
        return Z @ np.linalg.solve(Z.T @ A @ Z, Z.T @ r)
    nc = B.shape[0]
    kkt = np.block([[A, B.T.astype(complex)], [B.astype(complex), np.zeros((nc, nc))]])
    return np.linalg.lstsq(kkt, np.concatenate([r, np.zeros(nc)]), rcond=None)[0][:A.shape[0]]


def relax(A, B, C, solver="null"):
    """C + delta for the constrained correction problem with residual r = -A C."""
    return C + constrained_solve(A, B, -A @ C, solver)


def plane_wave_overlaps(nx, nt, nel, k, w, nquad=48):
    """fhat[e, i, n] = int int exp(i (k x(y) + w tau)) P_i(y) P_n(tau) dy dtau over element e."""
    y, wq = npleg.leggauss(nquad)
    Px, Pt = legendre_P(nx - 1, y), legendre_P(nt - 1, y)
    bt = (Pt * wq) @ np.exp(1j * w * y)
    out = []
    for e in range(nel):
        x = y if nel == 1 else 0.5 * (y - 1.0) + e   # children: x = (y - 1)/2 and (y + 1)/2
        ax = (Px * wq) @ np.exp(1j * k * x)
        out.append(np.outer(ax, bt).ravel())
    return np.concatenate(out)


def project(nx, nt, nel, fhat):
    """L2 projection; with two elements constrained to be continuous at the shared boundary."""
    W = weight(nx, nt, nel)
    if nel == 1:
        return fhat / np.diag(W)
    B = constraints(nx, nt, nel, left=False, right=False, initial=False, continuity=True)
    nc = B.shape[0]
    kkt = np.block([[W, B.T], [B, np.zeros((nc, nc))]])
    sol = np.linalg.solve(kkt, np.concatenate([fhat, np.zeros(nc)]))
    return sol[:W.shape[0]]


def measures(A, W, C):
    r = -A @ C
    return float(np.real(r.conj() @ (W @ r))), complex(C.conj() @ (A @ C))


def parent_transfers(nx, nt):
    """(I, P) between a parent element and its two children, acting on space only (the time basis is
    shared): I gives the children's coefficients of parent functions, P projects back (Sec. IV)."""
    return np.kron(le.interpolation(nx - 1), np.eye(nt)), np.kron(le.projection(nx - 1), np.eye(nt))


def coarse_correction(A2, C, nx, nt, solver="null"):
    """C + I dc, where dc solves the projected problem (P A2 I) dc = P r on the parent element under
    its own conditions, r = -A2 C (Eq. residual_rough; the correction interpolated back by
    Eq. correction_fine)."""
    I, P = parent_transfers(nx, nt)
    r = -A2 @ C
    return C + I @ constrained_solve(P @ A2 @ I, constraints(nx, nt, 1), P @ r, solver)


def relax_method(method, nx, nt, kappa, nu, C, solver="null"):
    """One relaxation of the trial coefficients C by the given method."""
    A1 = element_operator(nx, nt, kappa, nu)
    if method == "one":
        return relax(A1, constraints(nx, nt, 1), C, solver)
    A2 = np.kron(np.eye(2), A1)
    if method == "two":
        return relax(A2, constraints(nx, nt, 2), C, solver)
    assert method == "transfer"
    # coarse correction on the parent element, then each child element on its own (delta = 0 on both
    # of its ends)
    C = coarse_correction(A2, C, nx, nt, solver)
    n = nx * nt
    B1 = constraints(nx, nt, 1)
    out = C.copy()
    for e in range(2):
        out[e * n:(e + 1) * n] = relax(A1, B1, C[e * n:(e + 1) * n], solver)
    return out


def ratio_map(method, nx, nt, kappa, nu, ks, ws, solver="null"):
    """log10 N_after / N_before and log10 |S_after| / |S_before| on the (w, k) grid [len(ws), len(ks)]."""
    nel = 1 if method == "one" else 2
    A1 = element_operator(nx, nt, kappa, nu)
    A = A1 if nel == 1 else np.kron(np.eye(2), A1)
    W = weight(nx, nt, nel)
    lrN = np.empty((len(ws), len(ks)))
    lrS = np.empty((len(ws), len(ks)))
    for a, w in enumerate(ws):
        for b, k in enumerate(ks):
            C = project(nx, nt, nel, plane_wave_overlaps(nx, nt, nel, k, w))
            N0, S0 = measures(A, W, C)
            N1, S1 = measures(A, W, relax_method(method, nx, nt, kappa, nu, C, solver))
            lrN[a, b] = np.log10(N1 / N0)
            lrS[a, b] = np.log10(abs(S1) / abs(S0))
    return lrN, lrS
