"""The least-action linear system of one time step (oracle; test infrastructure only).

Spatial discretisation (a reading; the paper's method is basis-generic and its
worked basis is Legendre elements): finite differences on a uniform grid, which
is the basis chi_p with overlap O = h^d I, Hamiltonian matrix H = h^d (T + V0)
with T = -1/2 * (second-order central Laplacian, Dirichlet walls), and the
time-dependent potential E(t) x_axis (dipole coupling).

Stationarity (Eq. stationaryphase), with the initial condition imposed by
eliminating the Lagrange multipliers (Sec. I), tested against chi_q b_m:
  (M c)[q,m] = h^d sum_n ( i Qb[m,n] c[q,n] - Ub[m,n] (H c)[q,n] - x_q Eb[m,n] c[q,n] )
  f[q,m]     = h^d ( Ub0[m] (H psi0)[q] + x_q Eb0[m] psi0[q] )
so that M c = f, and the action residual (Eq. actionresidual) of a trial c is
r = f - M c.  The residual norm (Eq. residnorm) is N = r^dagger W r.

Weight W (a reading).  Eq. residnorm writes N = r O U r*, the L2 norm of a
function whose expansion coefficients are r.  The residual of Eq. actionresidual
holds projections onto the test functions, whose coefficients in the test space
are (O (x) Ub)^{-1} r; the norm of that residual function is therefore
    "dual"     W = (O (x) Ub)^{-1} = h^{-d} (I (x) Ub^{-1})     (default)
which is also the only choice that does not depend on which basis of the test
space is used.  Two alternatives are kept for comparison:
    "literal"  W = O (x) Ub = h^d (I (x) Ub)
    "identity" W = I.
The minimiser (M c = f) is the same for every W; only N and the relaxation path change.

Unknown ordering: index = p*K + (m-1), point-major (kron(spatial, time)).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1111_4363_gb300 import workloads as wl
from . import timebasis as tb


@dataclasses.dataclass
class Problem:
    dim: int
    shape: tuple          # numpy shape (slowest first)
    h: tuple              # spacing per numpy axis (slowest first)
    K: int
    dt: float
    V0: np.ndarray        # flat, real
    xlaser: np.ndarray    # flat, real: the dipole coordinate
    pulse: object         # workloads.Pulse or None

    @property
    def npoints(self) -> int:
        return int(np.prod(self.shape))

    @property
    def vol(self) -> float:
        """h^d, the FD overlap weight O_pp."""
        return float(np.prod(self.h))

    @staticmethod
    def from_workload(w: wl.Workload) -> "Problem":
        shape = w.shape
        h = tuple(w.h[a] for a in reversed(range(w.dim)))
        return Problem(dim=w.dim, shape=shape, h=h, K=w.nt, dt=w.dt,
                       V0=wl.potential(w).ravel().astype(np.float64),
                       xlaser=wl.laser_coordinate(w).ravel().astype(np.float64),
                       pulse=w.pulse)

    def field(self, t):
        return tb.pulse_field(self.pulse, t)


def second_difference_1d(n: int, h: float) -> sp.csr_matrix:
    """(u[k+1] - 2u[k] + u[k-1]) / h^2 with zero Dirichlet ghosts."""
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr") / (h * h)


def laplacian(shape, h) -> sp.csr_matrix:
    """Sum over axes of the 1D second difference (3/5/7-point stencil in 1/2/3 D)."""
    d = len(shape)
    L = sp.csr_matrix((int(np.prod(shape)),) * 2)
    for a in range(d):
        mats = [sp.identity(shape[b], format="csr") for b in range(d)]
        mats[a] = second_difference_1d(shape[a], h[a])
        term = mats[0]
        for m in mats[1:]:
            term = sp.kron(term, m, format="csr")
        L = L + term
    return L.tocsr()


def kinetic(prob: Problem) -> sp.csr_matrix:
    """T = -1/(2m) Laplacian, m = 1."""
    return (-0.5 * laplacian(prob.shape, prob.h)).tocsr()


def hamiltonian_operator(prob: Problem) -> sp.csr_matrix:
    """T + diag(V0): the static part of H per unit overlap (H_ij = h^d (T + V0)_ij)."""
    return (kinetic(prob) + sp.diags(prob.V0)).tocsr()


def time_matrices(prob: Problem, t0: float):
    Ub, Qb, Ub0 = tb.static_matrices(prob.K, prob.dt)
    Eb, Eb0 = tb.field_matrices(prob.K, prob.dt, t0, prob.field)
    return Ub, Qb, Ub0, Eb, Eb0


def weight_matrix(prob: Problem, Ub: np.ndarray, weight: str = "dual"):
    I = sp.identity(prob.npoints, format="csr")
    if weight == "dual":
        return (sp.kron(I, np.linalg.inv(Ub)) / prob.vol).tocsr()
    if weight == "literal":
        return (prob.vol * sp.kron(I, Ub)).tocsr()
    if weight == "identity":
        return sp.identity(prob.npoints * prob.K, format="csr")
    raise ValueError(weight)


def assemble(prob: Problem, t0: float, psi0: np.ndarray, weight: str = "dual"):
    """(M, f, W) of the step starting at t0 with initial state psi0 (flat, complex)."""
    Ub, Qb, Ub0, Eb, Eb0 = time_matrices(prob, t0)
    Hs = hamiltonian_operator(prob)
    I = sp.identity(prob.npoints, format="csr")
    X = sp.diags(prob.xlaser)
    v = prob.vol
    M = v * (sp.kron(I, 1j * Qb) - sp.kron(Hs, Ub) - sp.kron(X, Eb))
    M = M.tocsr()
    Hpsi = Hs @ psi0
    f = v * (np.kron(Hpsi, Ub0) + np.kron(prob.xlaser * psi0, Eb0))
    W = weight_matrix(prob, Ub, weight)
    return M, f.astype(np.complex128), W


def hamiltonian_row(prob: Problem, q: int):
    """Column indices and values of row q of T + diag(V0) (the 3/5/7-point stencil, Dirichlet walls)."""
    coord = np.unravel_index(q, prob.shape)
    cols, vals = [q], [float(prob.V0[q])]
    for a in range(prob.dim):
        w = -0.5 / (prob.h[a] * prob.h[a])
        vals[0] += -2.0 * w                       # -1/2 * (-2 / h^2)
        for step in (-1, 1):
            nb = list(coord)
            nb[a] += step
            if 0 <= nb[a] < prob.shape[a]:
                cols.append(int(np.ravel_multi_index(tuple(nb), prob.shape)))
                vals.append(w)
    return np.array(cols, dtype=np.int64), np.array(vals)


def residual_at(prob: Problem, t0: float, psi0: np.ndarray, c: np.ndarray, points) -> np.ndarray:
    """Rows of r = f - M c at the listed points, shape (len(points), K), from the stencil form of the
    same system as `assemble` (for grids too large to assemble):
      (M c)[q,m] = h^d sum_n ( i Qb[m,n] c[q,n] - Ub[m,n] (H c)[q,n] - x_q Eb[m,n] c[q,n] ),
      f[q,m]     = h^d ( Ub0[m] (H psi0)[q] + x_q Eb0[m] psi0[q] )."""
    Ub, Qb, Ub0, Eb, Eb0 = time_matrices(prob, t0)
    K, v = prob.K, prob.vol
    C = np.asarray(c).reshape(-1, K)
    out = np.empty((len(points), K), dtype=np.complex128)
    for j, q in enumerate(points):
        cols, vals = hamiltonian_row(prob, int(q))
        Hc = vals @ C[cols]                       # (H c)[q, :]
        Hpsi = vals @ psi0[cols]
        xq = prob.xlaser[q]
        f = v * (Ub0 * Hpsi + xq * Eb0 * psi0[q])
        Mc = v * (1j * (Qb @ C[q]) - Ub @ Hc - xq * (Eb @ C[q]))
        out[j] = f - Mc
    return out


def residual(M, f, c):
    """Action residual r = f - M c (Eq. actionresidual with the initial condition moved to f)."""
    return f - M @ c


def action_norm(r, W) -> float:
    """N = r^dagger W r (Eq. residnorm)."""
    return float(np.real(np.vdot(r, W @ r)))


def direct_solve(M, f):
    """The minimum-action coefficients of the step: M c = f by sparse LU."""
    return spla.splu(M.tocsc()).solve(f)


def advance(psi0: np.ndarray, c: np.ndarray, K: int) -> np.ndarray:
    """phi(t0+dt) = psi0 + sum_n c_n b_n(+1) = psi0 + 2 sum_{n odd} c_n (P_n(1) = 1, P_n(-1) = (-1)^n)."""
    C = c.reshape(-1, K)
    return psi0 + C @ tb.end_values(K)


def dipole(prob: Problem, psi: np.ndarray) -> float:
    """<x_axis> = h^d sum_p x_p |psi_p|^2 (unnormalised expectation)."""
    return float(prob.vol * np.sum(prob.xlaser * np.abs(psi) ** 2))
