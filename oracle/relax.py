"""Subvolume relaxation (oracle; test infrastructure only).

Sec. II: the trial coefficients are improved by minimising, in each subvolume U,
the residual norm N with the coefficients outside U held fixed; relaxations of
subvolumes that do not interact are independent and may run in parallel.

Two local problems are kept.  The default (least squares, below) is the norm
argument of Sec. II.  The paper's own preconditioner form (Sec. II, last
paragraphs) is the square Dirichlet problem: find delta_U with
L_U delta_U = -L_U phi, delta = 0 on the boundary of U and at t0, i.e. in the
discrete system the rows of U's test functions and the columns of U's unknowns,
    M_UU delta_U = (f - M c)_U,
which the paper notes need not decrease the action (the Lagrange multipliers of
the boundary conditions make it a critical point, not a minimum).

Local problem (reading of Sec. II, the norm argument; the paper's own square
Dirichlet form is noted there to be non-monotone): with G = M^dagger W M the
Hermitian positive-definite normal matrix and g = M^dagger W f,
    delta_U = argmin N(c + E_U delta) = G_UU^{-1} (g - G c)_U,
i.e. exact block Gauss-Seidel on G c = g, which never increases N.

Colouring: G couples points up to two stencil radii apart, so the 2^d classes
"block index parity per axis" make same-colour subvolumes non-interacting
(G_UV = 0) whenever every subvolume spans at least two points per axis.  The
same-colour updates are therefore computed from one residual and applied
together, which equals applying them one after another.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla


def block_counts(shape, sub):
    """Subvolumes per numpy axis; the last block on an axis may be short (ragged tail)."""
    return tuple(-(-shape[a] // sub[a]) for a in range(len(shape)))


def subvolumes(shape, sub):
    """List of (colour, point indices) in block-lexicographic order (numpy axis order).

    ``sub`` is given per numpy axis (slowest first).  The colour is
    sum over axes of (block index mod 2) << axis_id with x = axis_id 0.
    """
    d = len(shape)
    nb = block_counts(shape, sub)
    strides = [int(np.prod(shape[a + 1:])) for a in range(d)]
    out = []
    for bidx in itertools.product(*[range(n) for n in nb]):
        ranges = [range(bidx[a] * sub[a], min((bidx[a] + 1) * sub[a], shape[a])) for a in range(d)]
        pts = []
        for coord in itertools.product(*ranges):
            pts.append(sum(coord[a] * strides[a] for a in range(d)))
        colour = 0
        for a in range(d):
            axis_id = d - 1 - a          # numpy axis a is x (0) when a == d-1
            colour |= (bidx[a] & 1) << axis_id
        out.append((colour, np.array(sorted(pts), dtype=np.int64)))
    return out


def unknown_indices(points: np.ndarray, K: int) -> np.ndarray:
    return (points[:, None] * K + np.arange(K)[None, :]).ravel()


def block_update(G, g, x, idx) -> np.ndarray:
    """delta_U = G_UU^{-1} (g - G x)_U for one subvolume U (unknown indices idx): the exact
    minimisation of N over U with the rest of x fixed (Sec. II)."""
    G = G.tocsr()
    s = g[idx] - G[idx] @ x
    Guu = G[idx][:, idx].toarray()
    return sla.cho_solve(sla.cho_factor(Guu, lower=True), s)


class BlockRelaxation:
    """Exact coloured block Gauss-Seidel on a Hermitian positive-definite level operator G."""

    def __init__(self, G, shape, sub, K):
        self.G = G.tocsr()
        self.K = K
        self.ncolours = 1 << len(shape)
        self.blocks = []
        for colour, pts in subvolumes(shape, sub):
            idx = unknown_indices(pts, K)
            Guu = self.G[idx][:, idx].toarray()
            self.blocks.append((colour, idx, sla.cho_factor(Guu, lower=True)))

    def colour_pass(self, x, g, colour):
        s = g - self.G @ x
        updates = []
        for col, idx, fac in self.blocks:
            if col == colour:
                updates.append((idx, sla.cho_solve(fac, s[idx])))
        for idx, d in updates:
            x[idx] += d

    def sweep(self, x, g, after_colour=None):
        """One sweep = one pass over every colour in order 0 .. 2^d - 1."""
        for colour in range(self.ncolours):
            self.colour_pass(x, g, colour)
            if after_colour is not None:
                after_colour(colour)


def colouring_is_valid(G, shape, sub, K) -> bool:
    """True when no two distinct same-colour subvolumes are coupled by G (pin for the colouring)."""
    G = G.tocsr()
    blocks = subvolumes(shape, sub)
    owner = np.full(G.shape[0], -1, dtype=np.int64)
    colour_of = []
    for b, (colour, pts) in enumerate(blocks):
        owner[unknown_indices(pts, K)] = b
        colour_of.append(colour)
    coo = G.tocoo()
    nz = np.abs(coo.data) > 0
    bi, bj = owner[coo.row[nz]], owner[coo.col[nz]]
    cross = bi != bj
    same = np.array(colour_of)[bi[cross]] == np.array(colour_of)[bj[cross]]
    return not bool(np.any(same))


# ----------------------------------------------------------------------------- square form
def red_black_subvolumes(shape, sub):
    """(colour, point indices) per subvolume with the two-colour checkerboard colouring
    colour = (sum of block indices) mod 2.  M couples only edge neighbours (radius-1
    stencil), so two same-colour subvolumes, which touch at most at corners, never
    share a row of M."""
    d = len(shape)
    nb = block_counts(shape, sub)
    strides = [int(np.prod(shape[a + 1:])) for a in range(d)]
    out = []
    for bidx in itertools.product(*[range(n) for n in nb]):
        ranges = [range(bidx[a] * sub[a], min((bidx[a] + 1) * sub[a], shape[a])) for a in range(d)]
        pts = sorted(sum(coord[a] * strides[a] for a in range(d)) for coord in itertools.product(*ranges))
        out.append((int(sum(bidx)) % 2, np.array(pts, dtype=np.int64)))
    return out


def square_block_update(M, f, x, idx) -> np.ndarray:
    """delta_U = M_UU^{-1} (f - M x)_U for one subvolume U (unknown indices idx): the square
    Dirichlet form of the local problem (Sec. II); afterwards the residual rows of U vanish."""
    M = M.tocsr()
    r = f[idx] - M[idx] @ x
    return np.linalg.solve(M[idx][:, idx].toarray(), r)


class SquareRelaxation:
    """Red-black block Gauss-Seidel on M c = f with the square local problem of Sec. II."""

    def __init__(self, M, shape, sub, K):
        self.M = M.tocsr()
        self.K = K
        self.ncolours = 2
        self.blocks = []
        for colour, pts in red_black_subvolumes(shape, sub):
            idx = unknown_indices(pts, K)
            self.blocks.append((colour, idx, sla.lu_factor(self.M[idx][:, idx].toarray())))

    def colour_pass(self, x, f, colour, order=1):
        r = f - self.M @ x
        updates = [(idx, sla.lu_solve(fac, r[idx])) for col, idx, fac in self.blocks[::order] if col == colour]
        for idx, d in updates:
            x[idx] += d

    def sweep(self, x, f, after_colour=None):
        """One sweep = colour 0 then colour 1."""
        for colour in range(2):
            self.colour_pass(x, f, colour)
            if after_colour is not None:
                after_colour(colour)


def red_black_is_valid(A, shape, sub, K) -> bool:
    """True when no two distinct same-colour red-black subvolumes are coupled by A."""
    A = A.tocsr()
    blocks = red_black_subvolumes(shape, sub)
    owner = np.full(A.shape[0], -1, dtype=np.int64)
    colour_of = []
    for b, (colour, pts) in enumerate(blocks):
        owner[unknown_indices(pts, K)] = b
        colour_of.append(colour)
    coo = A.tocoo()
    nz = np.abs(coo.data) > 0
    bi, bj = owner[coo.row[nz]], owner[coo.col[nz]]
    cross = bi != bj
    same = np.array(colour_of)[bi[cross]] == np.array(colour_of)[bj[cross]]
    return not bool(np.any(same))
