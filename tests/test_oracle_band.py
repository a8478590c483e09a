"""Pin for the block band of the finest-level local factors (Sec. II's subvolume systems G_UU).

The finest-level operator couples grid points at most two steps apart (Manhattan distance, through
H^2), so in the subvolume's x-fastest point order G_UU couples unknowns only when their point indices
are at most d_max apart, d_max the largest index distance of such a pair.  A Cholesky factor has no
fill outside the envelope of its matrix, so a 16 x 16 block (I, J) of L whose nearest points,
floor(16 I / K) and floor((16 J + 15) / K), are more than d_max apart is exact zero.  The wide
factorisation and its solves skip those blocks, so this checks the bound (restated here from its
definition) against the oracle's own factors, on full and ragged subvolumes, and that it is tight.
"""
import dataclasses

import numpy as np
import pytest

from oracle import relax, system
from oracle.propagate import numpy_sub
from paper_1111_4363_gb300 import workloads as wl

BLK = 16


def band_blocks(dim, sub_xyz, K, nblk):
    maxd = 0
    for dz in range(-2, 3):
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                if abs(dx) + abs(dy) + abs(dz) > 2 or (dim < 2 and dy) or (dim < 3 and dz):
                    continue
                maxd = max(maxd, abs(dx + sub_xyz[0] * dy + sub_xyz[0] * sub_xyz[1] * dz))
    band = 0
    for d in range(1, nblk):
        for J in range(nblk - d):
            if (BLK * (J + d)) // K - (BLK * J + BLK - 1) // K <= maxd:
                band = d
    return band


def cases():
    w3 = dataclasses.replace(wl.hydrogen_3d(n=8, nsteps=4, ncomp=4, sub=4), n=(10, 8, 8), levels=1)
    w2 = dataclasses.replace(wl.softcore_2d(n=16, levels=1), nt=4, sub=(8, 8, 1), n=(20, 16, 1))
    w1 = dataclasses.replace(wl.harmonic_1d(), nt=8, sub=(32, 1, 1), n=(70, 1, 1), levels=1)
    return [("3d_4x4x4_K4", w3), ("2d_8x8_K4", w2), ("1d_32_K8", w1)]


@pytest.mark.parametrize("name,w", cases(), ids=[c[0] for c in cases()])
def test_local_factor_vanishes_outside_the_block_band(name, w):
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    M, f, W = system.assemble(prob, 0.2, psi0, w.weight)
    G = (M.conj().T @ W @ M).tocsr()
    K = prob.K
    full_n = int(np.prod(w.sub[:w.dim])) * K
    nblk = -(-full_n // BLK)
    B = band_blocks(w.dim, w.sub, K, nblk)
    assert B < nblk - 1, "the case must have blocks outside the band"
    tight = False
    nfull = 0
    for _, pts in relax.subvolumes(prob.shape, numpy_sub(w)):
        idx = relax.unknown_indices(pts, K)
        L = np.linalg.cholesky(G[idx][:, idx].toarray())
        n = len(idx)
        nb = -(-n // BLK)
        Lp = np.zeros((nb * BLK, nb * BLK), dtype=L.dtype)
        Lp[:n, :n] = L
        for I in range(nb):
            for J in range(I + 1):
                blk = Lp[I * BLK:(I + 1) * BLK, J * BLK:(J + 1) * BLK]
                if I - J > B:
                    assert np.abs(blk).max() == 0.0, (name, I, J)
                elif I - J == B and n == full_n and np.abs(blk).max() > 0.0:
                    tight = True
        nfull += n == full_n
    assert nfull > 0
    assert tight, "no nonzero block at the band's edge: the bound is not tight"


def test_band_of_the_production_subvolumes():
    # 3D 4 x 4 x 4 points x K = 4: d_max = 2 * 16 = 32, block (I, J) spans points 4 I .. and .. 4 J + 3,
    # so the band is 8 (28 of 136 blocks zero); 2D 8 x 8 x K = 4: d_max = 16, band 4 (66 of 136 zero)
    assert band_blocks(3, (4, 4, 4), 4, 16) == 8
    assert band_blocks(2, (8, 8, 1), 4, 16) == 4
    # 2D 4 x 4 x K = 4 (four blocks): d_max = 8, band 2
    assert band_blocks(2, (4, 4, 1), 4, 4) == 2
    # 1D 32 points x K = 8: d_max = 2, two points per block, band 1
    assert band_blocks(1, (32, 1, 1), 8, 16) == 1
