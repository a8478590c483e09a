"""Pins for the oracle's square-form subvolume relaxation (Sec. II, the preconditioner form
M_UU delta_U = (f - M c)_U with a red-black colouring)."""
import dataclasses

import numpy as np
import pytest

from oracle import relax, system
from paper_1111_4363_gb300 import workloads as wl


def square_case(n=16, dt=0.05, weight="dual"):
    w = dataclasses.replace(wl.softcore_2d(n=n, levels=1), dt=dt, weight=weight)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    M, f, W = system.assemble(prob, 0.35, psi0, weight)
    return w, prob, M.tocsr(), f, W


def rel_actions(R, M, f, W, nsweeps):
    """N(c)/N(0) after every colour pass, starting from c = 0."""
    x = np.zeros(M.shape[1], complex)
    N0 = system.action_norm(f, W)
    out = [1.0]
    for _ in range(nsweeps):
        R.sweep(x, f, after_colour=lambda col: out.append(system.action_norm(system.residual(M, f, x), W) / N0))
    return x, np.array(out)


def test_square_update_zeroes_the_block_residual():
    w, prob, M, f, W = square_case(n=12)
    x = wl.random_state(M.shape[1], 3) * 0.01
    blocks = relax.red_black_subvolumes(prob.shape, (4, 4))
    _, pts = blocks[4]                       # an interior block
    idx = relax.unknown_indices(pts, prob.K)
    r_before = system.residual(M, f, x)
    x[idx] += relax.square_block_update(M, f, x, idx)
    r_after = system.residual(M, f, x)
    assert np.max(np.abs(r_after[idx])) <= 1e-12 * np.max(np.abs(f))
    # rows outside U that couple to U changed; rows far away did not
    far = np.setdiff1d(np.arange(M.shape[0]), M[:, idx].nonzero()[0])
    assert np.array_equal(r_after[far], r_before[far])
    assert np.max(np.abs(r_after - r_before)) > 1e-6 * np.max(np.abs(r_before))


def test_one_block_over_the_whole_grid_is_the_direct_solve():
    w, prob, M, f, W = square_case(n=6)
    R = relax.SquareRelaxation(M, prob.shape, prob.shape, prob.K)
    assert len(R.blocks) == 1
    x = np.zeros(M.shape[1], complex)
    R.colour_pass(x, f, 0)
    xd = system.direct_solve(M, f)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_red_black_is_valid_for_M_but_not_for_the_normal_operator():
    w, prob, M, f, W = square_case(n=16)
    for sub in [(4, 4), (2, 2), (1, 1), (3, 5)]:
        assert relax.red_black_is_valid(M, prob.shape, sub, prob.K)
    # G = M^dagger W M has radius 2: a checkerboard couples corner neighbours
    G = (M.conj().T @ W @ M).tocsr()
    assert not relax.red_black_is_valid(G, prob.shape, (4, 4), prob.K)


def test_same_colour_updates_are_order_independent():
    w, prob, M, f, W = square_case(n=16)
    R = relax.SquareRelaxation(M, prob.shape, (4, 4), prob.K)
    x0 = wl.random_state(M.shape[1], 5) * 0.01
    a, b = x0.copy(), x0.copy()
    R.colour_pass(a, f, 1, order=1)
    R.colour_pass(b, f, 1, order=-1)
    assert np.array_equal(a, b)
    # applying the same-colour updates one at a time (each from the current x) gives the same
    c = x0.copy()
    for col, idx, _ in R.blocks:
        if col == 1:
            c[idx] += relax.square_block_update(M, f, c, idx)
    assert np.max(np.abs(c - a)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("sub", [(4, 4), (2, 2), (4, 2)])
def test_square_relaxation_converges_to_the_direct_solution(sub):
    w, prob, M, f, W = square_case(n=16, dt=0.05)
    R = relax.SquareRelaxation(M, prob.shape, sub, prob.K)
    x, N = rel_actions(R, M, f, W, 14)
    xd = system.direct_solve(M, f)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert N[-1] < 1e-20


def test_square_form_need_not_decrease_the_action():
    """Sec. II: the square local solve is not guaranteed to decrease the action.  With
    one-point subvolumes the first colour pass raises N; the least-squares form on the same
    problem lowers it on every pass."""
    w, prob, M, f, W = square_case(n=16, dt=0.05)
    _, N = rel_actions(relax.SquareRelaxation(M, prob.shape, (1, 1), prob.K), M, f, W, 1)
    assert N[1] > 1.1
    G = (M.conj().T @ W @ M).tocsr()
    g = M.conj().T @ (W @ f)
    R = relax.BlockRelaxation(G, prob.shape, (2, 2), prob.K)
    x = np.zeros(M.shape[1], complex)
    N0 = system.action_norm(f, W)
    prev = 1.0
    for colour in range(R.ncolours):
        R.colour_pass(x, g, colour)
        cur = system.action_norm(system.residual(M, f, x), W) / N0
        assert cur <= prev
        prev = cur


def test_square_form_diverges_where_least_squares_converges():
    """kappa = dt / (2 h^2) = 2.5: the square form diverges for every subvolume size tried, larger
    subvolumes holding out longer (Sec. II: a larger basis in the relaxation volume reduces the
    effect); the least-squares form converges."""
    w, prob, M, f, W = square_case(n=16, dt=0.2)
    first_rise = {}
    for sub in [(2, 2), (4, 4)]:
        _, N = rel_actions(relax.SquareRelaxation(M, prob.shape, sub, prob.K), M, f, W, 20)
        assert N[-1] > 1e3
        first_rise[sub] = int(np.argmax(N[1:] > N[:-1]))
    assert first_rise[(4, 4)] > first_rise[(2, 2)]
    G = (M.conj().T @ W @ M).tocsr()
    g = M.conj().T @ (W @ f)
    R = relax.BlockRelaxation(G, prob.shape, (4, 4), prob.K)
    x = np.zeros(M.shape[1], complex)
    N0, prev = system.action_norm(f, W), 1.0
    for _ in range(20):
        R.sweep(x, g)
        cur = system.action_norm(system.residual(M, f, x), W) / N0
        assert cur < prev
        prev = cur
    assert prev < 1e-3
