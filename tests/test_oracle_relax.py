"""Pins for the oracle's subvolume relaxation and multigrid (Secs. II, III, IV transfers)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import legendre_elements as le
from oracle import multigrid, relax, system
from paper_1111_4363_gb300 import workloads as wl


def small_2d(n=16, levels=2, weight="dual"):
    w = wl.softcore_2d(n=n, levels=levels)
    w.weight = weight
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    M, f, W = system.assemble(prob, 0.35, psi0, weight)
    return w, prob, M, f, W


def test_subvolume_partition_and_colours():
    shape, sub = (10, 12), (4, 4)       # ragged tail on the slow axis
    blocks = relax.subvolumes(shape, sub)
    pts = np.concatenate([p for _, p in blocks])
    assert sorted(pts.tolist()) == list(range(120))
    assert len(blocks) == 3 * 3
    assert sorted(set(c for c, _ in blocks)) == [0, 1, 2, 3]


@pytest.mark.parametrize("weight", ["dual", "literal", "identity"])
def test_colouring_valid_every_level(weight):
    w, prob, M, f, W = small_2d(n=16, levels=3, weight=weight)
    G0 = (M.conj().T @ W @ M).tocsr()
    h = multigrid.Hierarchy(G0, prob.shape, prob.K, (4, 4), 3)
    for G, shape in zip(h.G, h.shapes):
        assert relax.colouring_is_valid(G, shape, (4, 4), prob.K)
    # sanity of the check itself: a 2-colour checkerboard is NOT valid for the normal operator
    blocks = relax.subvolumes(prob.shape, (4, 4))
    owner = {}
    for b, (c, p) in enumerate(blocks):
        by, bx = divmod(b, 4)
        for q in p:
            owner[int(q)] = (by + bx) % 2
    G = G0.tocoo()
    pt_r, pt_c = G.row // prob.K, G.col // prob.K
    blk = {}
    for b, (c, p) in enumerate(blocks):
        for q in p:
            blk[int(q)] = b
    bad = any(blk[int(a)] != blk[int(b)] and owner[int(a)] == owner[int(b)] for a, b in zip(pt_r, pt_c))
    assert bad


def test_block_update_minimises_N_over_the_block():
    w, prob, M, f, W = small_2d(n=12, levels=1)
    G = (M.conj().T @ W @ M).tocsr()
    g = M.conj().T @ (W @ f)
    R = relax.BlockRelaxation(G, prob.shape, (4, 4), prob.K)
    c = wl.random_state(M.shape[1], 2) * 0.01
    R.colour_pass(c, g, 0)
    r = system.residual(M, f, c)
    grad = M.conj().T @ (W @ r)          # -dN/dc^* / 1
    for col, idx, _ in R.blocks:
        if col == 0:
            assert np.max(np.abs(grad[idx])) < 1e-10 * np.max(np.abs(g))
    # and a random perturbation inside a block never lowers N
    N = system.action_norm(r, W)
    rng = np.random.default_rng(0)
    idx = R.blocks[0][1]
    for _ in range(5):
        d = np.zeros_like(c)
        d[idx] = 1e-3 * (rng.standard_normal(len(idx)) + 1j * rng.standard_normal(len(idx)))
        assert system.action_norm(system.residual(M, f, c + d), W) >= N * (1 - 1e-14)


def test_single_block_update_is_the_blockwise_minimiser():
    """relax.block_update on one subvolume: zero block gradient of N afterwards, and the same update
    as the colour pass (same-colour blocks do not interact)."""
    w, prob, M, f, W = small_2d(n=12, levels=1)
    G = (M.conj().T @ W @ M).tocsr()
    g = M.conj().T @ (W @ f)
    R = relax.BlockRelaxation(G, prob.shape, (4, 4), prob.K)
    c0 = wl.random_state(M.shape[1], 6) * 0.01
    ref = c0.copy()
    R.colour_pass(ref, g, 1)
    for col, idx, _ in R.blocks:
        if col != 1:
            continue
        d = relax.block_update(G, g, c0, idx)
        np.testing.assert_allclose(d, (ref - c0)[idx], rtol=0, atol=1e-12 * np.max(np.abs(d)))
        c = c0.copy()
        c[idx] += d
        grad = M.conj().T @ (W @ system.residual(M, f, c))
        assert np.max(np.abs(grad[idx])) < 1e-10 * np.max(np.abs(g))


def test_same_colour_updates_are_independent():
    # computing all same-colour corrections from one residual equals applying them one by one
    w, prob, M, f, W = small_2d(n=16, levels=1)
    G = (M.conj().T @ W @ M).tocsr()
    g = M.conj().T @ (W @ f)
    R = relax.BlockRelaxation(G, prob.shape, (4, 4), prob.K)
    c0 = wl.random_state(M.shape[1], 4) * 0.01
    a = c0.copy()
    R.colour_pass(a, g, 1)
    b = c0.copy()
    import scipy.linalg as sla
    for col, idx, fac in R.blocks:
        if col == 1:
            s = g - G @ b
            b[idx] += sla.cho_solve(fac, s[idx])
    np.testing.assert_allclose(a, b, atol=1e-13 * np.max(np.abs(a)))


@pytest.mark.parametrize("weight", ["dual", "literal"])
def test_action_never_increases(weight):
    """N is non-increasing after every colour pass and after every coarse-grid correction."""
    w, prob, M, f, W = small_2d(n=16, levels=3, weight=weight)
    hist = []
    state = {}

    def hook(colour):
        hist.append(system.action_norm(system.residual(M, f, state["c"]), W))

    G0 = (M.conj().T @ W @ M).tocsr()
    g0 = M.conj().T @ (W @ f)
    h = multigrid.Hierarchy(G0, prob.shape, prob.K, (4, 4), 3, 1, 1, 2)
    c = np.zeros(M.shape[1], complex)
    state["c"] = c
    hist.append(system.action_norm(f, W))
    for _ in range(4):
        h.vcycle(0, c, g0, hook)
    assert len(hist) > 20
    for a, b in zip(hist[:-1], hist[1:]):
        assert b <= a * (1 + 1e-12) + 1e-30
    assert min(hist) >= 0


def test_1d_relaxation_converges_to_direct_solution():
    w = wl.harmonic_1d()
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    M, f, W = system.assemble(prob, 0.0, psi0)
    cd = system.direct_solve(M, f)
    c, hist, cyc, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, (8,), 1, 1, 0, 0, tol=1e-26,
                                           max_cycles=60)
    assert hist[-1] <= 1e-26 * hist[0]
    assert np.linalg.norm(c - cd) / np.linalg.norm(cd) < 1e-10
    assert cyc < 20


def test_2d_vcycle_converges_to_direct_solution():
    w, prob, M, f, W = small_2d(n=32, levels=3)
    cd = system.direct_solve(M, f)
    c, hist, cyc, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, (4, 4), 3, 1, 1, 2, tol=1e-24,
                                           max_cycles=40)
    assert hist[-1] <= 1e-24 * hist[0]
    assert np.linalg.norm(c - cd) / np.linalg.norm(cd) < 1e-9
    assert cyc <= 15


def test_lighter_galerkin_cycle_converges_to_direct_solution():
    """V(1,2) on the finest level with a (1,0) cycle on the Galerkin levels: the same minimiser, and
    coarse_nu equal to (nu1, nu2) reproduces the uniform cycle exactly."""
    w, prob, M, f, W = small_2d(n=32, levels=3)
    cd = system.direct_solve(M, f)
    c, hist, cyc, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, (4, 4), 3, 1, 2, 1, tol=1e-24,
                                           max_cycles=60, coarse_sub=(2, 2), coarse_nu=(1, 0))
    assert hist[-1] <= 1e-24 * hist[0]
    assert np.linalg.norm(c - cd) < 1e-9 * np.linalg.norm(cd)
    a, _, _, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, (4, 4), 3, 1, 2, 1, ncycles=2, coarse_sub=(2, 2))
    b, _, _, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, (4, 4), 3, 1, 2, 1, ncycles=2, coarse_sub=(2, 2),
                                      coarse_nu=(1, 2))
    assert np.array_equal(a, b)


def test_coarse_correction_is_galerkin_optimal():
    """With an exact coarse solve, c + I e_c minimises N over the coarse space (Eq. correction_fine)."""
    w, prob, M, f, W = small_2d(n=16, levels=2)
    G0 = (M.conj().T @ W @ M).tocsr()
    g0 = M.conj().T @ (W @ f)
    I = multigrid.interpolation(tuple(n // 2 for n in prob.shape), prob.K)
    c = wl.random_state(M.shape[1], 9) * 0.01
    s = g0 - G0 @ c
    Gc = (I.T @ G0 @ I).toarray()
    np.testing.assert_allclose(Gc, Gc.conj().T, atol=1e-12 * np.max(np.abs(Gc)))
    assert np.min(np.linalg.eigvalsh(Gc)) > 0
    ec = np.linalg.solve(Gc, I.T @ s)
    c2 = c + I @ ec
    grad_coarse = I.T @ (g0 - G0 @ c2)
    assert np.max(np.abs(grad_coarse)) < 1e-10 * np.max(np.abs(I.T @ s))


def test_fd_interpolation_reproduces_linear_functions():
    # cell-centred fine points x_{2J} = X_J - H/4, x_{2J+1} = X_J + H/4: 3/4, 1/4 weights are exact for
    # linear functions away from the walls
    nc = 9
    I1 = multigrid.interpolation_1d(nc).toarray()
    X = wl.axis_coordinates(nc, 2.0)
    x = wl.axis_coordinates(2 * nc, 1.0)
    u = 0.3 + 1.7 * X
    v = I1 @ u
    np.testing.assert_allclose(v[1:-1], 0.3 + 1.7 * x[1:-1], atol=1e-14)
    # 2D tensor product keeps the time index untouched
    I2 = multigrid.interpolation((3, 4), 2)
    assert I2.shape == (6 * 8 * 2, 3 * 4 * 2)


@pytest.mark.parametrize("nmax", [1, 2, 3, 5])
def test_legendre_element_transfers(nmax):
    """Sec. IV: (P^(L) + P^(R)) (I^(L) + I^(R)) = identity on the parent basis; E reproduces parent
    functions exactly on each child; O_parent = (1/2) E^T O_f E from the change of variables."""
    E = le.interpolation(nmax)
    P = le.projection(nmax)
    np.testing.assert_allclose(P @ E, np.eye(nmax + 1), atol=1e-13)
    O = le.overlap(nmax)
    np.testing.assert_allclose(O, np.diag([2.0 / (2 * n + 1) for n in range(nmax + 1)]), atol=1e-14)
    Of = np.block([[O, 0 * O], [0 * O, O]])
    np.testing.assert_allclose(0.5 * E.T @ Of @ E, O, atol=1e-13)
    from oracle.timebasis import legendre_P
    yp = np.linspace(-1, 1, 11)
    a = np.random.default_rng(nmax).standard_normal(nmax + 1)
    parent_left = a @ legendre_P(nmax, 0.5 * (yp - 1))
    child_left = (E[: nmax + 1] @ a) @ legendre_P(nmax, yp)
    np.testing.assert_allclose(child_left, parent_left, atol=1e-13)


def test_legendre_kinetic_matrix_closed_form():
    """Eq. Tmatelt: for i > j with i - j even the paper prints (-i(i+1) + j(j+1))/(2m), and 0 for i - j odd.
    The quadrature of the first line, -P_i P_j' |_{-1}^{1} + int P_i' P_j', reproduces it with the boundary
    term's indices exchanged (i.e. the printed value is T[j, i]); the reading is recorded with the others."""
    T = le.kinetic(7)
    for i in range(8):
        for j in range(i):
            expected = (-i * (i + 1) + j * (j + 1)) / 2.0 if (i - j) % 2 == 0 else 0.0
            assert T[j, i] == pytest.approx(expected, abs=1e-12)


def test_vcycle_contraction_is_independent_of_the_grid_size():
    """Sec. III: relaxing on a hierarchy of grids makes convergence independent of the finest grid's
    size.  The 2D soft-core problem (an indefinite H: bound states below zero, kinetic energies far
    above) at 32^2, 64^2 and 128^2, each down to a 16^2 coarsest level: N/N(0) after four V(1,1)
    cycles agrees within a factor 2 and falls below 1e-9 on every grid."""
    import scipy.sparse.linalg as sla
    w, prob, M, f, W = small_2d(n=32, levels=2)
    H = system.hamiltonian_operator(prob)
    lo = sla.eigsh(H, k=1, which="SA", return_eigenvectors=False)[0]
    hi = sla.eigsh(H, k=1, which="LA", return_eigenvectors=False)[0]
    assert lo < 0 < hi
    ratios = []
    for n, levels in ((32, 2), (64, 3), (128, 4)):
        w, prob, M, f, W = small_2d(n=n, levels=levels)
        _, hist, _, _ = multigrid.solve_step(M, f, W, prob.shape, prob.K, (4, 4), levels, 1, 1, 1, ncycles=4,
                                             coarse_sub=(2, 2))
        ratios.append(hist[-1] / hist[0])
    assert max(ratios) < 1e-9
    assert max(ratios) < 2 * min(ratios)


def test_stale_local_factors_keep_the_contraction():
    """The laser term changes the level operators by about 3e-5 (relative) per step in the 2D
    workload, so subvolume factors and Galerkin levels built 200 steps earlier relax the current
    step's residual as well as fresh ones: the same V(1,2) cycles to N/N(0) <= 1e-10, per-cycle
    ratios within 5%.  (Residuals always use the current operator, so the converged coefficients
    are the same minimiser either way.)"""
    w = wl.softcore_2d(n=64, levels=4)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    T = 10.0

    def normal(t):
        M, f, W = system.assemble(prob, t, psi0, w.weight)
        return M, f, W, (M.conj().T @ W @ M).tocsr(), M.conj().T @ (W @ f)

    M, f, W, G, g = normal(T)
    N0 = system.action_norm(f, W)
    hists = []
    for t_built in (T, T - 200 * w.dt):
        Gb = normal(t_built)[3]
        hier = multigrid.Hierarchy(Gb, prob.shape, prob.K, (4, 4), 4, 1, 2, 1, (2, 2), (1, 0))
        hier.G[0] = G
        hier.relax[0].G = G          # current residuals, factors of Gb
        c = np.zeros(M.shape[1], dtype=np.complex128)
        hist = []
        while not hist or (hist[-1] > 1e-10 and len(hist) < 10):
            hier.vcycle(0, c, g)
            hist.append(system.action_norm(system.residual(M, f, c), W) / N0)
        hists.append(np.array(hist))
    fresh, stale = hists
    assert len(fresh) == len(stale) <= 4
    assert np.all(np.abs(stale / fresh - 1) < 0.05)


def test_trial_weights_extrapolate_polynomials_exactly():
    """The trial of a step (the polynomial of degree q - 1 in the step index through the last q
    converged coefficient vectors, evaluated one step on) reproduces every polynomial of degree below
    q and no higher one: the weights used by the oracle's replay of the trial schedule."""
    from tests.helpers import TRIAL_WEIGHTS
    rng = np.random.default_rng(3)
    for q, a in TRIAL_WEIGHTS.items():
        for deg in range(q + 1):
            coef = rng.standard_normal(deg + 1)
            p = lambda s: np.polyval(coef, s)
            n = 7.0
            pred = sum(ai * p(n - 1 - i) for i, ai in enumerate(a))
            if deg < q:
                assert abs(pred - p(n)) < 1e-9 * max(1.0, abs(p(n)))
            else:
                assert abs(pred - p(n)) > 1e-6


@pytest.mark.parametrize("nmax", [1, 2, 3, 5])
def test_legendre_element_projection_is_the_l2_projection(nmax):
    """Sec. IV: P takes a function given on the two children to the parent coefficients of its L2-best
    approximation, a_j = (2j + 1)/2 int_{-1}^{1} f P_j dx.  Computed here by quadrature of the piecewise
    function itself (left child on [-1, 0] with local coordinate 2x + 1, right child on [0, 1] with
    2x - 1): any other left inverse of the interpolation (P I = identity alone does not fix P) fails."""
    from numpy.polynomial import legendre as L
    rng = np.random.default_rng(10 + nmax)
    cl, cr = rng.standard_normal(nmax + 1), rng.standard_normal(nmax + 1)
    q, wq = L.leggauss(nmax + 4)
    a = np.zeros(nmax + 1)
    for c, lo in ((cl, -1.0), (cr, 0.0)):
        x = lo + 0.5 * (q + 1.0)                      # Gauss nodes on the child's half of [-1, 1]
        local = 2.0 * x - (2.0 * lo + 1.0)            # the child's own Legendre coordinate
        f = L.legval(local, c)
        for j in range(nmax + 1):
            e = np.zeros(j + 1)
            e[j] = 1.0
            a[j] += 0.5 * np.sum(wq * f * L.legval(x, e)) * (2 * j + 1) / 2.0
    np.testing.assert_allclose(le.projection(nmax) @ np.concatenate([cl, cr]), a, atol=1e-13)


def test_fd_interpolation_reproduces_linear_functions_on_a_box():
    """The tensor-product interpolation on a 3D grid whose axes all differ (numpy order z, y, x):
    a linear function of the coarse cell centres comes out as the same linear function at the fine
    points away from the walls, for each of the K time functions separately.  Pins which 1D factor
    acts on which axis (a square grid cannot tell)."""
    coarse = (3, 4, 5)
    K = 2
    Hc = (0.8, 0.6, 0.5)                                  # coarse spacings; fine ones are half
    I = multigrid.interpolation(coarse, K)
    Xc = np.meshgrid(*[wl.axis_coordinates(n, h) for n, h in zip(coarse, Hc)], indexing="ij")
    Xf = np.meshgrid(*[wl.axis_coordinates(2 * n, h / 2) for n, h in zip(coarse, Hc)], indexing="ij")
    lin = lambda X: 0.3 + 1.7 * X[0] - 0.9 * X[1] + 0.4 * X[2]
    u = np.stack([lin(Xc).ravel(), -2.0 * lin(Xc).ravel()], axis=1).ravel()    # point-major, K = 2
    v = (I @ u).reshape(tuple(2 * n for n in coarse) + (K,))
    want = lin(Xf)
    inner = tuple(slice(1, 2 * n - 1) for n in coarse)
    np.testing.assert_allclose(v[inner + (0,)], want[inner], atol=1e-13)
    np.testing.assert_allclose(v[inner + (1,)], -2.0 * want[inner], atol=1e-13)
