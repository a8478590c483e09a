"""Pins for the oracle's Legendre-element convergence maps (Secs. IV-V: element matrices,
constrained relaxation, continuity projection, the plane-wave experiment)."""
import os

import numpy as np
import pytest

from oracle import legendre_elements as le
from oracle import lfa


@pytest.mark.parametrize("nx,nt", [(3, 3), (4, 5), (6, 6)])
def test_element_matrices_closed_forms(nx, nt):
    """Sec. IV: O and U from the orthogonality relation, Q_nm = 2 for n > m with n - m odd, and the
    kinetic element in the closed form of Eq. Tmatelt (row = test function)."""
    O, U, Qt, K = lfa.element_matrices(nx, nt)
    assert np.allclose(O, np.diag(2.0 / (2 * np.arange(nx) + 1)), atol=1e-14)
    assert np.allclose(U, np.diag(2.0 / (2 * np.arange(nt) + 1)), atol=1e-14)
    for m in range(nt):
        for n in range(nt):
            ref = 2.0 if (n > m and (n - m) % 2 == 1) else 0.0
            assert abs(Qt[m, n] - ref) < 1e-13
    for j in range(nx):
        for i in range(nx):
            ref = (j * (j + 1) - i * (i + 1)) / 2.0 if (i > j and (i - j) % 2 == 0) else 0.0
            assert abs(K[j, i] - ref) < 1e-12


@pytest.mark.parametrize("nx,nt", [(3, 3), (4, 4), (5, 3), (6, 6)])
def test_constraint_ranks(nx, nt):
    """Initial-time and end values meet at an element's two bottom corners (and, for two elements,
    at the bottom of the shared boundary), so Nx + 2 Nt conditions have rank Nx + 2 Nt - 2; for
    two elements 2 Nx + 3 Nt conditions have rank 2 Nx + 3 Nt - 3."""
    assert np.linalg.matrix_rank(lfa.constraints(nx, nt, 1)) == nx + 2 * nt - 2
    assert np.linalg.matrix_rank(lfa.constraints(nx, nt, 2)) == 2 * nx + 3 * nt - 3


def test_unconstrained_relaxation_is_the_exact_solve():
    """Without any condition the correction solves A delta = r exactly: the relaxed residual is 0."""
    A = lfa.element_operator(4, 4, 1.0, 0.5)
    C = lfa.project(4, 4, 1, lfa.plane_wave_overlaps(4, 4, 1, 1.3, -0.7))
    C1 = lfa.relax(A, np.zeros((0, 16)), C)
    assert np.linalg.norm(A @ C1) < 1e-12 * np.linalg.norm(A @ C)


@pytest.mark.parametrize("nel", [1, 2])
def test_null_space_solution_equals_the_bordered_system(nel):
    """The Lagrange-multiplier system [A B^T; B 0] solved by least squares (minimum norm, which
    copes with the repeated corner conditions) gives the same correction."""
    nx, nt = 4, 3
    A1 = lfa.element_operator(nx, nt, 0.1, -1.0)
    A = A1 if nel == 1 else np.kron(np.eye(2), A1)
    B = lfa.constraints(nx, nt, nel)
    C = lfa.project(nx, nt, nel, lfa.plane_wave_overlaps(nx, nt, nel, 2.1, 0.4))
    r = -A @ C
    nc = B.shape[0]
    kkt = np.block([[A, B.T.astype(complex)], [B.astype(complex), np.zeros((nc, nc))]])
    sol = np.linalg.lstsq(kkt, np.concatenate([r, np.zeros(nc)]), rcond=None)[0]
    assert np.linalg.norm(C + sol[:len(C)] - lfa.relax(A, B, C)) < 1e-11 * np.linalg.norm(C)


@pytest.mark.parametrize("method", ["one", "two", "transfer"])
def test_relaxation_keeps_initial_and_boundary_values(method):
    nx, nt = 5, 4
    nel = 1 if method == "one" else 2
    C = lfa.project(nx, nt, nel, lfa.plane_wave_overlaps(nx, nt, nel, -1.7, 2.2))
    C1 = lfa.relax_method(method, nx, nt, 1.0, 1.0, C)
    B = lfa.constraints(nx, nt, nel)
    assert np.linalg.norm(B @ (C1 - C)) < 1e-12 * np.linalg.norm(C)
    assert np.linalg.norm(C1 - C) > 1e-3 * np.linalg.norm(C)


def test_continuous_projection():
    """Two elements: the projected trial is continuous at x = 0; a constant is reproduced exactly,
    and the projection of a plane wave converges to it as Nx grows."""
    B = lfa.constraints(4, 3, 2, left=False, right=False, initial=False)
    C = lfa.project(4, 3, 2, lfa.plane_wave_overlaps(4, 3, 2, 2.5, 1.0))
    assert np.linalg.norm(B @ C) < 1e-13 * np.linalg.norm(C)
    C0 = lfa.project(4, 3, 2, lfa.plane_wave_overlaps(4, 3, 2, 0.0, 0.0))
    ref = np.zeros(24)
    ref[0] = ref[12] = 1.0
    assert np.allclose(C0, ref, atol=1e-13)
    # value at x = 0.5 (right child y' = 0), t = 0: sum_i C[i, n] P_i(0) P_n(0)
    errs = []
    for nx in (4, 6, 8):
        C = lfa.project(nx, 8, 2, lfa.plane_wave_overlaps(nx, 8, 2, 2.5, 1.0))
        Pi = le.legendre_P(nx - 1, np.array([0.0]))[:, 0]
        Pn = le.legendre_P(7, np.array([0.0]))[:, 0]
        v = Pi @ C[nx * 8:].reshape(nx, 8) @ Pn
        errs.append(abs(v - np.exp(1j * 2.5 * 0.5)))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-5


def test_maps_follow_sec_v():
    """Sec. V, qualitatively: a larger basis converges faster and shrinks the region where the
    residual norm grows (ratio > 1); relaxing the two elements through the parent-element transfer
    converges about as fast as relaxing both at once, and faster than one element alone."""
    ks = np.linspace(-6, 6, 9)
    ws = np.linspace(-6, 6, 9)
    small, _ = lfa.ratio_map("one", 3, 3, 1.0, 0.0, ks, ws)
    large, _ = lfa.ratio_map("one", 6, 6, 1.0, 0.0, ks, ws)
    assert np.median(large) < np.median(small) - 0.5
    assert np.mean(large > 0) < np.mean(small > 0)
    one, _ = lfa.ratio_map("one", 5, 5, 1.0, 0.0, ks, ws)
    two, _ = lfa.ratio_map("two", 5, 5, 1.0, 0.0, ks, ws)
    tr, _ = lfa.ratio_map("transfer", 5, 5, 1.0, 0.0, ks, ws)
    assert abs(np.median(tr) - np.median(two)) < 0.5
    assert np.median(tr) < np.median(one)


def test_two_by_two_element_has_no_free_parameter():
    """Nx = Nt = 2: the four conditions of one element have rank 4 = Nx Nt, so a relaxation cannot
    change the trial (log ratio 0); two elements keep 8 - 7 = 1 free parameter."""
    assert lfa.null_space(lfa.constraints(2, 2, 1)).shape[1] == 0
    assert lfa.null_space(lfa.constraints(2, 2, 2)).shape[1] == 1
    N, S = lfa.ratio_map("one", 2, 2, 1.0, 0.5, np.array([1.3, -2.0]), np.array([0.4]))
    assert np.all(N == 0.0) and np.all(S == 0.0)


def _sec5_facts():
    facts = {"kappa_nu": [], "counts": {}, "cost": {}}
    path = os.path.join(os.path.dirname(__file__), "golden", "sec5_plane_wave_experiment.txt")
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "kappa_nu":
            facts["kappa_nu"].append((float(f[1]), float(f[2])))
        elif f[0] == "counts":
            facts["counts"][f[1]] = (int(f[2]), int(f[3]), int(f[5]), int(f[7]))
        elif f[0] == "cost":
            facts["cost"][f[1]] = float(f[2])
    return facts


def test_sec5_printed_parameters_counts_and_costs(monkeypatch):
    """Sec. V as printed: the eight (kappa, nu) pairs of the figures; at Nx = Nt = 3 one element has
    9 free parameters and 9 constraint equations, two elements 18 and 12 (the 15 conditions of two
    elements, initial values per element included, have rank 12); the transfer method solves three
    systems of one element's size, 1.5 times the cost of relaxing each element separately, against
    4 times for both at once."""
    facts = _sec5_facts()
    assert lfa.KAPPA_NU == facts["kappa_nu"]
    nx, nt, params, ncons = facts["counts"]["one"]
    assert nx * nt == params
    assert lfa.constraints(nx, nt, 1).shape[0] == ncons
    nx, nt, params, ncons = facts["counts"]["two"]
    assert 2 * nx * nt == params
    assert np.linalg.matrix_rank(lfa.constraints(nx, nt, 2)) == ncons

    sizes = []
    solve = lfa.constrained_solve

    def counting(A, B, r, solver="null"):
        sizes.append(A.shape[0])
        return solve(A, B, r, solver)

    monkeypatch.setattr(lfa, "constrained_solve", counting)
    n = 4 * 4
    C = lfa.project(4, 4, 2, lfa.plane_wave_overlaps(4, 4, 2, 1.0, -0.5))
    cost = {}
    for method in ("two", "transfer"):
        sizes.clear()
        lfa.relax_method(method, 4, 4, 1.0, 0.0, C)
        cost[method] = sum(s ** 3 for s in sizes) / (2 * n ** 3)
    assert sizes == [n, n, n]
    assert cost == facts["cost"]


def test_slow_convergence_only_near_the_dispersion_curve():
    """Sec. V: with a large basis the residual norm falls nearly everywhere and grows only near the
    curve where the plane wave solves the equation (so the trial is already close to the minimum
    action wavefunction); for the dimensionless rows A that is -w = kappa k^2 + nu.  A small basis
    instead fails to converge over much of the plane."""
    ks = np.linspace(-3.0, 3.0, 7)
    ws = np.linspace(-5.0, 5.0, 11)
    W, K = np.meshgrid(ws, ks, indexing="ij")
    grows = {3: [0, 0], 8: [0, 0]}          # points where N grows: near the curve, away from it
    for nb in grows:
        for kappa, nu in lfa.KAPPA_NU:
            lrN, _ = lfa.ratio_map("one", nb, nb, kappa, nu, ks, ws)
            near = np.abs(W + kappa * K ** 2 + nu) <= 0.5
            grows[nb][0] += int(np.sum((lrN > 0) & near))
            grows[nb][1] += int(np.sum((lrN > 0) & ~near))
    assert grows[8][0] > 0 and grows[8][1] == 0
    assert grows[3][1] > 50


def _physical_rows(nx, nt, width, duration, V):
    """Rows of one element x in [x0, x0 + width], t in [0, duration] in physical units, by quadrature:
    int int P_j(y) P_m(tau) (i d/dt + 1/2 d^2/dx^2 - V) P_i(y) P_n(tau) dx dt, y and tau the element's
    Legendre variables (derivatives through the chain rule, x = x0 + width (y + 1)/2)."""
    from numpy.polynomial import legendre as L
    q, wq = L.leggauss(nx + nt + 4)
    e = np.eye(max(nx, nt))
    P = lambda k, d=0: L.legval(q, L.legder(e[k], d) if d else e[k])
    sx, st = 2.0 / width, 2.0 / duration
    jx, jt = width / 2.0 * wq, duration / 2.0 * wq
    A = np.zeros((nx * nt, nx * nt), dtype=complex)
    for j in range(nx):
        for m in range(nt):
            for i in range(nx):
                for n in range(nt):
                    ox = jx @ (P(j) * P(i))
                    ut = jt @ (P(m) * P(n))
                    dt_ = jt @ (P(m) * st * P(n, 1))
                    dxx = jx @ (P(j) * sx ** 2 * P(i, 2))
                    A[j * nt + m, i * nt + n] = 1j * ox * dt_ + 0.5 * dxx * ut - V * ox * ut
    return A


@pytest.mark.parametrize("width,duration,V", [(2.0, 2.0, 0.0), (0.3, 0.05, -1.7), (1.1, 0.4, 2.5)])
def test_dimensionless_rows_and_their_scaling(width, duration, V):
    """Eq. leastaction_dimensionless from the physical rows: divided by the element's half-width, they
    are i O Qt - 2 kappa K U - nu O U with kappa = p_max^2 dt / 2 and nu = V dt, p_max = 1/dx, where
    dx and dt are the element's half-extents (the Jacobians of its Legendre variables).  Hence
    (Sec. IV) doubling the element maps kappa to kappa/4 with nu unchanged, and halving the step maps
    (kappa, nu) to (kappa/2, nu/2)."""
    nx, nt = 4, 3
    hx, ht = width / 2.0, duration / 2.0
    kappa, nu = (1.0 / hx) ** 2 * ht / 2.0, V * ht
    A = _physical_rows(nx, nt, width, duration, V) / hx
    assert np.allclose(A, lfa.element_operator(nx, nt, kappa, nu), atol=1e-11 * np.abs(A).max())
    A2 = _physical_rows(nx, nt, 2 * width, duration, V) / (2 * hx)
    assert np.allclose(A2, lfa.element_operator(nx, nt, kappa / 4, nu), atol=1e-11 * np.abs(A2).max())
    Ah = _physical_rows(nx, nt, width, duration / 2, V) / hx
    assert np.allclose(Ah, lfa.element_operator(nx, nt, kappa / 2, nu / 2), atol=1e-11 * np.abs(Ah).max())


@pytest.mark.parametrize("nel", [1, 2])
def test_plane_wave_overlaps_closed_form(nel):
    """int_{-1}^{1} exp(i a y) P_n(y) dy = 2 i^n j_n(a) (spherical Bessel function): the trial's
    overlaps with one element, and with the children x = (y - 1)/2, (y + 1)/2 of two elements
    (a = k/2 and the phase exp(-+ i k/2))."""
    from scipy.special import spherical_jn
    nx, nt, k, w = 5, 4, 3.7, -2.2
    got = lfa.plane_wave_overlaps(nx, nt, nel, k, w).reshape(nel, nx, nt)
    bt = np.array([2 * 1j ** n * spherical_jn(n, w) for n in range(nt)])
    for e in range(nel):
        if nel == 1:
            ax = np.array([2 * 1j ** i * spherical_jn(i, k) for i in range(nx)])
        else:
            shift = -0.5 if e == 0 else 0.5
            ax = np.exp(1j * k * shift) * np.array([2 * 1j ** i * spherical_jn(i, k / 2) for i in range(nx)])
        assert np.allclose(got[e], np.outer(ax, bt), atol=1e-13)


@pytest.mark.parametrize("kappa,nu", [(1.0, 0.0), (0.1, -1.0), (10.0, 1.0)])
def test_transfer_coarse_step_solves_the_projected_problem(kappa, nu):
    """Eqs. residual_rough and correction_fine on two elements: the coarse step's correction is
    interpolated from the parent (delta = I d), d meets the parent's own conditions, and the projected
    residual P (r - A delta) has no component in the directions those conditions leave free.  I and P
    are the element transfers pinned against their definitions (children's expansions, L2 projection)."""
    from scipy.linalg import null_space
    nx, nt = 5, 4
    A2 = np.kron(np.eye(2), lfa.element_operator(nx, nt, kappa, nu))
    C = lfa.project(nx, nt, 2, lfa.plane_wave_overlaps(nx, nt, 2, 1.7, -0.9))
    delta = lfa.coarse_correction(A2, C, nx, nt) - C
    I = np.kron(le.interpolation(nx - 1), np.eye(nt))
    P = np.kron(le.projection(nx - 1), np.eye(nt))
    d = P @ delta
    assert np.linalg.norm(delta - I @ d) < 1e-12 * np.linalg.norm(delta)
    B1 = lfa.constraints(nx, nt, 1)
    assert np.linalg.norm(B1 @ d) < 1e-12 * np.linalg.norm(d)
    Z = null_space(B1)
    rc = P @ (-A2 @ (C + delta))
    assert np.linalg.norm(Z.T @ rc) < 1e-10 * np.linalg.norm(P @ (A2 @ C))
    assert np.linalg.norm(delta) > 1e-3 * np.linalg.norm(C)


@pytest.mark.parametrize("method", ["one", "two", "transfer"])
def test_correction_vanishes_at_the_initial_time_and_the_volume_ends(method):
    """Eqs. ic_correction, bc1_correction, bc2_correction and continuity, read off the correction as a
    function: delta(x, t) of one relaxation is zero at the initial time (tau = -1) everywhere and at
    both outer ends of the relaxation volume at all times, continuous across the inner boundary, and
    not zero at the end of the step (tau = +1).  Evaluated from the Legendre expansions themselves,
    not through the constraint rows."""
    from numpy.polynomial import legendre as L
    nx, nt = 5, 4
    nel = 1 if method == "one" else 2
    C = lfa.project(nx, nt, nel, lfa.plane_wave_overlaps(nx, nt, nel, -1.7, 2.2))
    D = (lfa.relax_method(method, nx, nt, 1.0, 1.0, C) - C).reshape(nel, nx, nt)
    s = np.linspace(-1.0, 1.0, 9)
    scale = max(np.abs(L.legval2d(a, b, D[e])) for e in range(nel) for a in s for b in s)
    for e in range(nel):
        assert np.max(np.abs(L.legval2d(s, -np.ones_like(s), D[e]))) < 1e-12 * scale
    assert np.max(np.abs(L.legval2d(-np.ones_like(s), s, D[0]))) < 1e-12 * scale
    assert np.max(np.abs(L.legval2d(np.ones_like(s), s, D[nel - 1]))) < 1e-12 * scale
    if nel == 2:
        jump = L.legval2d(np.ones_like(s), s, D[0]) - L.legval2d(-np.ones_like(s), s, D[1])
        assert np.max(np.abs(jump)) < 1e-12 * scale
    assert max(np.max(np.abs(L.legval2d(s, np.ones_like(s), D[e]))) for e in range(nel)) > 1e-3 * scale


@pytest.mark.parametrize("kappa,nu", [(1.0, 0.0), (0.3, -1.0)])
def test_action_by_quadrature_of_the_trial_function(kappa, nu):
    """S = C^H A C against the integral of conj(phi) (i d/dtau + kappa d^2/dy^2 - nu) phi over the
    element for the trial phi(y, tau) = sum C[i, n] P_i(y) P_n(tau), by a Gauss rule (the
    dimensionless rows of Eq. leastaction_dimensionless as an integral; the trial enters conjugated)."""
    from numpy.polynomial import legendre as L
    nx, nt = 5, 4
    C = lfa.project(nx, nt, 1, lfa.plane_wave_overlaps(nx, nt, 1, 1.3, -0.7))
    _, S = lfa.measures(lfa.element_operator(nx, nt, kappa, nu), lfa.weight(nx, nt, 1), C)
    q, wq = L.leggauss(12)
    Cm = C.reshape(nx, nt)
    Y, T = np.meshgrid(q, q, indexing="ij")
    phi = L.legval2d(Y, T, Cm)
    phi_t = L.legval2d(Y, T, L.legder(Cm, axis=1))
    phi_yy = L.legval2d(Y, T, L.legder(Cm, m=2, axis=0))
    S_quad = np.sum(np.outer(wq, wq) * np.conj(phi) * (1j * phi_t + kappa * phi_yy - nu * phi))
    assert abs(S - S_quad) < 1e-12 * max(1.0, abs(S_quad))
