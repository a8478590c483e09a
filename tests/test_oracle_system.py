"""Pins for the oracle's least-action system (Sec. I stationarity, initial condition, Eq. residnorm).

Each check is independent of the oracle's own assembly: closed forms derived by
hand, an exact symbolic derivation (sympy), a dense KKT system with explicit
Lagrange multipliers built from the paper's closed-form U and Q, eigen-expansions
of the discrete Hamiltonian, and the continuum free-packet solution.
"""
import functools
import math

import numpy as np
import pytest

from oracle import propagate, system
from paper_1111_4363_gb300 import workloads as wl


class ConstFieldProblem(system.Problem):
    e0 = 0.0

    def field(self, t):
        return self.e0 + 0.0 * np.asarray(t)


def one_point(K, z, dt=0.05):
    """A one-point grid whose Hamiltonian is the scalar E = z/dt (T_pp = 1/h^2 is cancelled by V0)."""
    return system.Problem(dim=1, shape=(1,), h=(1.0,), K=K, dt=dt, V0=np.array([z / dt - 1.0]),
                          xlaser=np.zeros(1), pulse=None)


def oracle_R(K, z):
    prob = one_point(K, z)
    psi1, _ = propagate.step_direct(prob, np.array([1.0 + 0j]), 0.0)
    return complex(psi1[0])


@functools.lru_cache(maxsize=None)
def sympy_R(K):
    """R_K(z) from the stationarity condition integrated exactly (symbolic), as a numpy-callable."""
    sy = pytest.importorskip("sympy")
    tau, z = sy.symbols("tau z")
    P = [sy.legendre(n, tau) for n in range(K + 1)]
    b = [P[n] - (-1) ** n * P[0] for n in range(1, K + 1)]
    cs = sy.symbols("c1:%d" % (K + 1))
    phi = 1 + sum(c * bn for c, bn in zip(cs, b))
    # int dt/2 dtau b_m (i d/dt - E) phi = int b_m (i dphi/dtau - (z/2) phi) dtau = 0
    eqs = [sy.integrate(bm * (sy.I * sy.diff(phi, tau) - z / 2 * phi), (tau, -1, 1)) for bm in b]
    sol = sy.solve(eqs, cs, dict=True)[0]
    expr = sy.simplify(phi.subs(sol).subs(tau, 1))
    return sy.lambdify(z, expr, "numpy")


@pytest.mark.parametrize("z", [0.05, 0.5, -0.3, 2.0])
def test_scalar_K1_closed_form(z):
    # K = 1 by hand: c (2i - 4z/3) = z psi0  =>  R = (1 - i z/3)/(1 + 2 i z/3)
    assert abs(oracle_R(1, z) - (1 - 1j * z / 3) / (1 + 2j * z / 3)) < 1e-15


@pytest.mark.parametrize("K", [2, 3, 4, 6])
def test_scalar_matches_symbolic(K):
    R = sympy_R(K)
    for z in (0.05, 0.5, -1.0, 3.0):
        assert abs(oracle_R(K, z) - complex(R(z))) < 1e-14


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_scalar_order_K(K):
    # global order K: |R_K(z) - exp(-iz)| ~ C z^{K+1}
    e1 = abs(oracle_R(K, 0.2) - np.exp(-0.2j))
    e2 = abs(oracle_R(K, 0.1) - np.exp(-0.1j))
    assert abs(math.log2(e1 / e2) - (K + 1)) < 0.1


def kinetic_by_loops(n, h):
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] = 1.0 / h ** 2
        if i > 0:
            T[i, i - 1] = -0.5 / h ** 2
        if i + 1 < n:
            T[i, i + 1] = -0.5 / h ** 2
    return T


@pytest.mark.parametrize("n,K,e0", [(8, 2, 0.0), (8, 2, 0.3), (6, 4, -0.7)])
def test_kkt_with_multipliers(n, K, e0):
    """Dense KKT of Sec. I (S' = S + sum lambda_i f_i^*) in the full basis P_0..P_K, with the
    paper's closed forms U_nm = (dt/2) 2 delta/(2n+1) and Q_nm = int P_n' P_m = 2 (n > m, n-m odd)."""
    h, dt = 0.4, 0.05
    rng = np.random.default_rng(3)
    x = (np.arange(n) - (n - 1) / 2) * h
    V0 = 0.5 * x ** 2 + rng.uniform(-0.5, 0.5, n)
    psi0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Kf = K + 1
    U = np.diag([dt / 2 * 2.0 / (2 * m + 1) for m in range(Kf)])
    Q = np.array([[2.0 if (nn > m and (nn - m) % 2 == 1) else 0.0 for m in range(Kf)] for nn in range(Kf)])
    Hs = kinetic_by_loops(n, h) + np.diag(V0)
    A = np.zeros((n * Kf, n * Kf), dtype=complex)        # row (j, m), column (i, nn)
    for j in range(n):
        for m in range(Kf):
            for i in range(n):
                for nn in range(Kf):
                    a = -Hs[i, j] * U[nn, m]
                    if i == j:
                        a += 1j * Q[nn, m] - x[i] * e0 * U[nn, m]
                    A[j * Kf + m, i * Kf + nn] = h * a
    B = np.zeros((n, n * Kf))
    for i in range(n):
        for nn in range(Kf):
            B[i, i * Kf + nn] = (-1.0) ** nn                  # P_n(t0) = P_n(-1)
    kkt = np.block([[A, B.T.astype(complex)], [B.astype(complex), np.zeros((n, n), complex)]])
    sol = np.linalg.solve(kkt, np.concatenate([np.zeros(n * Kf), psi0]))
    C = sol[: n * Kf].reshape(n, Kf)
    psi_end = C.sum(axis=1)                                   # P_n(+1) = 1

    prob = ConstFieldProblem(dim=1, shape=(n,), h=(h,), K=K, dt=dt, V0=V0, xlaser=x, pulse=None)
    prob.e0 = e0
    psi1, c = propagate.step_direct(prob, psi0, 0.0)
    np.testing.assert_allclose(psi1, psi_end, rtol=0, atol=1e-13 * np.max(np.abs(psi_end)))
    np.testing.assert_allclose(c.reshape(n, K), C[:, 1:], rtol=0, atol=1e-12 * np.max(np.abs(C)))


def test_eigen_expansion_and_norm_drift():
    """Time-independent H: the least-action step is diagonal in H's eigenbasis with factor R_K(E dt)."""
    w = wl.harmonic_1d()
    prob = system.Problem.from_workload(w)
    n, h, K, dt = w.n[0], w.h[0], w.nt, w.dt
    x = wl.axis_coordinates(n, h)
    E, V = np.linalg.eigh(kinetic_by_loops(n, h) + np.diag(0.5 * x ** 2))
    R = sympy_R(K)
    psi0 = wl.initial_state(w).ravel()
    nsteps = 3
    psi = psi0.copy()
    for k in range(nsteps):
        psi, _ = propagate.step_direct(prob, psi, k * dt)
    amp = V.T @ psi0
    factor = np.array([complex(R(e * dt)) for e in E])
    expected = V @ (factor ** nsteps * amp)
    np.testing.assert_allclose(psi, expected, rtol=0, atol=1e-12 * np.max(np.abs(expected)))
    # norm drift equals sum |a|^2 (|R|^{2k} - 1)
    drift = np.sum(np.abs(psi) ** 2) - np.sum(np.abs(psi0) ** 2)
    assert drift == pytest.approx(np.sum(np.abs(amp) ** 2 * (np.abs(factor) ** (2 * nsteps) - 1)), abs=1e-13)


def test_eigenstate_phase():
    """An exact eigenstate of a time-independent H evolves as exp(-iEt) up to k |R_K(E dt) - exp(-iE dt)|."""
    w = wl.harmonic_1d()
    prob = system.Problem.from_workload(w)
    n, h, K, dt = w.n[0], w.h[0], w.nt, w.dt
    x = wl.axis_coordinates(n, h)
    E, V = np.linalg.eigh(kinetic_by_loops(n, h) + np.diag(0.5 * x ** 2))
    psi0 = V[:, 1].astype(complex)
    psi = psi0.copy()
    nsteps = 20
    for k in range(nsteps):
        psi, _ = propagate.step_direct(prob, psi, k * dt)
    err = np.max(np.abs(psi - np.exp(-1j * E[1] * nsteps * dt) * psi0))
    bound = nsteps * abs(complex(sympy_R(K)(E[1] * dt)) - np.exp(-1j * E[1] * dt)) * np.max(np.abs(psi0))
    assert err <= bound * 1.01 + 1e-13
    assert err < 1e-9


def free_packet(x, t, k0=1.0):
    """Continuum free evolution of exp(-x^2/2 + i k0 x), m = 1, hbar = 1."""
    s = 1.0 + 1j * t
    return s ** -0.5 * np.exp(-((x - k0 * t) ** 2) / (2 * s) + 1j * k0 * x - 0.5j * k0 ** 2 * t)


def test_free_gaussian_second_order_in_h():
    errs = []
    for n in (201, 401):
        L = 20.0
        h = 2 * L / (n + 1)
        x = wl.axis_coordinates(n, h)
        prob = system.Problem(dim=1, shape=(n,), h=(h,), K=4, dt=0.05, V0=np.zeros(n), xlaser=x, pulse=None)
        psi = free_packet(x, 0.0)
        for k in range(20):
            psi, _ = propagate.step_direct(prob, psi, k * 0.05)
        errs.append(np.max(np.abs(psi - free_packet(x, 1.0))))
    order = math.log2(errs[0] / errs[1])
    assert abs(order - 2.0) < 0.3, (errs, order)
    assert errs[1] < 5e-3


def test_action_norm_is_nonnegative_and_zero_at_solution():
    w = wl.softcore_2d(n=12, levels=1)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    for weight in ("dual", "literal", "identity"):
        M, f, W = system.assemble(prob, 0.7, psi0, weight)
        c = wl.random_state(M.shape[1], 1)
        assert system.action_norm(system.residual(M, f, c), W) > 0
        cs = system.direct_solve(M, f)
        assert system.action_norm(system.residual(M, f, cs), W) < 1e-24 * system.action_norm(f, W)


def test_dual_weight_is_test_basis_invariant():
    """N with W = (O x Ub)^{-1} does not change when the test functions b_m are replaced by A b_m."""
    w = wl.softcore_2d(n=6, levels=1)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    M, f, W = system.assemble(prob, 0.2, psi0, "dual")
    c = wl.random_state(M.shape[1], 5)
    r = system.residual(M, f, c)
    A = np.random.default_rng(0).standard_normal((prob.K, prob.K)) + 3 * np.eye(prob.K)
    import scipy.sparse as sp
    from oracle import timebasis as tb
    Ub, _, _ = tb.static_matrices(prob.K, prob.dt)
    Ar = sp.kron(sp.identity(prob.npoints), A) @ r
    W2 = sp.kron(sp.identity(prob.npoints), np.linalg.inv(A @ Ub @ A.T)) / prob.vol
    assert system.action_norm(Ar, W2) == pytest.approx(system.action_norm(r, W), rel=1e-12)


@pytest.mark.parametrize("kind", ["1d", "2d", "2d_ragged", "3d"])
def test_pointwise_residual_matches_the_assembled_system(kind):
    """residual_at (stencil rows, for grids too large to assemble) against the sparse assembly."""
    import dataclasses
    if kind == "1d":
        w = wl.harmonic_1d()
    elif kind == "2d":
        w = wl.softcore_2d(n=16, levels=2)
    elif kind == "2d_ragged":
        w = dataclasses.replace(wl.softcore_2d(n=16, levels=1), n=(15, 11, 1))
    else:
        w = wl.hydrogen_3d(n=8, nsteps=3, ncomp=3, sub=2)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    t0 = 0.7
    M, f, W = system.assemble(prob, t0, psi0)
    c = wl.random_state(M.shape[1], 4) * 0.1
    r = system.residual(M, f, c).reshape(-1, w.nt)
    rng = np.random.default_rng(1)
    pts = np.unique(np.concatenate([[0, prob.npoints - 1], rng.integers(0, prob.npoints, 40)]))
    got = system.residual_at(prob, t0, psi0, c, pts)
    np.testing.assert_allclose(got, r[pts], rtol=0, atol=1e-13 * np.max(np.abs(r)))
    # c = 0 gives the right-hand side itself
    np.testing.assert_allclose(system.residual_at(prob, t0, psi0, np.zeros_like(c), pts),
                               f.reshape(-1, w.nt)[pts], rtol=0, atol=1e-14 * np.max(np.abs(f)))


def anisotropic_problem():
    """A 3D grid with a different extent and spacing on every axis (numpy order z, y, x)."""
    shape, h = (4, 5, 7), (0.45, 0.7, 0.3)
    rng = np.random.default_rng(11)
    n = int(np.prod(shape))
    return system.Problem(dim=3, shape=shape, h=h, K=2, dt=0.05, V0=rng.uniform(-1, 1, n),
                          xlaser=rng.uniform(-1, 1, n), pulse=None)


def test_laplacian_eigenvalues_on_an_anisotropic_grid():
    """The Dirichlet second difference on n points of spacing h has eigenvalues
    -(4 / h^2) sin^2(j pi / (2 (n + 1))), j = 1..n, and the grid Laplacian's are all sums of one per axis:
    pins which spacing belongs to which axis."""
    prob = anisotropic_problem()
    got = np.sort(np.linalg.eigvalsh(system.laplacian(prob.shape, prob.h).toarray()))
    per_axis = [-4.0 / h ** 2 * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
                for n, h in zip(prob.shape, prob.h)]
    want = np.sort((per_axis[0][:, None, None] + per_axis[1][None, :, None] + per_axis[2][None, None, :]).ravel())
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_stencil_rows_on_an_anisotropic_grid():
    """hamiltonian_row (the stencil form residual_at uses) equals the assembled T + diag(V0) row by row
    on a grid whose axes all differ."""
    prob = anisotropic_problem()
    Hs = system.hamiltonian_operator(prob).toarray()
    for q in range(prob.npoints):
        cols, vals = system.hamiltonian_row(prob, q)
        row = np.zeros(prob.npoints)
        np.add.at(row, cols, vals)
        np.testing.assert_allclose(row, Hs[q], rtol=0, atol=1e-12)


@pytest.mark.parametrize("weight", ["literal", "dual"])
def test_weights_are_l2_norms_of_residual_functions(weight):
    """Eq. residnorm read as a squared L2 norm over the step's space-time slab, by a Gauss rule in time
    with the b_n from scipy's Legendre polynomials and the grid functions' overlap h^d.  "literal":
    N = r O U r* is the norm of the function whose expansion coefficients are r,
    h^d sum_p int |sum_n r_pn b_n(t)|^2 dt.  "dual": the norm of the function g in the trial space
    whose projections onto the test functions are r (its coefficients solve the overlap system
    h^d U g_p = r_p)."""
    from scipy.special import eval_legendre
    w = wl.softcore_2d(n=6, levels=1)
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    M, f, W = system.assemble(prob, 0.2, psi0, weight)
    r = system.residual(M, f, wl.random_state(M.shape[1], 8)).reshape(-1, prob.K)
    q, wq = np.polynomial.legendre.leggauss(prob.K + 4)
    b = np.array([eval_legendre(n, q) - (-1.0) ** n for n in range(1, prob.K + 1)])   # b_n(tau_q)
    jac = 0.5 * prob.dt                                                                # dt = (dt/2) dtau
    if weight == "literal":
        coef = r
    else:
        gram = prob.vol * jac * (b * wq) @ b.T                                         # h^d int b_m b_n dt
        coef = np.linalg.solve(gram, r.T).T
    N_quad = prob.vol * jac * np.sum(wq * np.abs(coef @ b) ** 2)
    assert system.action_norm(r.ravel(), W) == pytest.approx(N_quad, rel=1e-12)


def test_problem_from_an_anisotropic_workload_pairs_extents_with_spacings():
    """Problem.from_workload stores the grid slowest axis first; each axis keeps its own extent and
    spacing: the Laplacian's spectrum is the sum over the workload's axes a of
    -(4 / h_a^2) sin^2(j pi / (2 (n_a + 1))), and the laser coordinate varies along its axis only."""
    import dataclasses
    w = dataclasses.replace(wl.hydrogen_3d(n=8, nsteps=4, ncomp=2, sub=2), n=(7, 5, 4), h=(0.3, 0.7, 0.45))
    w = dataclasses.replace(w, pulse=dataclasses.replace(w.pulse, axis=1))
    prob = system.Problem.from_workload(w)
    got = np.sort(np.linalg.eigvalsh(system.laplacian(prob.shape, prob.h).toarray()))
    per_axis = [-4.0 / w.h[a] ** 2 * np.sin(np.arange(1, w.n[a] + 1) * np.pi / (2 * (w.n[a] + 1))) ** 2
                for a in range(3)]
    want = np.sort((per_axis[0][:, None, None] + per_axis[1][None, :, None] + per_axis[2][None, None, :]).ravel())
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))
    X = prob.xlaser.reshape(prob.shape)                     # numpy order (z, y, x): y is numpy axis 1
    np.testing.assert_array_equal(X, np.broadcast_to(X[:1, :, :1], X.shape))
    np.testing.assert_allclose(X[0, :, 0], (np.arange(w.n[1]) - (w.n[1] - 1) / 2) * w.h[1], atol=1e-15)
