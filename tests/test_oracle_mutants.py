"""Planted mistakes in the oracle, each of which one of its pins must catch.

The oracle is trusted because the pins in test_oracle_*.py tie it to facts outside itself: closed
forms of Secs. I and IV, a dense KKT system with explicit multipliers, the exact block minimiser of
Sec. II, Galerkin optimality (Sec. III), scipy's adaptive quadrature, the Sec. V facts the paper
prints.  This file checks that those pins can fail.  Each case plants one plausible mistake in the
oracle -- a dropped term, a wrong sign, index or Jacobian, a transposed operand, a misread
definition -- by patching one oracle function for the duration of the case (CPU only; the CUDA path
is not involved), then runs the named pins and requires at least one of them to fail.  A pin that
raises an AssertionError, or a linear-algebra error (a Cholesky factor that no longer exists),
counts as failing; any other exception is a broken case and errors the test.
"""
import dataclasses
import types

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import adjoint, lfa, multigrid, relax, system
from oracle import legendre_elements as le
from oracle import timebasis as tb
from tests import test_oracle_adjoint as pa
from tests import test_oracle_lfa as pl
from tests import test_oracle_relax as pr
from tests import test_oracle_square as pq
from tests import test_oracle_system as ps
from tests import test_oracle_timebasis as pt


def _wrap(mp, module, name, make):
    """Replace module.name by make(original)."""
    mp.setattr(module, name, make(getattr(module, name)))


# ------------------------------------------------------------------------------ time basis
def b_adds_p0(mp):
    # b_n = P_n + (-1)^n P_0 instead of P_n - (-1)^n P_0 (the initial condition of Sec. I eliminated
    # with the wrong sign); P_0 = 1, so the mistake adds 2 (-1)^n
    def make(orig):
        def b_functions(K, tau):
            b, db = orig(K, tau)
            return b + 2.0 * np.array([(-1.0) ** n for n in range(1, K + 1)])[:, None], db
        return b_functions
    _wrap(mp, tb, "b_functions", make)
    return [(pt.test_ub_closed_form, 3, 0.7), (pt.test_qb_closed_form, 3)]


def qb_derivative_on_test_function(mp):
    def make(orig):
        return lambda K, dt, nquad=None: (lambda m: (m[0], m[1].T, m[2]))(orig(K, dt, nquad))
    _wrap(mp, tb, "static_matrices", make)
    return [(pt.test_qb_closed_form, 4), (ps.test_scalar_matches_symbolic, 3)]


def ub_without_jacobian(mp):
    # int b_m b_n dtau without the dt/2 of dt = (dt/2) dtau
    def make(orig):
        return lambda K, dt, nquad=None: (lambda m: (m[0] * 2.0 / dt, m[1], m[2] * 2.0 / dt))(orig(K, dt, nquad))
    _wrap(mp, tb, "static_matrices", make)
    return [(pt.test_ub_closed_form, 3, 0.7), (ps.test_scalar_K1_closed_form, 0.5)]


def envelope_two_sigma_squared(mp):
    # exp(-(t - tc)^2 / (2 sigma^2)) instead of exp(-((t - tc) / sigma)^2)
    def pulse_field(pulse, t):
        t = np.asarray(t, dtype=np.float64)
        e = np.zeros_like(t)
        for a, w, tc, s in zip(pulse.amp, pulse.omega, pulse.t_center, pulse.sigma):
            e = e + a * (np.exp(-(t - tc) ** 2 / (2 * s * s)) if s > 0 else 1.0) * np.sin(w * t)
        return e
    mp.setattr(tb, "pulse_field", pulse_field)
    return [(pt.test_pulse_field_by_value,), (pt.test_field_matrices_against_adaptive_quadrature, 0.0)]


def carrier_in_time_from_centre(mp):
    # sin(omega (t - tc)) instead of sin(omega t)
    def pulse_field(pulse, t):
        t = np.asarray(t, dtype=np.float64)
        e = np.zeros_like(t)
        for a, w, tc, s in zip(pulse.amp, pulse.omega, pulse.t_center, pulse.sigma):
            e = e + a * (np.exp(-((t - tc) / s) ** 2) if s > 0 else 1.0) * np.sin(w * (t - tc))
        return e
    mp.setattr(tb, "pulse_field", pulse_field)
    return [(pt.test_pulse_field_by_value,), (pt.test_field_matrices_against_adaptive_quadrature, 4.35)]


def step_time_centred_at_t0(mp):
    # t = t0 + tau dt/2 instead of t0 + (tau + 1) dt/2
    def make(orig):
        return lambda K, dt, t0, field, nquad=None: orig(K, dt, t0 - 0.5 * dt, field, nquad)
    _wrap(mp, tb, "field_matrices", make)
    return [(pt.test_field_matrices_constant_and_linear,), (pt.test_field_matrices_against_adaptive_quadrature, 0.0)]


def component_field_keeps_its_amplitude(mp):
    # dE/da_k taken as a_k E_k instead of the unit-amplitude E_k
    def make(orig):
        return lambda pulse, k, t: pulse.amp[k] * orig(pulse, k, t)
    _wrap(mp, tb, "pulse_component_field", make)
    return [(pt.test_pulse_field_by_value,), (pa.test_amplitude_gradient_matches_finite_differences, 1)]


def field_quadrature_too_coarse(mp):
    # K + 1 Gauss nodes for the field matrices: exact for polynomials only, not for the pulses
    def make(orig):
        return lambda K, dt, t0, field, nquad=None: orig(K, dt, t0, field, nquad if nquad else K + 1)
    _wrap(mp, tb, "field_matrices", make)
    return [(pt.test_quadrature_converged_for_pulses,)]


def end_value_without_p0_part(mp):
    # phi(t0 + dt) = psi0 + sum_n c_n, forgetting that b_n(+1) = 1 - (-1)^n
    mp.setattr(tb, "end_values", lambda K: np.ones(K))
    return [(ps.test_scalar_K1_closed_form, 0.5), (pt.test_end_values,)]


# ------------------------------------------------------------------------------ the step's system
def kinetic_without_half(mp):
    _wrap(mp, system, "kinetic", lambda orig: lambda prob: (2.0 * orig(prob)).tocsr())
    return [(ps.test_kkt_with_multipliers, 8, 2, 0.0), (ps.test_eigen_expansion_and_norm_drift,)]


def laplacian_with_neumann_walls(mp):
    # the end rows of the second difference with -1/h^2 (a reflecting wall) instead of Dirichlet's -2/h^2
    def make(orig):
        def second_difference_1d(n, h):
            A = orig(n, h).tolil()
            A[0, 0] = A[n - 1, n - 1] = -1.0 / (h * h)
            return A.tocsr()
        return second_difference_1d
    _wrap(mp, system, "second_difference_1d", make)
    return [(ps.test_laplacian_eigenvalues_on_an_anisotropic_grid,), (ps.test_scalar_K1_closed_form, 0.5)]


def _patch_time_matrices(mp, change):
    def make(orig):
        return lambda prob, t0: change(*orig(prob, t0))
    _wrap(mp, system, "time_matrices", make)


def time_derivative_sign(mp):
    # -i Q instead of i Q in the stationarity rows (Eq. stationaryphase)
    _patch_time_matrices(mp, lambda Ub, Qb, Ub0, Eb, Eb0: (Ub, -Qb, Ub0, Eb, Eb0))
    return [(ps.test_scalar_K1_closed_form, 0.5), (ps.test_kkt_with_multipliers, 8, 2, 0.0)]


def dipole_coupling_sign(mp):
    _patch_time_matrices(mp, lambda Ub, Qb, Ub0, Eb, Eb0: (Ub, Qb, Ub0, -Eb, -Eb0))
    return [(ps.test_kkt_with_multipliers, 8, 2, 0.3)]


def initial_state_field_term_dropped(mp):
    # f without the x_q Eb0 psi0 part of the initial condition
    _patch_time_matrices(mp, lambda Ub, Qb, Ub0, Eb, Eb0: (Ub, Qb, Ub0, Eb, 0.0 * Eb0))
    return [(ps.test_kkt_with_multipliers, 8, 2, 0.3)]


def dual_weight_without_inverse(mp):
    def make(orig):
        def weight_matrix(prob, Ub, weight="dual"):
            if weight == "dual":
                return (sp.kron(sp.identity(prob.npoints), Ub) / prob.vol).tocsr()
            return orig(prob, Ub, weight)
        return weight_matrix
    _wrap(mp, system, "weight_matrix", make)
    return [(ps.test_dual_weight_is_test_basis_invariant,)]


def _patch_weight(mp, name, build):
    def make(orig):
        def weight_matrix(prob, Ub, weight="dual"):
            return build(prob, Ub) if weight == name else orig(prob, Ub, weight)
        return weight_matrix
    _wrap(mp, system, "weight_matrix", make)


def literal_weight_overlap_inverted(mp):
    # O (x) U with the grid overlap h^d divided instead of multiplied
    _patch_weight(mp, "literal", lambda prob, Ub: (sp.kron(sp.identity(prob.npoints), Ub) / prob.vol).tocsr())
    return [(ps.test_weights_are_l2_norms_of_residual_functions, "literal")]


def dual_weight_overlap_inverted(mp):
    # (O (x) U)^{-1} with h^d multiplied instead of divided (the basis invariance holds for any scale)
    _patch_weight(mp, "dual", lambda prob, Ub: (prob.vol * sp.kron(sp.identity(prob.npoints), np.linalg.inv(Ub))).tocsr())
    return [(ps.test_weights_are_l2_norms_of_residual_functions, "dual"), (ps.test_dual_weight_is_test_basis_invariant,)]


def stencil_row_without_potential(mp):
    def make(orig):
        def hamiltonian_row(prob, q):
            cols, vals = orig(prob, q)
            vals = vals.copy()
            vals[0] -= prob.V0[q]
            return cols, vals
        return hamiltonian_row
    _wrap(mp, system, "hamiltonian_row", make)
    return [(ps.test_pointwise_residual_matches_the_assembled_system, "2d")]


def problem_spacings_in_workload_order(mp):
    # Problem.from_workload keeping the workload's x-first spacings on the slowest-first grid
    def make(orig):
        def from_workload(w):
            prob = orig(w)
            prob.h = tuple(reversed(prob.h))
            return prob
        return staticmethod(from_workload)
    mp.setattr(system.Problem, "from_workload", make(system.Problem.from_workload))
    return [(ps.test_problem_from_an_anisotropic_workload_pairs_extents_with_spacings,)]


def laplacian_spacing_on_the_wrong_axis(mp):
    # each axis's second difference divided by another axis's h^2 (the spacings taken in x-first order)
    _wrap(mp, system, "laplacian", lambda orig: lambda shape, h: orig(shape, tuple(reversed(h))))
    return [(ps.test_laplacian_eigenvalues_on_an_anisotropic_grid,)]


def stencil_row_spacing_on_the_wrong_axis(mp):
    def make(orig):
        return lambda prob, q: orig(dataclasses.replace(prob, h=tuple(reversed(prob.h))), q)
    _wrap(mp, system, "hamiltonian_row", make)
    return [(ps.test_stencil_rows_on_an_anisotropic_grid,)]


def action_norm_without_conjugate(mp):
    # r^T W r instead of r^dagger W r (Eq. residnorm)
    mp.setattr(system, "action_norm", lambda r, W: float(np.real(np.dot(r, W @ r))))
    return [(ps.test_action_norm_is_nonnegative_and_zero_at_solution,), (pr.test_block_update_minimises_N_over_the_block,)]


def adjoint_solve_with_transpose(mp):
    # mu_k = M_k^{-T} B^T lambda_{k+1} instead of M_k^{-dagger}: the adjoint module's sparse LU is
    # handed M^T (the conjugate of the M^dagger it is given); the forward solves are untouched
    real = adjoint.spla
    mp.setattr(adjoint, "spla", types.SimpleNamespace(splu=lambda A: real.splu(A.conj().tocsc())))
    return [(pa.test_amplitude_gradient_matches_finite_differences, 1), (pa.test_initial_state_gradient_matches_finite_differences,)]


def dipole_without_overlap(mp):
    # the objective sum_p x_p |psi_p|^2 without h^d, while its derivative keeps it
    mp.setattr(system, "dipole", lambda prob, psi: float(np.sum(prob.xlaser * np.abs(psi) ** 2)))
    return [(pa.test_initial_state_gradient_matches_finite_differences,)]


# ------------------------------------------------------------------------------ relaxation (Sec. II)
def checkerboard_colouring(mp):
    # two colours by the parity of the block-index sum: right for M's radius-1 rows, wrong for the
    # radius-2 normal operator G = M^dagger W M
    def make(orig):
        def subvolumes(shape, sub):
            nb = relax.block_counts(shape, sub)
            out = orig(shape, sub)
            return [(int(sum(np.unravel_index(b, nb))) % 2, pts) for b, (_, pts) in enumerate(out)]
        return subvolumes
    _wrap(mp, relax, "subvolumes", make)
    return [(pr.test_colouring_valid_every_level, "dual")]


def residual_once_per_sweep(mp):
    # every colour updated from the residual taken at the start of the sweep (Jacobi across colours)
    def sweep(self, x, g, after_colour=None):
        s = g - self.G @ x
        updates = [(idx, sla.cho_solve(fac, s[idx])) for _, idx, fac in self.blocks]
        for colour in range(self.ncolours):
            for (col, _, _), (idx, d) in zip(self.blocks, updates):
                if col == colour:
                    x[idx] += d
            if after_colour is not None:
                after_colour(colour)
    mp.setattr(relax.BlockRelaxation, "sweep", sweep)
    return [(pr.test_action_never_increases, "dual"), (pr.test_2d_vcycle_converges_to_direct_solution,)]


def local_solve_with_transpose(mp):
    # G_UU^T (= conj G_UU for the Hermitian G) factored instead of G_UU
    def make(orig):
        def __init__(self, G, shape, sub, K):
            orig(self, G, shape, sub, K)
            self.blocks = [(col, idx, sla.cho_factor(self.G[idx][:, idx].toarray().T, lower=True))
                           for col, idx, _ in self.blocks]
        return __init__
    _wrap(mp, relax.BlockRelaxation, "__init__", make)
    return [(pr.test_single_block_update_is_the_blockwise_minimiser,), (pr.test_block_update_minimises_N_over_the_block,)]


# ------------------------------------------------------------------------------ multigrid (Sec. III)
def interpolation_from_far_neighbour(mp):
    # fine 2J <- 3/4 c_J + 1/4 c_{J+1} (and 2J+1 from c_{J-1}): the 1/4 weight on the wrong side
    def interpolation_1d(nc):
        rows, cols, vals = [], [], []
        for J in range(nc):
            for fi, nb in ((2 * J, J + 1), (2 * J + 1, J - 1)):
                rows.append(fi); cols.append(J); vals.append(0.75)
                if 0 <= nb < nc:
                    rows.append(fi); cols.append(nb); vals.append(0.25)
        return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc, nc))
    mp.setattr(multigrid, "interpolation_1d", interpolation_1d)
    return [(pr.test_fd_interpolation_reproduces_linear_functions,)]


def interpolation_axes_reversed(mp):
    # the 1D factors of the tensor product taken in x-first order while the grid is stored z-first
    def interpolation(coarse_shape, K):
        I = None
        for n in reversed(coarse_shape):
            m = multigrid.interpolation_1d(n)
            I = m if I is None else sp.kron(I, m, format="csr")
        return sp.kron(I, sp.identity(K), format="csr")
    mp.setattr(multigrid, "interpolation", interpolation)
    return [(pr.test_fd_interpolation_reproduces_linear_functions_on_a_box,)]


def coarse_residual_before_presmoothing(mp):
    # the V-cycle restricts the residual taken before its pre-smoothing sweeps instead of after them
    def make(orig):
        def vcycle(self, l, x, g, after_colour=None):
            if self.L == 1 or l == self.L - 1:
                return orig(self, l, x, g, after_colour)
            hook = after_colour if l == 0 else None
            nu1, nu2 = (self.nu1, self.nu2) if l == 0 else self.coarse_nu
            s = g - self.G[l] @ x
            for _ in range(nu1):
                self.relax[l].sweep(x, g, hook)
            xc = np.zeros(self.I[l].shape[1], dtype=x.dtype)
            self.vcycle(l + 1, xc, self.I[l].T @ s)
            x += self.I[l] @ xc
            if after_colour is not None and l == 0:
                after_colour(-1)
            for _ in range(nu2):
                self.relax[l].sweep(x, g, hook)
        return vcycle
    _wrap(mp, multigrid.Hierarchy, "vcycle", make)
    return [(pr.test_action_never_increases, "dual")]


def coarse_operator_quartered(mp):
    # the Galerkin operator I^T G I divided by 4, the factor a rediscretisation on a grid of twice the
    # spacing would carry for the kinetic term: every coarse correction comes out four times too large
    def make(orig):
        def __init__(self, G0, shape0, K, sub, levels, *args, **kw):
            orig(self, G0, shape0, K, sub, levels, *args, **kw)
            for l in range(1, self.L):
                self.G[l] = (0.25 * self.G[l]).tocsr()
                R = self.relax[l]
                R.G = self.G[l]
                R.blocks = [(col, idx, (0.5 * c, low)) for col, idx, (c, low) in R.blocks]   # chol(G/4) = chol(G)/2
        return __init__
    _wrap(mp, multigrid.Hierarchy, "__init__", make)
    return [(pr.test_action_never_increases, "dual")]


# ------------------------------------------------------------------------------ square form, elements, maps
def square_solve_with_transpose(mp):
    def square_block_update(M, f, x, idx):
        M = M.tocsr()
        return np.linalg.solve(M[idx][:, idx].toarray().T, f[idx] - M[idx] @ x)
    mp.setattr(relax, "square_block_update", square_block_update)
    return [(pq.test_square_update_zeroes_the_block_residual,)]


def element_children_swapped(mp):
    # the left child's interpolation rows taken from the right child
    def make(orig):
        def interpolation(nmax):
            E = orig(nmax)
            return np.vstack([E[nmax + 1:], E[:nmax + 1]])
        return interpolation
    _wrap(mp, le, "interpolation", make)
    return [(pr.test_legendre_element_transfers, 3)]


def projection_without_overlap_weights(mp):
    # the unweighted left inverse (E^T E)^{-1} E^T of the interpolation instead of the L2 projection
    # (it too gives P I = identity)
    _wrap(mp, le, "projection", lambda orig: lambda nmax: np.linalg.pinv(le.interpolation(nmax)))
    return [(pr.test_legendre_element_projection_is_the_l2_projection, 3)]


def transfer_restricts_with_the_plain_transpose(mp):
    # the residual taken to the parent element by I^T instead of the projection P
    _wrap(mp, lfa, "parent_transfers", lambda orig: lambda nx, nt: (lambda IP: (IP[0], IP[0].T))(orig(nx, nt)))
    return [(pl.test_transfer_coarse_step_solves_the_projected_problem, 1.0, 0.0),
            (pl.test_maps_follow_sec_v,)]


def lfa_initial_condition_at_the_step_end(mp):
    # the correction held at tau = +1 (P_n(1) = 1) instead of the initial time tau = -1
    def make(orig):
        def constraints(nx, nt, nel, left=True, right=True, initial=True, continuity=True):
            rest = orig(nx, nt, nel, left, right, False, continuity)
            if not initial:
                return rest
            n = nx * nt
            rows = np.zeros((nel * nx, nel * n))
            for e in range(nel):
                for i in range(nx):
                    rows[e * nx + i, e * n + i * nt: e * n + (i + 1) * nt] = 1.0
            return np.vstack([rows, rest.reshape(-1, nel * n)])
        return constraints
    _wrap(mp, lfa, "constraints", make)
    return [(pl.test_correction_vanishes_at_the_initial_time_and_the_volume_ends, "one"),
            (pl.test_relaxation_keeps_initial_and_boundary_values, "one")]


def lfa_action_without_conjugate(mp):
    # S = C^T A C instead of C^H A C
    _wrap(mp, lfa, "measures", lambda orig: lambda A, W, C: (orig(A, W, C)[0], complex(C @ (A @ C))))
    return [(pl.test_action_by_quadrature_of_the_trial_function, 1.0, 0.0)]


def lfa_derivative_on_test_function(mp):
    def make(orig):
        return lambda nx, nt: (lambda m: (m[0], m[1], m[2].T, m[3]))(orig(nx, nt))
    _wrap(mp, lfa, "element_matrices", make)
    return [(pl.test_element_matrices_closed_forms, 3, 3), (pl.test_dimensionless_rows_and_their_scaling, 2.0, 2.0, 0.0)]


def lfa_kinetic_sign(mp):
    _wrap(mp, lfa, "element_operator", lambda orig: lambda nx, nt, kappa, nu: orig(nx, nt, -kappa, nu))
    return [(pl.test_dimensionless_rows_and_their_scaling, 0.3, 0.05, -1.7)]


def lfa_potential_sign(mp):
    # +nu O U in the element rows (the potential term with the wrong sign)
    _wrap(mp, lfa, "element_operator", lambda orig: lambda nx, nt, kappa, nu: orig(nx, nt, kappa, -nu))
    return [(pl.test_dimensionless_rows_and_their_scaling, 0.3, 0.05, -1.7),
            (pl.test_slow_convergence_only_near_the_dispersion_curve,)]


def lfa_weight_inverted(mp):
    # the element weight (O x U)^{-1} instead of the printed O x U
    def weight(nx, nt, nel):
        O, U, _, _ = lfa.element_matrices(nx, nt)
        return np.kron(np.eye(nel), np.kron(np.linalg.inv(O), np.linalg.inv(U)))
    mp.setattr(lfa, "weight", weight)
    return [(pl.test_continuous_projection,)]


def lfa_residual_sign(mp):
    # relaxing with r = +A C instead of the residual -A C of Eq. actionresidual
    solve = lfa.constrained_solve
    mp.setattr(lfa, "relax", lambda A, B, C, solver="null": C + solve(A, B, A @ C, solver))
    return [(pl.test_unconstrained_relaxation_is_the_exact_solve,)]


MUTANTS = [
    # time basis
    b_adds_p0, qb_derivative_on_test_function, ub_without_jacobian, envelope_two_sigma_squared,
    carrier_in_time_from_centre, step_time_centred_at_t0, component_field_keeps_its_amplitude,
    field_quadrature_too_coarse, end_value_without_p0_part,
    # the step's system and its adjoint
    kinetic_without_half, laplacian_with_neumann_walls, time_derivative_sign, dipole_coupling_sign,
    initial_state_field_term_dropped, dual_weight_without_inverse, literal_weight_overlap_inverted,
    dual_weight_overlap_inverted, stencil_row_without_potential, problem_spacings_in_workload_order,
    laplacian_spacing_on_the_wrong_axis,
    stencil_row_spacing_on_the_wrong_axis, action_norm_without_conjugate, adjoint_solve_with_transpose,
    dipole_without_overlap,
    # relaxation and multigrid
    checkerboard_colouring, residual_once_per_sweep, local_solve_with_transpose,
    interpolation_from_far_neighbour, interpolation_axes_reversed, coarse_residual_before_presmoothing,
    coarse_operator_quartered,
    # square form, Legendre elements, plane-wave maps
    square_solve_with_transpose, element_children_swapped, projection_without_overlap_weights,
    transfer_restricts_with_the_plain_transpose, lfa_derivative_on_test_function, lfa_kinetic_sign,
    lfa_potential_sign, lfa_weight_inverted, lfa_residual_sign, lfa_initial_condition_at_the_step_end,
    lfa_action_without_conjugate,
]


def _fails(pin, *args):
    try:
        pin(*args)
    except (AssertionError, np.linalg.LinAlgError):
        return True
    return False


@pytest.mark.parametrize("plant", MUTANTS, ids=[m.__name__ for m in MUTANTS])
def test_a_pin_catches_the_planted_mistake(plant, monkeypatch):
    pins = plant(monkeypatch)
    caught = [pin.__name__ for pin, *args in pins if _fails(pin, *args)]
    assert caught, "no pin fails under the planted mistake: " + ", ".join(p.__name__ for p, *_ in pins)
