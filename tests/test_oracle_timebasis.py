"""Pins for the oracle's time basis (closed forms of Sec. IV; Gauss-Legendre quadrature rules)."""
import numpy as np
import pytest

from oracle import timebasis as tb

KS = [1, 2, 3, 4, 6, 8]


@pytest.mark.parametrize("K", KS)
def test_legendre_identities(K):
    # Sec. IV: P_n(1) = 1, P_n'(1) = n(n+1)/2, P_n(-y) = (-1)^n P_n(y)
    y = np.linspace(-1, 1, 7)
    P = tb.legendre_P(K, y)
    dP1 = tb.legendre_dP(K, np.array([1.0]))[:, 0]
    for n in range(K + 1):
        assert tb.legendre_P(K, np.array([1.0]))[n, 0] == pytest.approx(1.0, abs=1e-13)
        assert dP1[n] == pytest.approx(n * (n + 1) / 2, abs=1e-12)
        np.testing.assert_allclose(tb.legendre_P(K, -y)[n], (-1) ** n * P[n], atol=1e-15)


@pytest.mark.parametrize("K", KS)
@pytest.mark.parametrize("dt", [0.05, 0.7])
def test_ub_closed_form(K, dt):
    # Sec. IV orthogonality int P_n P_m = 2 delta/(2n+1)  =>  (dt/2) int b_m b_n = dt (delta/(2m+1) + (-1)^{m+n})
    Ub, _, Ub0 = tb.static_matrices(K, dt)
    m = np.arange(1, K + 1)
    closed = dt * (np.diag(1.0 / (2 * m + 1)) + np.outer((-1.0) ** m, (-1.0) ** m))
    np.testing.assert_allclose(Ub, closed, rtol=0, atol=1e-15 * max(1, dt * K))
    # (dt/2) int b_m P_0 = (dt/2)(0 - (-1)^m 2)
    np.testing.assert_allclose(Ub0, -dt * (-1.0) ** m, atol=1e-15)


@pytest.mark.parametrize("K", KS)
def test_qb_closed_form(K):
    # Sec. IV: int P_n' P_m = 2 if n > m and n - m odd, else 0 (derivative on the trial function n),
    # and int P_0 P_n' = P_n(1) - P_n(-1) = 1 - (-1)^n.
    _, Qb, _ = tb.static_matrices(K, 0.1)
    closed = np.zeros((K, K))
    for m in range(1, K + 1):
        for n in range(1, K + 1):
            q = 2.0 if (n > m and (n - m) % 2 == 1) else 0.0
            closed[m - 1, n - 1] = q - (-1.0) ** m * (1.0 - (-1.0) ** n)
    np.testing.assert_allclose(Qb, closed, atol=1e-13)


def test_field_matrices_constant_and_linear():
    K, dt, t0 = 6, 0.3, 1.7
    Ub, _, Ub0 = tb.static_matrices(K, dt)
    Eb, Eb0 = tb.field_matrices(K, dt, t0, lambda t: 0.37 + 0 * t)
    np.testing.assert_allclose(Eb, 0.37 * Ub, atol=1e-15)
    np.testing.assert_allclose(Eb0, 0.37 * Ub0, atol=1e-15)
    # E(t) = t: t = t0 + (tau+1) dt/2; tau P_m = ((m+1) P_{m+1} + m P_{m-1})/(2m+1) (Bonnet recursion)
    Eb, _ = tb.field_matrices(K, dt, t0, lambda t: t)
    Tau = np.zeros((K + 2, K + 2))          # int tau P_i P_j over the full basis P_0..P_{K+1}
    for i in range(K + 2):
        for j in range(K + 2):
            if j == i + 1:
                Tau[i, j] = 2.0 * (i + 1) / ((2 * i + 1) * (2 * i + 3))
            elif j == i - 1:
                Tau[i, j] = 2.0 * i / ((2 * i - 1) * (2 * i + 1))
    B = np.zeros((K, K + 2))                # b_m = P_m - (-1)^m P_0
    for m in range(1, K + 1):
        B[m - 1, m] = 1.0
        B[m - 1, 0] = -(-1.0) ** m
    closed = (t0 + dt / 2) * Ub + (dt / 2) ** 2 * (B @ Tau @ B.T)
    np.testing.assert_allclose(Eb, closed, atol=1e-14)


def test_quadrature_converged_for_pulses():
    # K + 8 Gauss nodes: doubling them changes the field matrices by < 1e-15 relative (smooth envelopes)
    from paper_1111_4363_gb300 import workloads as wl
    w = wl.hydrogen_3d(n=8, nsteps=400)
    field = lambda t: tb.pulse_field(w.pulse, t)
    for t0 in (0.0, 3.3, 11.9):
        a, a0 = tb.field_matrices(4, 0.05, t0, field)
        b, b0 = tb.field_matrices(4, 0.05, t0, field, nquad=24)
        scale = 0.05 * float(np.sum(np.abs(w.pulse.amp)))   # dt * max |E|
        assert np.max(np.abs(a - b)) <= 1e-15 * scale
        assert np.max(np.abs(a0 - b0)) <= 1e-15 * scale


def test_end_values():
    # phi(t0+dt) weights b_n(1) = 1 - (-1)^n: 2 for odd n, 0 for even n
    np.testing.assert_array_equal(tb.end_values(5), [2, 0, 2, 0, 2])
