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


def test_pulse_field_by_value():
    """E(t) where its value is known without the formula: each envelope is 1 at its centre and
    e^-1 one width sigma away on either side (exp(-((t - tc)/sigma)^2), not exp(-(t - tc)^2/(2 sigma^2))),
    sigma = 0 leaves the bare sin(omega t) of the absolute time t, and components add."""
    import math
    from paper_1111_4363_gb300 import workloads as wl
    amp, om, tc, sg = 0.3, 0.7, 5.0, 2.0
    one = wl.Pulse(amp=[amp], omega=[om], t_center=[tc], sigma=[sg])
    e = tb.pulse_field(one, np.array([tc, tc + sg, tc - sg, tc + 2 * sg]))
    np.testing.assert_allclose(e[0], amp * math.sin(om * tc), rtol=1e-15)
    np.testing.assert_allclose(e[1], amp * math.exp(-1.0) * math.sin(om * (tc + sg)), rtol=1e-14)
    np.testing.assert_allclose(e[2], amp * math.exp(-1.0) * math.sin(om * (tc - sg)), rtol=1e-14)
    np.testing.assert_allclose(e[3], amp * math.exp(-4.0) * math.sin(om * (tc + 2 * sg)), rtol=1e-14)
    bare = wl.Pulse(amp=[amp], omega=[om], t_center=[tc], sigma=[0.0])
    t = np.array([0.0, 0.4, 3.1, 17.25])
    np.testing.assert_allclose(tb.pulse_field(bare, t), amp * np.sin(om * t), rtol=1e-15, atol=1e-17)
    # the 2D workload's field 0.05 sin(0.057 t): zero at t = 0, 0.05 at the first crest t = pi/(2 0.057)
    w2 = wl.softcore_2d(n=32, levels=1)
    crest = math.pi / (2 * 0.057)
    np.testing.assert_allclose(tb.pulse_field(w2.pulse, np.array([0.0, crest])), [0.0, 0.05], atol=1e-16)
    two = wl.Pulse(amp=[amp, -0.2], omega=[om, 1.3], t_center=[tc, 1.0], sigma=[sg, 0.0])
    t = np.linspace(-3.0, 9.0, 13)
    np.testing.assert_allclose(tb.pulse_field(two, t), tb.pulse_field(one, t) - 0.2 * np.sin(1.3 * t), atol=1e-16)
    # the unit-amplitude component fields: E = sum_k amp_k E_k, and each E_k is 1 x its sine at its centre
    w3 = wl.hydrogen_3d(n=8, nsteps=400)
    t = np.linspace(0.0, 20.0, 41)
    parts = sum(a * tb.pulse_component_field(w3.pulse, k, t) for k, a in enumerate(w3.pulse.amp))
    np.testing.assert_allclose(parts, tb.pulse_field(w3.pulse, t), atol=1e-16)
    for k in (0, 7, 31):
        c = w3.pulse.t_center[k]
        np.testing.assert_allclose(tb.pulse_component_field(w3.pulse, k, np.array([c]))[0],
                                   math.sin(w3.pulse.omega[k] * c), rtol=1e-15, atol=1e-17)


@pytest.mark.parametrize("t0", [0.0, 4.35])
def test_field_matrices_against_adaptive_quadrature(t0):
    """Eb and Eb0 of one Gaussian-enveloped component against scipy's adaptive quadrature of
    (dt/2) int b_m b_n E(t(tau)) dtau with t(tau) = t0 + (tau + 1) dt/2, the b_n from scipy's own
    Legendre polynomials: pins the step's time variable as well as the envelope."""
    import math
    from scipy import integrate, special
    from paper_1111_4363_gb300 import workloads as wl
    K, dt = 4, 0.6
    p = wl.Pulse(amp=[0.8], omega=[1.1], t_center=[t0 + 0.2], sigma=[0.35])
    Eb, Eb0 = tb.field_matrices(K, dt, t0, lambda t: tb.pulse_field(p, t))

    def b(n, tau):
        return special.eval_legendre(n, tau) - (-1.0) ** n

    def field(tau):
        t = t0 + 0.5 * (tau + 1.0) * dt
        return 0.8 * math.exp(-((t - (t0 + 0.2)) / 0.35) ** 2) * math.sin(1.1 * t)

    for m in range(1, K + 1):
        ref0 = 0.5 * dt * integrate.quad(lambda x: b(m, x) * field(x), -1, 1, epsabs=1e-15, epsrel=1e-13)[0]
        assert Eb0[m - 1] == pytest.approx(ref0, rel=1e-10, abs=1e-15)
        for n in range(1, K + 1):
            ref = 0.5 * dt * integrate.quad(lambda x: b(m, x) * b(n, x) * field(x), -1, 1,
                                            epsabs=1e-15, epsrel=1e-13)[0]
            assert Eb[m - 1, n - 1] == pytest.approx(ref, rel=1e-10, abs=1e-15), (m, n)
