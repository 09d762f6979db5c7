"""Pins of the oracle's parameter formulas (Sec. 3.B) against each other and
against the slip law they are built to realise.

Each identity links two equations the paper prints separately, so a
transcription slip in either (a dropped term, a wrong sign or index) breaks
it.
"""
import math

import numpy as np
import pytest

from oracle import params as P

RNG = np.random.default_rng(1234)
GAMMAS = RNG.uniform(0.01, 1.0, 64)
TAUS = [0.55, 0.8, 1.2, 1.6056, 2.6973, 5.0]


@pytest.mark.parametrize("tau_s", TAUS)
@pytest.mark.parametrize("sigma", [1.0, 0.7])
def test_uniform_tau_q_equals_general_formula(tau_s, sigma):
    """Eq. NSliCoertstq = Eq. SliCoeffrtstq at l from Eq. Eqexlva, for any gamma."""
    L1, L2 = P.slip_coefficients(sigma)
    for E in (-0.65, -0.3, 0.2):
        l = P.l_of_gamma(GAMMAS, tau_s, L1, E)
        tq = P.tau_q_general(l, GAMMAS, tau_s, L1, L2)
        np.testing.assert_allclose(tq, P.tau_q_uniform(tau_s, L1, L2, E), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("tau_s", TAUS)
def test_r_of_gamma_equals_general_formula(tau_s):
    """Eq. NSliCoertsr = Eq. SliCoeffrtsr at l from Eq. Eqexlva."""
    L1, _ = P.slip_coefficients(1.0)
    for E in (-0.65, 0.1):
        l = P.l_of_gamma(GAMMAS, tau_s, L1, E)
        np.testing.assert_allclose(P.r_of_gamma(GAMMAS, tau_s, L1, E), P.r_general(l, tau_s, L1),
                                   rtol=1e-13)


@pytest.mark.parametrize("Kn", [0.001, 0.02, 0.05, 0.1])
def test_tuned_parameters_realise_the_slip_law(Kn):
    """Eq. NumeriSlip with r (Eq. SliCoeffrtsr) and tau_q (Eq. SliCoeffrtstq)
    equals Eq. PhyscPoiSlip for any (l, gamma)."""
    L1, L2 = P.slip_coefficients(1.0)
    for H in (4.0, 16.5, 31.8, 60.0):
        ts = P.tau_s_from_kn(Kn, H)
        l = RNG.uniform(-0.3, 1.5, GAMMAS.shape)
        r = P.r_general(l, ts, L1)
        tq = P.tau_q_general(l, GAMMAS, ts, L1, L2)
        us = P.slip_velocity_kn(r, l, GAMMAS, ts, tq, Kn)
        np.testing.assert_allclose(us, P.slip_velocity_physical(L1, L2, Kn), rtol=1e-11)


def test_eqmislip_equals_kn_form():
    """Eq. EqMiSlip with delta_x/H from Eq. tKnrela equals Eq. NumeriSlip."""
    for _ in range(200):
        r, l, g = RNG.uniform(0.2, 1.0), RNG.uniform(-0.4, 2.0), RNG.uniform(0.01, 1.0)
        tq, Kn, H = RNG.uniform(0.55, 3.0), RNG.uniform(0.001, 0.2), RNG.uniform(3, 80)
        ts = P.tau_s_from_kn(Kn, H)
        a = P.slip_velocity_numeric(r, l, g, ts, tq, H)
        b = P.slip_velocity_kn(r, l, g, ts, tq, Kn)
        assert a == pytest.approx(b, rel=1e-11, abs=1e-14)


def test_wall_recursion_with_parabola_gives_eqmislip():
    """Put the slip parabola Eq. OrSnumve into u_1 = A u_0 + B a + C u_w
    (Eq. NumerSana, Eq. u1u0Coeff) and solve for u_s: it must equal
    Eq. EqMiSlip (nu from Eq. EqViscos, u_c = a H^2 / 8 nu)."""
    for _ in range(200):
        r, l, g = RNG.uniform(0.2, 1.0), RNG.uniform(-0.4, 2.0), RNG.uniform(0.01, 1.0)
        ts, tq, H = RNG.uniform(0.6, 4.0), RNG.uniform(0.55, 3.0), RNG.uniform(3, 80)
        a = 1e-6
        nu = P.viscosity(ts)
        uc = a * H * H / (8 * nu)
        A, B, C = P.wall_recursion_coefficients(r, l, g, ts, tq)
        p0 = 4 * uc * g / H * (1 - g / H)
        p1 = 4 * uc * (1 + g) / H * (1 - (1 + g) / H)
        # p1 + us = A (p0 + us) + B a   (u_w = 0)
        us = (A * p0 + B * a - p1) / (1 - A)
        assert us / uc == pytest.approx(P.slip_velocity_numeric(r, l, g, ts, tq, H), rel=1e-8)


def test_halfway_dbb_parameters_are_the_l0_gamma_half_case():
    """Eq. SliCoeffHar / Eq. SliCoeffHata are Eq. SliCoeffrtsr /
    Eq. SliCoeffrtstq at l = 0, gamma = 1/2."""
    L1, L2 = P.slip_coefficients(1.0)
    for ts in TAUS:
        assert P.r_halfway(ts, L1) == pytest.approx(P.r_general(0.0, ts, L1), rel=1e-14)
        assert P.tau_q_halfway(ts, L1, L2) == pytest.approx(
            P.tau_q_general(0.0, 0.5, ts, L1, L2), rel=1e-13)
        assert P.tau_q_l0(0.5, ts, L1, L2) == pytest.approx(P.tau_q_halfway(ts, L1, L2), rel=1e-13)


def test_E_bound_is_the_tau_q_half_threshold():
    """Eq. EqECond: tau_q of Eq. NSliCoertstq equals 1/2 exactly at E_max,
    exceeds it below."""
    for sigma in (1.0, 0.8):
        L1, L2 = P.slip_coefficients(sigma)
        for ts in TAUS:
            Em = P.E_upper_bound(ts, L1, L2)
            assert P.tau_q_uniform(ts, L1, L2, Em) == pytest.approx(0.5, abs=1e-12)
            assert P.tau_q_uniform(ts, L1, L2, Em - 0.05) > 0.5
            assert P.tau_q_uniform(ts, L1, L2, Em + 0.05) < 0.5


def test_no_slip_limit():
    """L1 = L2 = 0 (Sec. 3.B, first comment): r = 1 and
    tau_q = -3E/2 - 1/4; halfway bounce-back at the magic value
    (tau_s - 1/2)(tau_q - 1/2) = 3/16 for gamma = 1/2, l = 0."""
    for ts in TAUS:
        for E in (-0.65, -0.9):
            np.testing.assert_allclose(P.r_of_gamma(GAMMAS, ts, 0.0, E), 1.0, rtol=1e-15)
            assert P.tau_q_uniform(ts, 0.0, 0.0, E) == pytest.approx(-1.5 * E - 0.25, rel=1e-14)
        tq = P.tau_q_general(0.0, 0.5, ts, 0.0, 0.0)
        assert (ts - 0.5) * (tq - 0.5) == pytest.approx(3.0 / 16.0, rel=1e-13)


def test_slip_coefficients_and_E_policy():
    """Sec. 4: sigma = 1 gives L1 = 0.8183, L2 = 1/pi + L1^2/2; the E policy
    keeps tau_q > 1/2 for every case."""
    L1, L2 = P.slip_coefficients(1.0)
    assert L1 == pytest.approx(0.8183, abs=1e-15)
    assert L2 == pytest.approx(1 / math.pi + 0.5 * 0.8183 ** 2, abs=1e-15)
    for Kn in (0.001, 0.01, 0.05, 0.1):
        for H in (8, 31.8, 60, 400):
            par = P.Parameters(Kn, H)
            assert par.tau_q > 0.5
            assert par.E <= -0.65
            parc = P.Parameters(Kn, H, L1=1.0, L2=0.0)
            assert parc.tau_q > 0.5


def test_l_clamp():
    """Sec. 3.B: l := 0 where Eq. Eqexlva gives l < -0.4, r follows Eq.
    SliCoeffrtsr with that l."""
    par = P.Parameters(0.01, 60.0, L1=1.0, L2=0.0)
    g = np.array([1e-6, 0.01, 0.05, 0.3, 0.9])
    raw = P.l_of_gamma(g, par.tau_s, par.L1, par.E)
    r, l = par.per_link(g)
    np.testing.assert_array_equal(l, np.where(raw < -0.4, 0.0, raw))
    np.testing.assert_allclose(r, P.r_general(l, par.tau_s, par.L1), rtol=1e-15)
    unclamped = raw >= -0.4
    np.testing.assert_allclose(r[unclamped], P.r_of_gamma(g[unclamped], par.tau_s, par.L1, par.E),
                               rtol=1e-13)
