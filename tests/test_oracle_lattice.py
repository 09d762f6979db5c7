"""Pins of the oracle's collision, forcing and streaming (Sec. 2).

Closed-form moment identities and exact invariants of the MRT-LBE with Guo
forcing: mass conservation, the momentum gain of rho a per node and step,
and the equilibrium fixed point.
"""
import numpy as np
import pytest

from oracle import params as P
from paper_2012_14707_gb300 import cases


def _feq(rho, ux, uy):
    cu = P.CX * ux + P.CY * uy
    return P.W * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


def test_M_is_orthogonal_and_oracle_inverse_matches(oracle_mod):
    """M M^T = diag(9, 36, 36, 6, 12, 6, 12, 4, 4); the oracle's
    Gauss-Jordan M^-1 equals numpy's inverse of the printed M."""
    np.testing.assert_array_equal(P.M @ P.M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4.0]))
    o = oracle_mod.OracleLBM(cases.periodic_box(3, 3), P.Parameters(0.05, 10.0))
    np.testing.assert_allclose(o.minv(), np.linalg.inv(P.M), atol=1e-15)
    np.testing.assert_allclose(o.minv() @ P.M, np.eye(9), atol=1e-14)


def test_equilibrium_moments_closed_form():
    """M f_eq (Eq. LBEequi) = rho (1, -2 + 3u^2, 1 - 3u^2, ux, -ux, uy, -uy,
    ux^2 - uy^2, ux uy)."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        rho, ux, uy = rng.uniform(0.8, 1.2), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
        u2 = ux * ux + uy * uy
        want = rho * np.array([1, -2 + 3 * u2, 1 - 3 * u2, ux, -ux, uy, -uy, ux * ux - uy * uy, ux * uy])
        np.testing.assert_allclose(P.M @ _feq(rho, ux, uy), want, atol=1e-15)


def test_forcing_moments_closed_form():
    """M Fbar (Eq. LBEforce with c_i) = rho (0, 6u.a, -6u.a, ax, -ax, ay,
    -ay, 2(ux ax - uy ay), ux ay + uy ax); hence sum F = 0, sum c F = rho a."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        ux, uy, ax, ay = rng.uniform(-0.1, 0.1, 4)
        ca = P.CX * ax + P.CY * ay
        cu = P.CX * ux + P.CY * uy
        Fb = P.W * rho * (3 * ca + 9 * (cu * ca - (ux * ax + uy * ay) / 3))
        ua = ux * ax + uy * ay
        want = rho * np.array([0, 6 * ua, -6 * ua, ax, -ax, ay, -ay, 2 * (ux * ax - uy * ay),
                               ux * ay + uy * ax])
        np.testing.assert_allclose(P.M @ Fb, want, atol=1e-16)


def _random_state(nx, ny, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    rho = 1 + amp * rng.standard_normal((ny, nx))
    ux = amp * rng.standard_normal((ny, nx))
    uy = amp * rng.standard_normal((ny, nx))
    f = np.stack([P.W[i] * rho * (1 + 3 * (P.CX[i] * ux + P.CY[i] * uy)
                                  + 4.5 * (P.CX[i] * ux + P.CY[i] * uy) ** 2
                                  - 1.5 * (ux * ux + uy * uy)) for i in range(9)])
    f += amp * 0.1 * rng.standard_normal(f.shape)
    return f


def test_periodic_box_conserves_mass_and_gains_momentum(oracle_mod):
    """Fully periodic box: total mass is conserved and total momentum
    grows by a * (total mass) every step (Guo forcing, Eq. MomentPost)."""
    ax, ay = 2e-5, -1e-5
    case = cases.periodic_box(12, 10, ax=ax, ay=ay)
    o = oracle_mod.OracleLBM(case, P.Parameters(0.05, 10.0))
    f0 = _random_state(12, 10, 3)
    o.set_f(f0)
    m0 = f0.sum()
    jx0 = (P.CX[:, None, None] * f0).sum()
    jy0 = (P.CY[:, None, None] * f0).sum()
    n = 500
    o.step(n)
    f = o.get_f()
    # round-off only: ~1e-16 per node update, random-walk accumulated
    assert f.sum() == pytest.approx(m0, rel=1e-13)
    assert (P.CX[:, None, None] * f).sum() == pytest.approx(jx0 + n * ax * m0, rel=1e-11)
    assert (P.CY[:, None, None] * f).sum() == pytest.approx(jy0 + n * ay * m0, rel=1e-11)
    res, mass = o.residual()
    assert mass == pytest.approx(m0, rel=1e-13)


def test_rest_and_uniform_flow_are_fixed_points(oracle_mod):
    """f = w (rest) and f = f_eq(1, U) (uniform flow) with a = 0 stay
    unchanged: m = m_eq makes the collision the identity."""
    case = cases.periodic_box(6, 5)
    o = oracle_mod.OracleLBM(case, P.Parameters(0.05, 10.0))
    o.step(10)
    np.testing.assert_allclose(o.get_f(), np.broadcast_to(P.W[:, None, None], (9, 5, 6)),
                               rtol=0, atol=4e-16)
    U = (0.03, -0.02)
    feq = _feq(1.0, *U)
    fu = np.broadcast_to(feq[:, None, None], (9, 5, 6)).copy()
    o.set_f(fu)
    o.step(50)
    np.testing.assert_allclose(o.get_f(), fu, rtol=0, atol=1e-14)  # 50 steps of round-off
    assert o.residual()[0] < 1e-13


def test_streaming_moves_populations_along_c(oracle_mod):
    """With every relaxation time 1 and no force the collision maps f to
    f_eq(rho, u); a single step then moves f_eq_i(x) to x + c_i."""
    case = cases.periodic_box(7, 6)
    par = P.Parameters(0.05, 10.0, tau_s=1.0, tau_q_fixed=1.0, tau_e=1.0, tau_eps=1.0)
    o = oracle_mod.OracleLBM(case, par)
    f0 = _random_state(7, 6, 9)
    o.set_f(f0)
    o.step(1)
    rho = f0.sum(0)
    ux = (P.CX[:, None, None] * f0).sum(0) / rho
    uy = (P.CY[:, None, None] * f0).sum(0) / rho
    want = np.empty_like(f0)
    for i in range(9):
        fe = P.W[i] * rho * (1 + 3 * (P.CX[i] * ux + P.CY[i] * uy)
                             + 4.5 * (P.CX[i] * ux + P.CY[i] * uy) ** 2 - 1.5 * (ux * ux + uy * uy))
        want[i] = np.roll(np.roll(fe, int(P.CX[i]), axis=1), int(P.CY[i]), axis=0)
    np.testing.assert_allclose(o.get_f(), want, atol=1e-15)


def test_rejects_bad_links(oracle_mod):
    """A missing link, a link into fluid or gamma outside (0, 1] is refused."""
    case = cases.channel(4, 6, 0.5, 0.5, Kn=0.05)
    par = P.Parameters(0.05, 6.0)
    import dataclasses
    bad = dataclasses.replace(case, link_x=case.link_x[1:], link_y=case.link_y[1:],
                              link_dir=case.link_dir[1:], link_q=case.link_q[1:],
                              link_ubx=case.link_ubx[1:], link_uby=case.link_uby[1:])
    with pytest.raises(ValueError):
        oracle_mod.OracleLBM(bad, par)
    q = case.link_q.copy()
    q[0] = 0.0
    with pytest.raises(ValueError):
        oracle_mod.OracleLBM(dataclasses.replace(case, link_q=q), par)
    d = case.link_dir.copy()
    d[0] = 4 if d[0] != 4 else 2
    with pytest.raises(ValueError):
        oracle_mod.OracleLBM(dataclasses.replace(case, link_dir=d), par)


@pytest.mark.parametrize("threads", [2, 5])
def test_openmp_build_is_bitwise_the_single_threaded_one(oracle_mod, threads):
    """The OpenMP build (row loops over threads) and the single-threaded build
    of the same source give bitwise the same states, residual and mass: a
    cylinder array and an annulus with a moving wall, from a perturbed state."""
    import math

    from paper_2012_14707_gb300 import cases
    for c in (cases.cylinder_array(90, 60, 2, Kn=0.02, ax=1e-5),
              cases.annulus(40, 8.0, 16.0, 0.05, 0.05 * math.sqrt(1 / 3) / 8)):
        par = P.Parameters(c.Kn, c.H, L1=1.0, L2=0.0)
        f0 = cases.random_populations(c.nx, c.ny, 3)
        one = oracle_mod.OracleLBM(c, par)
        many = oracle_mod.OracleLBM(c, par, threads=threads)
        assert one.threads == 1 and many.threads == threads
        for o in (one, many):
            o.set_f(f0)
            o.step(57)
        np.testing.assert_array_equal(many.get_f(), one.get_f())
        assert many.residual() == one.residual()


def test_residuals_of_a_uniformly_accelerating_box(oracle_mod):
    """A periodic box from rest under a body force a: u^n = (n + 1/2) a at
    every node (j gains rho a per step; Eq. FluidMacr adds a / 2), so the
    one-step residual after n steps is 1 / (n + 1/2) and the interval
    residual over steps m..n is (n - m) |a| / ((n - m) (n + 1/2) |a|), the
    same value; a second call with no step in between gives 0."""
    c = cases.periodic_box(9, 5, ax=3e-6, ay=-2e-6)
    o = oracle_mod.OracleLBM(c, P.Parameters(c.Kn, c.H))
    o.step(1)
    assert o.residual()[0] == pytest.approx(1 / 1.5, rel=1e-9)
    assert o.residual_interval() == pytest.approx(1 / 1.5, rel=1e-9)
    o.step(40)
    assert o.residual()[0] == pytest.approx(1 / 41.5, rel=1e-9)
    assert o.residual_interval() == pytest.approx(1 / 41.5, rel=1e-9)
    assert o.residual_interval() == 0.0
    # set_f makes the new state the reference
    o.set_f(o.get_f())
    o.step(7)
    assert o.residual_interval() == pytest.approx(1 / 48.5, rel=1e-9)
