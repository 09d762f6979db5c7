"""Pins of the oracle's boundary scheme (Eq. EqNewBDSC) against the paper's
closed forms for flows it solves exactly (Sec. 3.B, Sec. 4.A.1) and against
the analytic cylindrical Couette solution (Sec. 4.B, to within
discretisation error).

The steady channel solutions are exact up to O(Ma^2) (compressible
equilibrium), so the tolerances sit far below any first-order effect of a
wrong coefficient, sign or index.
"""
import math

import numpy as np
import pytest

from oracle import params as P
from paper_2012_14707_gb300 import cases


def _profile(o, m):
    rho, ux, uy = o.fields()
    return ux[1:m + 1, 0], uy[1:m + 1, 0], rho[1:m + 1, 0]


def test_halfway_bounce_back_magic_parameter_is_exact(oracle_mod):
    """r = 1, l = 0, gamma = 1/2 is halfway bounce-back (Remarks 1-2); with
    (tau_s - 1/2)(tau_q - 1/2) = 3/16 the no-slip parabola is exact and mass
    is conserved."""
    m = 16
    c = cases.channel(4, m, 0.5, 0.5, Kn=0.05, ax=1e-6)
    ts = 1.3
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=0.5 + 3 / 16 / (ts - 0.5),
                       l_mode="zero", r_fixed=1.0)
    o = oracle_mod.OracleLBM(c, par)
    m0 = o.residual()[1]
    o.run_to(1e-12, 100000)
    ux, uy, _ = _profile(o, m)
    y = np.arange(m) + 0.5
    want = c.ax / (2 * P.viscosity(ts)) * y * (c.H - y)
    np.testing.assert_allclose(ux, want, rtol=1e-8)
    assert np.abs(uy).max() < 1e-12
    # exact in exact arithmetic; ~1e5 steps of FP64 round-off here
    assert o.residual()[1] == pytest.approx(m0, rel=1e-10)


@pytest.mark.parametrize("gb,gt", [(0.5, 0.75), (1.0, 0.55), (0.7, 0.7)])
def test_zhao_no_slip_limit_is_exact(oracle_mod, gb, gt):
    """L1 = L2 = 0 (Sec. 3.B): r = 1, l from Eq. Eqexlva and
    tau_q = -3E/2 - 1/4 give the no-slip parabola with walls at distance
    gamma from the first and last fluid rows.  (Distance ratios with l >= 0:
    with r = 1 a negative l grows unstable in this channel.)"""
    m = 12
    c = cases.channel(4, m, gb, gt, Kn=0.05, ax=1e-6)
    par = P.Parameters(0.0, c.H, tau_s=1.4, L1=0.0, L2=0.0, E=-0.52)
    assert par.tau_q == pytest.approx(-1.5 * -0.52 - 0.25)
    assert (par.per_link(np.array([gb, gt]))[1] >= 0).all()
    o = oracle_mod.OracleLBM(c, par)
    o.run_to(1e-12, 200000)
    ux, _, _ = _profile(o, m)
    y = np.arange(m) + gb
    want = c.ax / (2 * P.viscosity(1.4)) * y * (c.H - y)
    np.testing.assert_allclose(ux, want, rtol=1e-7)


@pytest.mark.parametrize("r,l,g,ts,tq", [
    (0.6, 0.0, 0.5, 1.2, 1.2),
    (0.7, 0.3, 0.25, 1.2, 1.2),
    (0.45, 0.8, 0.9, 2.0, 0.9),
    (0.85, 0.1, 0.15, 0.9, 1.4),
])
def test_untuned_slip_matches_eqmislip(oracle_mod, r, l, g, ts, tq):
    """Any (r, l, gamma, tau_s, tau_q), equal gamma on both walls
    (Fig. 4 setup): the steady profile is the parabola plus the slip of
    Eq. EqMiSlip, at every node."""
    m = 16
    c = cases.channel(4, m, g, g, Kn=0.05, ax=1e-6)
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=tq, l_mode=l, r_fixed=r)
    o = oracle_mod.OracleLBM(c, par)
    o.run_to(1e-12, 400000)
    ux, _, _ = _profile(o, m)
    uc = c.ax * c.H ** 2 / (8 * P.viscosity(ts))
    want = P.poiseuille_profile(np.arange(m) + g, c.H, uc,
                                P.slip_velocity_numeric(r, l, g, ts, tq, c.H))
    np.testing.assert_allclose(ux / uc, want / uc, rtol=0, atol=2e-8)


def test_tuned_slip_poiseuille_4x32(oracle_mod):
    """Tuned parameters (Eqs. Eqexlva-NSliCoertstq, E = -0.65), gamma 0.5
    below and 0.3 above, Kn = 0.05: the profile is Eq. numvelo."""
    c = cases.config_poiseuille()
    par = P.Parameters(c.Kn, c.H)
    o = oracle_mod.OracleLBM(c, par)
    o.run_to(1e-12, 200000)
    ux, _, _ = _profile(o, 32)
    uc = c.ax * c.H ** 2 / (8 * P.viscosity(par.tau_s))
    Us = P.slip_velocity_physical(par.L1, par.L2, c.Kn)
    want = P.poiseuille_profile(np.arange(32) + 0.5, c.H, uc, Us)
    np.testing.assert_allclose(ux / uc, want / uc, rtol=0, atol=1e-8)


@pytest.mark.parametrize("Kn", [0.02, 0.1])
def test_tuned_slip_with_four_nodes(oracle_mod, Kn):
    """Sec. 4.A.1 (Fig. 5): gamma = 1/2 and l = gamma with r, tau_q from
    Eqs. SliCoeffrtsr-SliCoeffrtstq reproduce Eq. numvelo even with four
    fluid rows."""
    m = 4
    c = cases.channel(4, m, 0.5, 0.5, Kn=Kn, ax=1e-6)
    ts = P.tau_s_from_kn(Kn, c.H)
    L1, L2 = P.slip_coefficients(1.0)
    par = P.Parameters(Kn, c.H, l_mode="gamma", tau_q_fixed=P.tau_q_general(0.5, 0.5, ts, L1, L2))
    o = oracle_mod.OracleLBM(c, par)
    o.run_to(1e-12, 200000)
    ux, _, _ = _profile(o, m)
    uc = c.ax * c.H ** 2 / (8 * P.viscosity(ts))
    want = P.poiseuille_profile(np.arange(m) + 0.5, c.H, uc, P.slip_velocity_physical(L1, L2, Kn))
    np.testing.assert_allclose(ux / uc, want / uc, rtol=0, atol=1e-8)


@pytest.mark.parametrize("r,l,g", [(0.6, 0.2, 0.5), (0.8, 0.4, 0.3)])
def test_moving_wall_matches_wall_recursion(oracle_mod, r, l, g):
    """Plane Couette flow (a = 0, lower wall at rest, upper wall at U): the
    steady profile is linear, u = alpha + beta y, and at each wall row
    u_1 = A u_0 + C u_w with A, C of Eq. u1u0Coeff.  This pins the wall
    velocity term of Eq. EqNewBDSC."""
    m, U = 10, 1e-4  # small U keeps the O(Ma^2) compressibility error below 1e-9
    c = cases.channel(4, m, g, g, Kn=0.05, ax=0.0, u_top=U)
    ts, tq = 1.3, 1.1
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=tq, l_mode=l, r_fixed=r)
    o = oracle_mod.OracleLBM(c, par)
    o.run_to(1e-13, 400000)
    ux, _, _ = _profile(o, m)
    A, _, C = P.wall_recursion_coefficients(r, l, g, ts, tq)
    # bottom: y0 = g, y1 = 1 + g, u_w = 0; top (mirrored): y0 = H - g, y1 = H - 1 - g, u_w = U
    H = c.H
    M = np.array([[1 - A, (1 + g) - A * g],
                  [1 - A, (H - 1 - g) - A * (H - g)]])
    alpha, beta = np.linalg.solve(M, [0.0, C * U])
    want = alpha + beta * (np.arange(m) + g)
    np.testing.assert_allclose(ux / U, want / U, rtol=0, atol=2e-9)


def _steady_channel_from_wall_relations(H, g_bot, g_top, nu, a, rel_bot, rel_top, uw_bot, uw_top):
    """(alpha, beta, kappa) of u(y) = alpha + beta y + kappa y^2, y from the
    lower wall: kappa = -a / (2 nu) is the bulk (the MRT rows reproduce
    u_{j+1} - 2 u_j + u_{j-1} = -a / nu exactly), and alpha, beta follow
    from the relation u_1 = A u_0 + B a + C u_w at each wall row (the upper
    wall mirrored, y -> H - y)."""
    kappa = -a / (2 * nu)
    rows, rhs = [], []
    for (A, B, C), y0, y1, uw in ((rel_bot, g_bot, 1 + g_bot, uw_bot),
                                  (rel_top, H - g_top, H - 1 - g_top, uw_top)):
        rows.append([1 - A, y1 - A * y0])
        rhs.append(B * a + C * uw - kappa * (y1 * y1 - A * y0 * y0))
    alpha, beta = np.linalg.solve(np.array(rows), np.array(rhs))
    return alpha, beta, kappa


def test_printed_reading_coefficient_of_the_measured_case():
    """r = 0.6, l = 0, gamma = 1/2, tau_s = 1.2: the printed reading gives
    A' = 67/27 where Eq. u1u0Coeff gives 19/9; B is the same."""
    A, B, C = P.wall_recursion_coefficients(0.6, 0.0, 0.5, 1.2, 1.1)
    Ap, Bp, Cp = P.wall_recursion_coefficients_printed(0.6, 0.0, 0.5, 1.2, 1.1)
    assert A == pytest.approx(19 / 9, rel=1e-14)
    assert Ap == pytest.approx(67 / 27, rel=1e-14)
    assert Bp == B and A + C == pytest.approx(1.0) and Ap + Cp == pytest.approx(1.0)


@pytest.mark.parametrize("r,l,g", [(0.6, 0.0, 0.5), (0.6, 0.2, 0.5), (0.8, 0.4, 0.3),
                                   (0.45, 0.9, 0.85)])
def test_printed_reading_plane_couette_matches_its_wall_recursion(oracle_mod, r, l, g):
    """Maxwell part at the wall velocity (diffuse_mode 1, Eq. EqNewBDSC as
    printed), plane Couette flow (a = 0, upper wall at U): the steady linear
    profile satisfies u_1 = A' u_0 + C' u_w at each wall row, node by node,
    and misses the relation of Eq. u1u0Coeff (so a slip in the Maxwell term's
    velocity, sign or weight fails here)."""
    m, U = 10, 1e-4
    c = cases.channel(4, m, g, g, Kn=0.05, ax=0.0, u_top=U)
    ts, tq = 1.3, 1.1
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=tq, l_mode=l, r_fixed=r)
    o = oracle_mod.OracleLBM(c, par, diffuse_mode=1)
    o.run_to(1e-13, 400000)
    ux, _, _ = _profile(o, m)
    y = np.arange(m) + g
    rel = P.wall_recursion_coefficients_printed(r, l, g, ts, tq)
    al, be, _ = _steady_channel_from_wall_relations(c.H, g, g, P.viscosity(ts), 0.0, rel, rel, 0.0, U)
    np.testing.assert_allclose(ux / U, (al + be * y) / U, rtol=0, atol=2e-9)
    rel0 = P.wall_recursion_coefficients(r, l, g, ts, tq)
    al0, be0, _ = _steady_channel_from_wall_relations(c.H, g, g, P.viscosity(ts), 0.0, rel0, rel0, 0.0,
                                                      U)
    assert np.abs(ux - (al0 + be0 * y)).max() / U > 1e-3


@pytest.mark.parametrize("r,l,g,ts,tq", [
    (0.6, 0.0, 0.5, 1.2, 1.2),
    (0.7, 0.3, 0.25, 1.2, 1.2),
    (0.45, 0.8, 0.9, 2.0, 0.9),
    (0.85, 0.1, 0.15, 0.9, 1.4),
])
def test_printed_reading_untuned_poiseuille_matches_its_wall_recursion(oracle_mod, r, l, g, ts, tq):
    """diffuse_mode 1, force-driven channel with walls at rest, any
    (r, l, gamma, tau_s, tau_q): the steady profile is the bulk parabola
    whose wall rows satisfy u_1 = A' u_0 + B a, at every node.  (With the
    walls at rest the printed Maxwell part is w_i rho_f: no momentum enters
    through it, which is why A' exceeds A.)"""
    m = 16
    c = cases.channel(4, m, g, g, Kn=0.05, ax=1e-6)
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=tq, l_mode=l, r_fixed=r)
    o = oracle_mod.OracleLBM(c, par, diffuse_mode=1)
    o.run_to(1e-12, 400000)
    ux, _, _ = _profile(o, m)
    nu = P.viscosity(ts)
    uc = c.ax * c.H ** 2 / (8 * nu)
    rel = P.wall_recursion_coefficients_printed(r, l, g, ts, tq)
    al, be, ka = _steady_channel_from_wall_relations(c.H, g, g, nu, c.ax, rel, rel, 0.0, 0.0)
    y = np.arange(m) + g
    np.testing.assert_allclose(ux / uc, (al + be * y + ka * y * y) / uc, rtol=0, atol=2e-8)


@pytest.mark.parametrize("mode", [0, 1])
def test_force_and_moving_wall_with_unequal_walls(oracle_mod, mode):
    """Both readings with a force, a moving upper wall and different gamma,
    l, r on the two walls (the tuned Sec. 3.B parameters): the steady
    profile follows the parabola fixed by each wall's own relation --
    Eq. u1u0Coeff for the default reading, A', B, C' for the printed one."""
    m, U = 12, 2e-5
    gb, gt = 0.35, 0.8
    c = cases.channel(4, m, gb, gt, Kn=0.03, ax=1e-6, u_top=U)
    par = P.Parameters(c.Kn, c.H)
    o = oracle_mod.OracleLBM(c, par, diffuse_mode=mode)
    o.run_to(1e-13, 400000)
    ux, _, _ = _profile(o, m)
    (rb, rt), (lb, lt) = par.per_link(np.array([gb, gt]))
    fn = P.wall_recursion_coefficients_printed if mode else P.wall_recursion_coefficients
    nu = P.viscosity(par.tau_s)
    al, be, ka = _steady_channel_from_wall_relations(
        c.H, gb, gt, nu, c.ax, fn(rb, lb, gb, par.tau_s, par.tau_q), fn(rt, lt, gt, par.tau_s, par.tau_q),
        0.0, U)
    y = np.arange(m) + gb
    uc = c.ax * c.H ** 2 / (8 * nu)
    np.testing.assert_allclose(ux / uc, (al + be * y + ka * y * y) / uc, rtol=0, atol=2e-8)


def test_literal_reading_differs_only_when_r_below_one(oracle_mod):
    """The two readings of the Maxwell part coincide for r = 1 (no Maxwell
    part) and differ otherwise."""
    m = 8
    c = cases.channel(4, m, 0.4, 0.6, Kn=0.05, ax=1e-6)
    outs = {}
    for r in (1.0, 0.7):
        for mode in (0, 1):
            par = P.Parameters(c.Kn, c.H, tau_s=1.2, tau_q_fixed=1.1, l_mode=0.3, r_fixed=r)
            o = oracle_mod.OracleLBM(c, par, diffuse_mode=mode)
            o.step(300)
            outs[(r, mode)] = o.get_f()
    np.testing.assert_array_equal(outs[(1.0, 0)], outs[(1.0, 1)])
    assert np.abs(outs[(0.7, 0)] - outs[(0.7, 1)]).max() > 1e-9


def _couette_error(oracle_mod, n, R1, R2, Kn, L1=1.0, mode=0):
    om = 0.01 * math.sqrt(1 / 3) / R1
    c = cases.annulus(n, R1, R2, Kn, om, 0.0)
    par = P.Parameters(Kn, c.H, L1=L1, L2=0.0)
    o = oracle_mod.OracleLBM(c, par, diffuse_mode=mode)
    o.run_to(1e-11, 200000)
    rho, ux, uy = o.fields()
    cc = c.meta["center"]
    yy, xx = np.mgrid[0:n, 0:n]
    dx, dy = xx - cc, yy - cc
    rr = np.hypot(dx, dy)
    fl = c.solid == 0
    ut = (-dy * ux + dx * uy) / np.where(rr > 0, rr, 1)
    ua = P.couette_profile(rr, R1, R2, om, 0.0, Kn * (R2 - R1))
    ua0 = P.couette_profile(rr, R1, R2, om, 0.0, 0.0)
    nrm = np.sqrt((ua[fl] ** 2).sum())
    return (np.sqrt(((ut - ua)[fl] ** 2).sum()) / nrm, np.sqrt(((ut - ua0)[fl] ** 2).sum()) / nrm)


def test_couette_slip_solution(oracle_mod):
    """Cylindrical Couette flow (Eq. EqAnaMicro, sigma = 1, L1 = 1, L2 = 0):
    at Kn = 0.01 the tangential velocity is within 1 % (rel. L2) of the slip
    solution; at Kn = 0.05 within 3 %, and well closer to it than to the
    no-slip solution."""
    e_slip, _ = _couette_error(oracle_mod, 72, 16, 32, 0.01)
    assert e_slip < 0.01
    e_slip, e_noslip = _couette_error(oracle_mod, 40, 8, 16, 0.05)
    assert e_slip < 0.03
    assert e_noslip > 2.5 * e_slip
