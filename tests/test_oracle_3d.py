"""Pins of the D3Q19 oracle (the three-dimensional extension the paper names
as future work, Sec. 5).

The paper derives its boundary scheme and parameters in two dimensions.  The
same channel analysis (Sec. 3.B, Eqs. EqMicroBound -> NumerSana) carried out
for D3Q19 -- flow u_x(z) between walls normal to z -- involves the x-odd
moments j_x, q_x, p_xz and the third-order m_x, and reaches exactly the wall
relation of Eq. u1u0Coeff when m_x relaxes with tau_q.  With that choice the
two-dimensional closed forms (Eq. numvelo, Eq. EqMiSlip, the plane Couette
relation, and the printed reading's relation) pin the 3-D oracle node by
node; with another relaxation time of m they do not.
"""
import numpy as np
import pytest

from oracle import params as P
from paper_2012_14707_gb300 import cases


def test_d3q19_lattice_and_moment_basis(oracle_mod):
    c, w = oracle_mod.d3q19_lattice()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose((w[:, None] * c).sum(0), 0.0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-15)
    # fourth moments of the isotropic lattice: sum w c_a^4 = 1/3, c_a^2 c_b^2 = 1/9
    assert (w * c[:, 0] ** 4).sum() == pytest.approx(1 / 3)
    assert (w * c[:, 0] ** 2 * c[:, 1] ** 2).sum() == pytest.approx(1 / 9)
    # the velocities as the case generator numbers them
    np.testing.assert_array_equal(c, cases.C3)
    o = oracle_mod.OracleLBM3D(cases.periodic_box3d(3, 3, 3), P.Parameters(0.05, 3.0))
    M = o.moment_matrix()
    G = M @ M.T
    np.testing.assert_allclose(G - np.diag(np.diag(G)), 0.0, atol=1e-12)
    # M f_eq(rho, 0) = rho (1, -11, 3, 0, ...)
    meq = M @ (w * 1.3)
    np.testing.assert_allclose(meq[:3], [1.3, -11 * 1.3, 3 * 1.3], rtol=1e-13)
    np.testing.assert_allclose(meq[3:], 0.0, atol=1e-13)


def test_accelerating_box_conserves_mass_and_gains_momentum(oracle_mod):
    """Periodic box under a body force: mass stays, u^n = (n + 1/2) a at every
    node (Eq. FluidMacr and Guo forcing)."""
    a = (2e-6, -1e-6, 3e-6)
    c = cases.periodic_box3d(4, 3, 5, a=a)
    o = oracle_mod.OracleLBM3D(c, P.Parameters(0.05, 3.0))
    m0 = o.residual()[1]
    o.step(30)
    rho, ux, uy, uz = o.fields()
    assert o.residual()[1] == pytest.approx(m0, rel=1e-14)
    for u, ai in zip((ux, uy, uz), a):
        np.testing.assert_allclose(u, 30.5 * ai, rtol=1e-9)


def test_rest_is_a_fixed_point(oracle_mod):
    c = cases.sphere_array3d(16, 3, r_range=(2.0, 3.5), seed=2, a=(0.0, 0.0, 0.0))
    o = oracle_mod.OracleLBM3D(c, P.Parameters(c.Kn, c.H))
    f0 = o.get_f()
    o.step(5)
    np.testing.assert_allclose(o.get_f()[:, c.solid == 0], f0[:, c.solid == 0], rtol=0, atol=1e-15)


def _profile3d(o, m):
    rho, ux, uy, uz = o.fields()
    return ux[1:m + 1, 0, 0], uz[1:m + 1, 0, 0]


def test_tuned_slip_poiseuille_3d_matches_numvelo(oracle_mod):
    """Tuned parameters (Eqs. Eqexlva-NSliCoertstq), walls at gamma 0.5 and
    0.3, Kn 0.05, m = 32: the profile is Eq. numvelo, node by node, as in 2-D."""
    m = 32
    c = cases.channel3d(2, 2, m, 0.5, 0.3, Kn=0.05, ax=1e-6)
    par = P.Parameters(c.Kn, c.H)
    o = oracle_mod.OracleLBM3D(c, par)
    o.run_to(1e-12, 200000)
    ux, uz = _profile3d(o, m)
    uc = c.a[0] * c.H ** 2 / (8 * P.viscosity(par.tau_s))
    want = P.poiseuille_profile(np.arange(m) + 0.5, c.H, uc,
                                P.slip_velocity_physical(par.L1, par.L2, c.Kn))
    np.testing.assert_allclose(ux / uc, want / uc, rtol=0, atol=1e-8)
    # a normal velocity of second order only (the two unequal walls exchange
    # mass through the diffuse part, O(Ma^2), outside the linear analysis)
    assert np.abs(uz).max() < 1e-5 * uc


@pytest.mark.parametrize("r,l,g,ts,tq", [(0.7, 0.3, 0.25, 1.2, 1.2), (0.45, 0.8, 0.9, 2.0, 0.9)])
def test_untuned_slip_3d_matches_eqmislip(oracle_mod, r, l, g, ts, tq):
    m = 16
    c = cases.channel3d(2, 2, m, g, g, Kn=0.05, ax=1e-6)
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=tq, l_mode=l, r_fixed=r)
    o = oracle_mod.OracleLBM3D(c, par)
    o.run_to(1e-12, 400000)
    ux, _ = _profile3d(o, m)
    uc = c.a[0] * c.H ** 2 / (8 * P.viscosity(ts))
    want = P.poiseuille_profile(np.arange(m) + g, c.H, uc,
                                P.slip_velocity_numeric(r, l, g, ts, tq, c.H))
    np.testing.assert_allclose(ux / uc, want / uc, rtol=0, atol=2e-8)


@pytest.mark.parametrize("mode", [0, 1])
def test_plane_couette_3d_matches_the_wall_relation(oracle_mod, mode):
    """a = 0, upper wall moving along x: the linear profile satisfies the
    wall relation of each reading (Eq. u1u0Coeff for mode 0, A', C' for the
    printed mode 1)."""
    m, U, g, r, l = 10, 1e-4, 0.3, 0.8, 0.4
    c = cases.channel3d(2, 2, m, g, g, Kn=0.05, ax=0.0, u_top=U)
    ts, tq = 1.3, 1.1
    par = P.Parameters(c.Kn, c.H, tau_s=ts, tau_q_fixed=tq, l_mode=l, r_fixed=r)
    o = oracle_mod.OracleLBM3D(c, par, diffuse_mode=mode)
    o.run_to(1e-13, 400000)
    ux, _ = _profile3d(o, m)
    A, _, C = (P.wall_recursion_coefficients_printed if mode else P.wall_recursion_coefficients)(
        r, l, g, ts, tq)
    H = c.H
    Mx = np.array([[1 - A, (1 + g) - A * g], [1 - A, (H - 1 - g) - A * (H - g)]])
    alpha, beta = np.linalg.solve(Mx, [0.0, C * U])
    np.testing.assert_allclose(ux / U, (alpha + beta * (np.arange(m) + g)) / U, rtol=0, atol=2e-9)


def test_the_third_order_relaxation_time_matters(oracle_mod):
    """Negative control: with m relaxing at another rate than tau_q the 3-D
    channel leaves Eq. numvelo (the equivalence above is not automatic)."""
    m = 16
    c = cases.channel3d(2, 2, m, 0.5, 0.3, Kn=0.05, ax=1e-6)
    par = P.Parameters(c.Kn, c.H)

    class Other(P.Parameters):
        def relaxation_times_d3q19(self):
            t = super().relaxation_times_d3q19()
            t[16:19] = 1.0
            return t

    other = Other(c.Kn, c.H)
    o = oracle_mod.OracleLBM3D(c, other)
    o.run_to(1e-12, 200000)
    ux, _ = _profile3d(o, m)
    uc = c.a[0] * c.H ** 2 / (8 * P.viscosity(par.tau_s))
    want = P.poiseuille_profile(np.arange(m) + 0.5, c.H, uc,
                                P.slip_velocity_physical(par.L1, par.L2, c.Kn))
    assert np.abs(ux - want).max() / uc > 1e-4
