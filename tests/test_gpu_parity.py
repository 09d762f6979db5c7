"""GPU (liblbm.so through the C ABI) against the FP64 oracle, on the same
seeded inputs.

Tolerances: FP64 storage -- populations element by element within 1e-13
absolute (populations are O(0.1); this leaves room for summation-order
round-off over a few hundred steps only).  FP32 deviation storage --
velocity relative L2 <= 1e-5 and mass drift |M_gpu - M_oracle| / M_oracle(0)
<= 1e-10, the accuracy targets of the FP32 path.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import params as P
from paper_2012_14707_gb300 import cases
from paper_2012_14707_gb300 import build as lbm_build
from paper_2012_14707_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm_build.build()
    lbm.load()
    oracle.build()


def _pair(case, precision, start_seed=None, amp=1e-3, **kw):
    """Oracle and GPU solver on the same case, parameters and start state."""
    okw = {}
    gkw = dict(precision=precision)
    for k in ("l_mode", "diffuse_mode", "E", "L1", "L2", "tau_s", "bgk"):
        if k in kw:
            gkw[k] = kw[k]
    if kw.get("bgk"):
        okw["bgk"] = True
    if "r" in kw:
        gkw["r"] = kw["r"]
        okw["r_fixed"] = kw["r"]
    if "tau_q" in kw:
        gkw["tau_q"] = kw["tau_q"]
        okw["tau_q_fixed"] = kw["tau_q"]
    par = P.Parameters(case.Kn, case.H, L1=kw.get("L1"), L2=kw.get("L2"), E=kw.get("E"),
                       tau_s=kw.get("tau_s"), l_mode=kw.get("l_mode", "paper"), **okw)
    o = oracle.OracleLBM(case, par, diffuse_mode=kw.get("diffuse_mode", 0))
    g = lbm.Solver(case, **gkw)
    if start_seed is not None:
        f0 = cases.random_populations(case.nx, case.ny, start_seed, amp)
        o.set_f(f0)
        g.set_f(f0)
    return o, g


def _fluid_f(case, f):
    """Populations of fluid nodes only (solid nodes carry no state)."""
    return f[:, case.solid == 0]


def _vel_rel_l2(case, a, b):
    fl = case.solid == 0
    num = ((a[1] - b[1])[fl] ** 2 + (a[2] - b[2])[fl] ** 2).sum()
    den = (b[1][fl] ** 2 + b[2][fl] ** 2).sum()
    return math.sqrt(num / den)


CASES = {
    "poiseuille": lambda: cases.config_poiseuille(),
    "annulus": lambda: cases.annulus(40, 8.0, 16.0, 0.05, 0.05 * math.sqrt(1 / 3) / 8),
    "cylinders": lambda: cases.cylinder_array(300, 150, 5, Kn=0.02, ax=1e-5),
    "box": lambda: cases.periodic_box(70, 45, ax=2e-5, ay=-1e-5),
    "column": lambda: cases.periodic_box(1, 7, ax=1e-5),
    "row": lambda: cases.periodic_box(33, 1, ay=1e-5),
    "channel_moving": lambda: cases.channel(37, 9, 0.2, 0.85, Kn=0.05, ax=1e-6, u_top=0.01),
    "inclined": lambda: cases.inclined_channel(120, 1.2, 16, Kn=0.0194),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("diffuse_mode", [0, 1])
def test_fp64_populations_match_oracle(name, diffuse_mode):
    c = CASES[name]()
    kw = dict(L1=1.0, L2=0.0) if name == "annulus" else {}
    o, g = _pair(c, "fp64", start_seed=11, diffuse_mode=diffuse_mode, **kw)
    for n in (1, 37, 162):
        o.step(n)
        g.step(n)
        np.testing.assert_allclose(_fluid_f(c, g.get_f()), _fluid_f(c, o.get_f()), rtol=0, atol=1e-13)
    ro, mo = o.residual()
    rg, mg = g.residual()
    assert rg == pytest.approx(ro, rel=1e-8, abs=1e-300)
    assert mg == pytest.approx(mo, rel=1e-13)
    fo, fg = o.fields(), g.fields()
    for a, b in zip(fg, fo):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_one_row_channel_matches_oracle(precision, tol):
    """A channel one fluid row high (moving upper wall): every node has the
    links j and opp(j) of three direction pairs, so Eq. EqNewBDSC of one
    link reads the unknown population the other link set a step earlier
    (f_jb from the link tail rather than from a neighbour)."""
    c = cases.channel(8, 1, 0.4, 0.7, Kn=0.05, ax=1e-5, u_top=0.01)
    assert c.n_fluid == 8 and c.n_links == 48
    o, g = _pair(c, precision, start_seed=5)
    for n in (1, 37, 162):
        o.step(n)
        g.step(n)
        np.testing.assert_allclose(_fluid_f(c, g.get_f()), _fluid_f(c, o.get_f()), rtol=0, atol=tol)


@pytest.mark.parametrize("l_mode,extra", [
    ("zero", {}), ("gamma", {}), ("2gamma", {}), ("gamma2", {}), ("gamma2+gamma", {}),
    (0.35, {"r": 0.7, "tau_q": 0.9}),
])
def test_fp64_scheme_variants_match_oracle(l_mode, extra):
    c = CASES["cylinders"]()
    o, g = _pair(c, "fp64", start_seed=3, l_mode=l_mode, **extra)
    o.step(120)
    g.step(120)
    np.testing.assert_allclose(_fluid_f(c, g.get_f()), _fluid_f(c, o.get_f()), rtol=0, atol=1e-13)
    r_g, l_g = g.link_params()
    np.testing.assert_allclose(r_g, o.link_r, rtol=1e-13)
    np.testing.assert_allclose(l_g, o.link_l, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_velocity_and_mass_match_oracle(name):
    """From rest, 2000 steps.  Velocity rel. L2 <= 1e-5 everywhere (measured
    5e-8 to 6e-7: the collision adds its small change to the stored
    deviations).  Mass drift against the oracle trajectory: <= 1e-10 with
    stationary walls.  Moving walls (u_b ~ 0.03 and 0.01 here) exchange
    mass with the fluid every step in tiny net amounts (~1e-8 per link and
    step) computed from wall populations of size ~1e-3; their FP32 rounding
    is the same every step once the flow is steady, so it adds up linearly
    (up to 9e-9 relative after 2000 steps): held to 3e-8.  The periodic
    boxes accelerate without bound (u ~ 0.04; measured up to 3.6e-10): held
    to 1e-9."""
    c = CASES[name]()
    kw = dict(L1=1.0, L2=0.0) if name == "annulus" else {}
    o, g = _pair(c, "fp32", **kw)
    m0 = o.residual()[1]
    mass_tol = {"box": 1e-9, "column": 1e-9, "row": 1e-9, "annulus": 3e-8,
                "channel_moving": 3e-8}.get(name, 1e-10)
    for n in (500, 1500):
        o.step(n)
        g.step(n)
        assert _vel_rel_l2(c, g.fields(), o.fields()) <= 1e-5
        assert abs(g.residual()[1] - o.residual()[1]) / m0 <= mass_tol


def test_poiseuille_steady_state_fp64_and_fp32():
    """4 x 32 channel run to residual 1e-10: FP64 meets Eq. numvelo like the
    oracle; FP32 meets the oracle's steady profile within 1e-5."""
    c = cases.config_poiseuille()
    par = P.Parameters(c.Kn, c.H)
    uc = c.ax * c.H ** 2 / (8 * P.viscosity(par.tau_s))
    want = P.poiseuille_profile(np.arange(32) + 0.5, c.H, uc,
                                P.slip_velocity_physical(par.L1, par.L2, c.Kn))
    g64 = lbm.Solver(c, precision="fp64")
    steps, res = g64.run_to(1e-10, 100000)
    assert res < 1e-10
    ux = g64.fields()[1][1:33, 0]
    np.testing.assert_allclose(ux / uc, want / uc, rtol=0, atol=5e-8)
    g32 = lbm.Solver(c, precision="fp32")
    g32.run_to(1e-9, 100000)
    ux32 = g32.fields()[1][1:33, 0]
    assert np.sqrt(((ux32 - ux) ** 2).sum() / (ux ** 2).sum()) <= 1e-5


@pytest.mark.parametrize("Kn,bound", [(0.01, 0.01), (0.05, 0.04), (0.1, 0.07)])
def test_couette_256_parity_and_slip(Kn, bound):
    """256^2 annulus (R1 = 60, R2 = 120): FP64 and FP32 follow the oracle
    over 300 steps; the FP32 steady state is within `bound` (rel. L2) of
    the analytic first-order slip solution Eq. EqAnaMicro and closer to it
    than to the no-slip solution.  (The scheme realises the planar slip law;
    its departure from the curved-wall solution grows with Kn: the oracle
    gives 0.7 % at Kn 0.01 and 2.6-2.9 % at Kn 0.05 on 40^2-136^2
    annuli.)"""
    c = cases.config_couette(Kn)
    for prec in ("fp64", "fp32"):
        o, g = _pair(c, prec, L1=1.0, L2=0.0)
        o.step(300)
        g.step(300)
        if prec == "fp64":
            np.testing.assert_allclose(_fluid_f(c, g.get_f()), _fluid_f(c, o.get_f()), rtol=0,
                                       atol=1e-13)
        else:
            assert _vel_rel_l2(c, g.fields(), o.fields()) <= 1e-5
    g = lbm.Solver(c, precision="fp32", L1=1.0, L2=0.0)
    g.run_to(1e-9, 400000)
    rho, ux, uy = g.fields()
    m = c.meta
    yy, xx = np.mgrid[0:c.ny, 0:c.nx]
    dx, dy = xx - m["center"], yy - m["center"]
    rr = np.hypot(dx, dy)
    fl = c.solid == 0
    ut = (-dy * ux + dx * uy) / np.where(rr > 0, rr, 1)
    ua = P.couette_profile(rr, m["R1"], m["R2"], m["omega1"], 0.0, Kn * (m["R2"] - m["R1"]))
    ua0 = P.couette_profile(rr, m["R1"], m["R2"], m["omega1"], 0.0, 0.0)
    err = np.sqrt(((ut - ua)[fl] ** 2).sum() / (ua[fl] ** 2).sum())
    err0 = np.sqrt(((ut - ua0)[fl] ** 2).sum() / (ua[fl] ** 2).sum())
    assert err < bound
    assert err < err0


def test_full_size_throughput_case_matches_oracle():
    """8192 x 4096 random-cylinder channel, FP32 in the benchmark's launch
    configuration: two steps from a seeded perturbed state, every node
    against the oracle."""
    c = cases.config_throughput()
    o, g = _pair(c, "fp32", start_seed=21, amp=1e-3)
    o.step(2)
    g.step(2)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None]
    a, b = _fluid_f(c, g.get_f()), _fluid_f(c, o.get_f())
    # FP32 deviation storage: |error| ~ 1e-7 of the deviation scale amp * w
    np.testing.assert_allclose((a - w) / w, (b - w) / w, rtol=0, atol=2e-8)


def test_nonfinite_state_is_reported():
    c = CASES["box"]()
    g = lbm.Solver(c, precision="fp32")
    f = cases.random_populations(c.nx, c.ny, 1)
    f[3, 10, 20] = np.nan
    g.set_f(f)
    g.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        g.residual()
    assert ei.value.code == lbm.LBM_EUNSTABLE


@pytest.mark.parametrize("name", ["poiseuille", "cylinders", "inclined"])
def test_fp64_bgk_matches_oracle(name):
    """BGK reading of Sec. 3.B (one relaxation time, E for tau_q = tau_s)."""
    c = CASES[name]()
    o, g = _pair(c, "fp64", start_seed=4, bgk=True)
    o.step(150)
    g.step(150)
    np.testing.assert_allclose(_fluid_f(c, g.get_f()), _fluid_f(c, o.get_f()), rtol=0, atol=1e-13)
    assert g.info().tau_q == pytest.approx(g.info().tau_s, rel=1e-12)


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}  # 8 and 11 significant bits


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("name", ["cylinders", "annulus", "channel_moving", "inclined"])
def test_16bit_one_step_is_the_oracle_step_rounded_to_storage(name, precision):
    """Both sides start from the same state, one that the 16-bit storage
    holds exactly (a seeded state imported by the GPU and read back), and
    take one step.  A streamed population is the oracle's value rounded once
    to storage: |error| <= u |f_i - w_i| with u the unit round-off, plus a
    floor for the FP32 arithmetic.  A link population also carries the
    roundings of the post-collision values it is built from, and the rest
    population those of the eight others (it closes the mass balance):
    <= u (|f_i - w_i| + 10 s), s the node's largest deviation."""
    c = CASES[name]()
    kw = dict(L1=1.0, L2=0.0) if name == "annulus" else {}
    o, g = _pair(c, precision, start_seed=7, amp=1e-3, **kw)
    o.set_f(g.get_f())
    o.step(1)
    g.step(1)
    fl = c.solid == 0
    a = g.get_f()[:, fl] - W9[:, None]
    b = o.get_f()[:, fl] - W9[:, None]
    u = UNIT_ROUNDOFF[precision]
    s = np.abs(b).max(axis=0)
    err = np.abs(a - b)
    link = np.zeros((9, c.ny, c.nx), bool)
    link[np.asarray(c.link_dir), np.asarray(c.link_y), np.asarray(c.link_x)] = True
    link = link[:, fl]
    link[0] = True
    floor = 2.0 ** -20 * s
    plain = ~link
    assert (err[plain] <= u * np.abs(b[plain]) + np.broadcast_to(floor, b.shape)[plain]).all()
    assert (err[link] <= u * (np.abs(b[link]) + 10 * np.broadcast_to(s, b.shape)[link])).all()
    # and not a loose bound in practice: the typical error is a fraction of one rounding
    assert np.median(err[plain] / (u * np.abs(b[plain]) + 1e-300)) <= 0.5


# Velocity rel. L2 and mass drift against the oracle after 500 steps from rest
# (bounds ~2x the values measured on a GB300).  BF16 keeps 8 significant bits
# of each deviation: ~1e-3 to 1e-2 in velocity where u ~ 1e-3 to 1e-2, and the
# slow 4 x 32 channel (u ~ 2e-4, deviations ~ 2e-5) loses most of its profile
# -- BF16 storage does not meet a 1e-3 target there.  FP16 (deviations x 4096)
# keeps 11 bits: 2e-4 to 2e-3.
BOUNDS_16 = {
    ("bf16", "annulus"): (3e-3, 3e-4), ("bf16", "cylinders"): (1.5e-2, 2e-6),
    ("bf16", "channel_moving"): (3e-2, 1.2e-4), ("bf16", "poiseuille"): (0.25, 2e-8),
    ("fp16", "annulus"): (4e-4, 3e-5), ("fp16", "cylinders"): (8e-4, 3e-7),
    ("fp16", "channel_moving"): (4e-3, 1.3e-6), ("fp16", "poiseuille"): (2e-3, 1e-9),
}


@pytest.mark.parametrize("precision,name", list(BOUNDS_16))
def test_16bit_velocity_and_mass_after_500_steps(precision, name):
    c = CASES[name]()
    kw = dict(L1=1.0, L2=0.0) if name == "annulus" else {}
    o, g = _pair(c, precision, **kw)
    m0 = o.residual()[1]
    o.step(500)
    g.step(500)
    vb, mb = BOUNDS_16[(precision, name)]
    assert _vel_rel_l2(c, g.fields(), o.fields()) <= vb
    assert abs(g.residual()[1] - o.residual()[1]) / m0 <= mb
