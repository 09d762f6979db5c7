"""Batched solver (lbm_batch_*) against lone solvers and the oracle."""
import numpy as np
import pytest

import oracle
from oracle import params as P
from paper_2012_14707_gb300 import build as lbm_build
from paper_2012_14707_gb300 import cases, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm_build.build()
    lbm.load()
    oracle.build()


def _small_batch():
    return cases.batch_cases(7, seed=3, nx_range=(40, 130), ny_range=(40, 96),
                             kn_range=(0.01, 0.1))


def test_case_in_batch_is_bitwise_the_case_alone():
    """Every case of a mixed batch converges at the same step, to bitwise the
    same fields, as the same case run alone with the same check interval."""
    cl = _small_batch()
    b = lbm.Batch(cl, precision="fp32")
    steps, res, total = b.run_to(1e-6, 8000, check_every=100)
    assert (steps != 0).any()
    for k, c in enumerate(cl):
        s = lbm.Solver(c, precision="fp32", residual_every=100)
        n, r = s.run_to(1e-6, 8000)
        if steps[k] > 0:
            assert n == steps[k], (k, n, steps[k])
        got = b.fields(k)
        want = s.fields()
        for a, w in zip(got, want):
            np.testing.assert_array_equal(a, w)


def test_batch_matches_oracle_fp64():
    """FP64 batch of three different cases, 300 steps, against the oracle."""
    cl = _small_batch()[:3]
    b = lbm.Batch(cl, precision="fp64")
    steps, res, total = b.run_to(0.0, 300, check_every=100)
    assert total == 300 and (steps == 0).all()
    for k, c in enumerate(cl):
        o = oracle.OracleLBM(c, P.Parameters(c.Kn, c.H))
        o.step(300)
        for a, w in zip(b.fields(k), o.fields()):
            np.testing.assert_allclose(a, w, rtol=0, atol=1e-12)


def test_batch_reset_and_info():
    cl = _small_batch()[:2]
    b = lbm.Batch(cl, precision="fp32")
    info = b.info()
    assert info["total_nodes"] == sum(c.nx * c.ny for c in cl)
    assert info["total_fluid"] == sum(c.n_fluid for c in cl)
    assert info["cta_threads"] in (64, 128, 256)
    s1 = b.run_to(0.0, 200, 100)
    f1 = b.fields(1)
    b.reset()
    s2 = b.run_to(0.0, 200, 100)
    for a, w in zip(b.fields(1), f1):
        np.testing.assert_array_equal(a, w)
    with pytest.raises(lbm.LbmError):
        b.run_to(1e-6, 100, check_every=3)


def test_batch_of_awkward_sizes_is_bitwise_the_cases_alone():
    """Cases smaller than a warp, of exactly one 256-node chunk, one node
    more, and a walled channel share the node arena (each case starts on a
    256-node chunk); 300 steps of each in the batch equal 300 steps alone."""
    cl = [cases.periodic_box(1, 7, ax=1e-5),
          cases.periodic_box(16, 16, ax=1e-5, ay=-2e-6),
          cases.periodic_box(257, 1, ax=1e-5),
          cases.config_poiseuille(),
          cases.cylinder_array(70, 45, 2, Kn=0.02, ax=1e-5)]
    assert [c.n_fluid for c in cl[:3]] == [7, 256, 257]
    b = lbm.Batch(cl, precision="fp32")
    info = b.info()
    chunks = sum((max(c.n_fluid, 1) + 255) // 256 for c in cl)
    assert info["n_ctas"] * info["cta_threads"] == 256 * chunks
    steps, res, total = b.run_to(0.0, 300, check_every=100)
    assert total == 300 and (steps == 0).all()
    for k, c in enumerate(cl):
        s = lbm.Solver(c, precision="fp32")
        s.step(300)
        for a, w in zip(b.fields(k), s.fields()):
            np.testing.assert_array_equal(a, w)
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_stochastic_rounding_and_exact_mass_cases_in_a_batch_are_the_cases_alone(precision):
    """16-bit batches round stochastically with random bits keyed by the
    case's step count (the batch's device counter plus the step's place in
    the graph), FP32 cases with a moving wall (and one that asks for it) run
    the exact-mass step in the batch's own kernel for them: 300 steps of
    each case in the batch equal 300 steps alone, bit for bit."""
    cl = [cases.channel(37, 9, 0.2, 0.85, Kn=0.05, ax=1e-6, u_top=0.01),
          cases.cylinder_array(70, 45, 2, Kn=0.02, ax=1e-5),
          cases.periodic_box(40, 30, ax=1e-5, ay=-3e-6),
          cases.annulus(40, 8.0, 16.0, 0.05, 0.05 * (1 / 3) ** 0.5 / 8)]
    prm = [{}, {}, {"mass_mode": 1}, {"L1": 1.0, "L2": 0.0}]
    b = lbm.Batch(cl, precision=precision, params=prm)
    steps, res, total = b.run_to(0.0, 300, check_every=100)
    assert total == 300 and (steps == 0).all()
    for k, c in enumerate(cl):
        s = lbm.Solver(c, precision=precision, **prm[k])
        if precision == "fp32":
            assert s.info().exact_mass == (0 if k == 1 else 1)
        s.step(300)
        for a, w in zip(b.fields(k), s.fields()):
            np.testing.assert_array_equal(a, w)
        s.close()


def test_interval_residual_in_a_batch_is_the_case_alone():
    """residual_mode 1 in a batch: each case retires at the same step as the
    same case run alone with the same check interval, FP32, tolerance 1e-8."""
    cl = _small_batch()[:4]
    prm = [{"residual_mode": 1}] * len(cl)
    b = lbm.Batch(cl, precision="fp32", params=prm)
    steps, res, total = b.run_to(1e-8, 30000, check_every=100)
    assert (steps > 0).any()
    for k, c in enumerate(cl):
        s = lbm.Solver(c, precision="fp32", residual_every=100, residual_mode=1)
        n, r = s.run_to(1e-8, 30000)
        if steps[k] > 0:
            assert n == steps[k] and r < 1e-8, (k, n, steps[k])
            for a, w in zip(b.fields(k), s.fields()):
                np.testing.assert_array_equal(a, w)
        s.close()


def test_autotuned_launch_is_no_slower_than_the_fixed_default():
    """The autotuner's launch shape against the fixed default (128 threads,
    L2 prefetch on), each timed over 2000 steps of the same 96-case batch
    (tol 0: every case runs all steps), best of three."""
    import time

    cl = cases.batch_cases(96, seed=5)
    b = lbm.Batch(cl, precision="fp32")

    def timed():
        b.reset()
        t0 = time.perf_counter()
        b.run_to(0.0, 2000, check_every=100)
        return time.perf_counter() - t0

    timed()
    t_auto = min(timed() for _ in range(3))
    b.set_launch(128, True)
    timed()
    t_fixed = min(timed() for _ in range(3))
    b.close()
    assert t_auto <= 1.10 * t_fixed, (t_auto, t_fixed)


def test_set_launch_rejects_other_shapes():
    b = lbm.Batch(cases.batch_cases(2, seed=1), precision="bf16")
    with pytest.raises(lbm.LbmError):
        b.set_launch(256, True)
    with pytest.raises(lbm.LbmError):
        b.set_launch(96, False)
    b.set_launch(64, False)
    steps, _, _ = b.run_to(1e-3, 200, check_every=100)
    b.close()


def test_full_size_batch_matches_oracle_on_sampled_cases():
    """The 512-case batched workload as the benchmark runs it (FP32, the
    interval residual, the autotuned launch), 300 steps from rest; the
    largest and the smallest case of each geometry against the FP64 oracle:
    velocity rel. L2 <= 1e-5, and mass drift <= 1e-10 where no wall moves
    (the FP32 targets)."""
    cl = cases.batch_cases(512, seed=0)
    b = lbm.Batch(cl, precision="fp32", params=[{"residual_mode": 1}] * len(cl))
    steps, res, total = b.run_to(0.0, 300, check_every=100)
    assert total == 300 and (steps == 0).all()
    pick = []
    for kind in ("channel", "annulus", "cylinders"):
        ks = sorted((k for k, c in enumerate(cl) if c.meta["batch_kind"] == kind),
                    key=lambda k: cl[k].n_fluid)
        pick += [ks[0], ks[-1]]
    for k in pick:
        c = cl[k]
        fl = c.solid == 0
        o = oracle.OracleLBM(c, P.Parameters(c.Kn, c.H), threads=oracle.host_cores())
        m0 = o.fields()[0][fl].sum()
        o.step(300)
        rg, ug, vg = b.fields(k)
        ro, uo, vo = o.fields()
        num = ((ug - uo)[fl] ** 2 + (vg - vo)[fl] ** 2).sum()
        den = (uo[fl] ** 2 + vo[fl] ** 2).sum()
        assert np.sqrt(num / den) <= 1e-5, (k, c.name)
        if c.meta["batch_kind"] != "annulus":
            assert abs(rg[fl].sum() - ro[fl].sum()) / m0 <= 1e-10, (k, c.name)
    b.close()
