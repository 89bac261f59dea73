"""GPU seed-atom weights (Alg. 1-2) and coordination seeding vs the oracle.

* explicit seeds: lambda, blend weights and evaluated sets bit-exact, FP64
  forces within 1e-10 eV/A of the oracle (method and plain blend), linear and
  cubic blending, float32 potentials keep float64 weights;
* coordination rule: the seed mask equals the oracle's coordination criterion
  bit for bit, for the instantaneous counts of the first evaluation and for the
  mean over a period of MD steps, and the weights follow;
* argument checks, and switching back to geometric regions.
"""
import numpy as np
import pytest

import oracle
from paper_2502_19081_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def mx():
    from paper_2502_19081_gb300 import build, mix
    build.build()
    return mix


def _max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


def _check_weights(ctx, om, x):
    lam, w = ctx.lam()
    olam, ow = om.lam(x)
    assert np.array_equal(lam, olam) and np.array_equal(w, ow)
    fl, ae, ac = ctx.sets()
    ofl = om.sets(x)
    assert np.array_equal(fl, ofl)
    assert np.array_equal(ae, np.nonzero(ofl & 4)[0]) and np.array_equal(ac, np.nonzero(ofl & 8)[0])
    return lam


@pytest.mark.parametrize("blend", [0, 1])
def test_explicit_seeds_match_oracle(mx, blend):
    wl = I.small_fe_box(31)
    seeds = [7, 7, 200, 511]
    rcore, rb = 2.6, 4.0
    ctx = mx.open_context(wl, blend=blend)
    ctx.set_seeds(seeds, rcore, rb)
    ctx.forces()
    x, _, F, _ = ctx.get_state()
    om = oracle.Model(wl, blend=blend)
    om.set_atomic(np.array(seeds), rcore, rb)
    lam = _check_weights(ctx, om, x)
    assert (lam == 1.0).sum() > len(set(seeds)) and ((lam > 0) & (lam < 1)).sum() > 0
    mask, k = ctx.seeds()
    assert k == 3 and np.array_equal(np.nonzero(mask)[0], [7, 200, 511])
    FB, _, _ = om.forces(x, oracle.MODE_METHOD)
    FA, _, _ = om.forces(x, oracle.MODE_PLAIN)
    assert _max_abs(F[:, :3], FB[:, :3]) < TOL64 and _max_abs(F[:, :3], FA[:, :3]) < TOL64


def test_seed_weights_float32_potentials(mx):
    wl = I.small_fe_box(32)
    ctx = mx.open_context(wl, precision=mx.MIX_FP32)
    ctx.set_seeds([100], 2.6, 3.5)
    ctx.forces()
    x, _, F, _ = ctx.get_state()
    om = oracle.Model(wl)
    om.set_atomic(np.array([100]), 2.6, 3.5)
    _check_weights(ctx, om, x)
    FB, _, _ = om.forces(x, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], FB[:, :3]) <= 1e-3


def test_coordination_seeds_first_evaluation(mx):
    """Si vacancy: with r_coord between the first (2.35 A) and second (3.84 A)
    neighbour shells the under-coordinated atoms (z <= 3) are the vacancy's
    four neighbours."""
    wl = I.si_vacancy()
    ctx = mx.open_context(wl)
    ctx.set_seed_rule(3.0, 0.0, 3.0, 1, 2.6, 3.5)
    ctx.forces()
    x, _, F, _ = ctx.get_state()
    om = oracle.Model(wl)
    z = om.coordination(x, 3.0)
    expect = (z <= 3).astype(np.uint8)
    mask, k = ctx.seeds()
    assert np.array_equal(mask, expect) and k == 4
    om.set_atomic(expect.astype(bool), 2.6, 3.5)
    _check_weights(ctx, om, x)
    FB, _, _ = om.forces(x, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], FB[:, :3]) < TOL64


def test_coordination_seeds_follow_the_trajectory(mx):
    """period 1: the seeds of every step are the criterion at that step's positions."""
    wl = I.si_vacancy()
    ctx = mx.open_context(wl)
    rz = 2.42          # inside the thermal spread of the first shell: seeds change along the run
    ctx.set_seed_rule(rz, 0.0, 3.0, 1, 2.6, 3.5)
    ctx.forces()
    om = oracle.Model(wl)
    for _ in range(4):
        ctx.step(wl.dt, 3)
        x, _, _, _ = ctx.get_state()
        expect = (om.coordination(x, rz) <= 3).astype(np.uint8)
        mask, _ = ctx.seeds()
        assert np.array_equal(mask, expect)
        om.set_atomic(expect.astype(bool), 2.6, 3.5)
        _check_weights(ctx, om, x)


@pytest.mark.parametrize("tune", [False, True])
def test_coordination_mean_over_a_period(mx, tune):
    """The counts are averaged over `period` steps; the launch-shape tuner's
    extra evaluations in the middle of a period leave the averaging alone."""
    wl = I.si_vacancy()
    ctx = mx.open_context(wl)
    rz, period, lo, hi = 2.42, 3, 3.4, 3.8
    ctx.set_seed_rule(rz, lo, hi, period, 2.6, 3.5)
    ctx.forces()
    om = oracle.Model(wl)
    x0, _, _, _ = ctx.get_state()
    z0 = om.coordination(x0, rz)
    assert np.array_equal(ctx.seeds()[0], ((z0 >= lo) & (z0 <= hi)).astype(np.uint8))
    zs = np.zeros(wl.system.n, dtype=np.int64)
    for k in range(period):
        ctx.step(wl.dt, 1)
        x, _, _, _ = ctx.get_state()
        zs += om.coordination(x, rz)
        if tune and k == 0:
            ctx.tune(2)
    mean = zs / float(period)
    expect = ((mean >= lo) & (mean <= hi)).astype(np.uint8)
    mask, k = ctx.seeds()
    assert np.array_equal(mask, expect)
    om.set_atomic(expect.astype(bool), 2.6, 3.5)
    _check_weights(ctx, om, x)
    # the seeds hold between refreshes
    ctx.step(wl.dt, 1)
    assert np.array_equal(ctx.seeds()[0], expect)


def test_seed_arguments_checked_and_regions_restored(mx):
    wl = I.small_fe_box(33)
    ctx = mx.open_context(wl)
    for bad in (lambda: ctx.set_seeds([wl.system.n], 2.0, 3.0),
                lambda: ctx.set_seeds([-1], 2.0, 3.0),
                lambda: ctx.set_seeds([0], 2.0, 100.0),
                lambda: ctx.set_seeds([0], -1.0, 3.0),
                lambda: ctx.set_seed_rule(3.0, 0, 3, 0, 2.0, 3.0),
                lambda: ctx.set_seed_rule(3.0, 4, 3, 1, 2.0, 3.0),
                lambda: ctx.set_seed_rule(100.0, 0, 3, 1, 2.0, 3.0)):
        with pytest.raises(mx.MixError) as e:
            bad()
        assert e.value.code == mx.MIX_EINVAL
    ctx.set_seeds([], 2.0, 3.0)
    ctx.forces()
    lam, _ = ctx.lam()
    assert np.all(lam == 0.0)
    ctx.set_regions(wl.regions)
    ctx.forces()
    x, _, _, _ = ctx.get_state()
    _check_weights(ctx, oracle.Model(wl), x)
