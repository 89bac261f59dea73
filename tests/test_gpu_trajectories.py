"""Long trajectories against the oracle on the GPU's own bits (GPU).

MD is chaotic, so two implementations' trajectories part after a few hundred
steps; the protocol instead downloads the GPU state every 100 steps and has the
oracle re-evaluate the evaluated sets (bit-exact) and the forces (1e-10 eV/A
in float64; the 1e-3 eV/A gate for float and for the bf16 hi/lo readout) at
exactly those positions.

* Fe dumbbell (8,001 atoms): 1000 steps in float64 and in float, checkpoints
  every 100 steps;
* screw cylinder (256,000 atoms): 64 sampled atoms (core, ramp, expensive
  buffer, cheap only) at step 0 and after 100 steps in float64 and in float,
  and every 100 steps up to 500 with the bf16 hi/lo readout, the whole set
  compared exactly; with the plain bf16 readout every 100 steps up to 500,
  every atom's force within the gate of the float64 path at the same
  positions and 64 sampled atoms within the gate of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2502_19081_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mx():
    from paper_2502_19081_gb300 import build, mix
    build.build()
    return mix


def _max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-3)])
def test_fe_dumbbell_1000_steps_checkpoints(mx, prec, tol):
    wl = I.fe_dumbbell()
    ctx = mx.open_context(wl, precision=prec)
    om = oracle.Model(wl)
    worst = 0.0
    for k in range(10):
        ctx.step(wl.dt, 100)
        x, _, F, step = ctx.get_state()
        assert step == 100 * (k + 1)
        fl, _, _ = ctx.sets()
        assert np.array_equal(fl, om.sets(x)), step
        FB, _, _ = om.forces(x, oracle.MODE_METHOD)
        err = _max_abs(F[:, :3], FB[:, :3])
        worst = max(worst, err)
        assert err < tol, (step, err)
    st = ctx.stats()
    assert st["rebuilds"] >= 2 and st["n_exp"] > 1000


def _sample(rng, lam, fl, k):
    pick = []
    for sel in (lam == 1.0, (lam > 0) & (lam < 1), (lam == 0) & ((fl & 4) > 0), (fl & 4) == 0):
        idx = np.nonzero(sel)[0]
        pick += list(rng.choice(idx, k, replace=False))
    return np.array(pick)


@pytest.mark.parametrize("prec,tol,nblocks", [(0, 1e-10, 1), (1, 1e-3, 1), (3, 1e-3, 5)])
def test_screw_cylinder_checkpoints(mx, prec, tol, nblocks):
    wl = I.fe_screw()
    ctx = mx.open_context(wl, precision=prec)
    om = oracle.Model(wl)
    rng = np.random.default_rng(7)
    for k in range(nblocks + 1):
        if k:
            ctx.step(wl.dt, 100)
        x, _, F, step = ctx.get_state()
        assert step == 100 * k
        fl, _, _ = ctx.sets()
        assert np.array_equal(fl, om.sets(x)), step
        lam, _ = ctx.lam()
        pick = _sample(rng, lam, fl, 16)
        Fs = om.forces_sampled(x, pick)
        assert _max_abs(F[pick, :3], Fs[:, :3]) < tol, step


def test_screw_cylinder_plain_bf16_within_gate_500_steps(mx):
    """The screw cylinder with the plain bf16 readout (the precision its
    throughput is quoted in) for 500 steps: every 100 steps the evaluated sets
    equal the oracle's, every atom's force is within the 1e-3 eV/A gate of the
    float64 path evaluated at the same positions (which itself matches the
    oracle to 1e-10), and 64 sampled atoms are within the gate of the oracle."""
    wl = I.fe_screw()
    ctx = mx.open_context(wl, precision=mx.MIX_BF16)
    ref = mx.open_context(wl, precision=mx.MIX_FP64)
    om = oracle.Model(wl)
    rng = np.random.default_rng(11)
    for k in range(6):
        if k:
            ctx.step(wl.dt, 100)
        x, v, F, step = ctx.get_state()
        assert step == 100 * k
        fl, _, _ = ctx.sets()
        assert np.array_equal(fl, om.sets(x)), step
        ref.set_state(x, v, None, step)
        ref.forces()
        _, _, F64, _ = ref.get_state()
        assert _max_abs(F[:, :3], F64[:, :3]) < 1e-3, step
        lam, _ = ctx.lam()
        pick = _sample(rng, lam, fl, 16)
        Fs = om.forces_sampled(x, pick)
        assert _max_abs(F[pick, :3], Fs[:, :3]) < 1e-3, step
        assert _max_abs(F64[pick, :3], Fs[:, :3]) < 1e-10, step
    ctx.close()
    ref.close()
