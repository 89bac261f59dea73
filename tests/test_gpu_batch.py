"""Batches and autotuning through the C ABI (GPU).

A batch advances independent replicas with one graph launch per step; each
member must end bit-identical to the same replica stepped alone (kernels are
deterministic and no kernel reads another member's data).  Autotuning times
force evaluations only and must leave the state unchanged.
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


def _replicas():
    ace, spl = I.element_potentials("Si", np.random.default_rng(1), 5.0, 8, 3, 3)
    specs = [(300, "vacancy", 300.0), (700, "interstitial", 900.0), (1500, "vacancy", 1500.0),
             (2500, "interstitial", 600.0), (450, "vacancy", 1200.0), (1100, "interstitial", 450.0)]
    return [I.si_replica(50 + k, n, dfc, t, ace, spl) for k, (n, dfc, t) in enumerate(specs)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fused", [True, False])
def test_batch_equals_members_alone(mx, prec, fused):
    wls = _replicas()
    alone = []
    for wl in wls:
        c = mx.open_context(wl, precision=prec)
        c.step(1.0, 20)
        alone.append(c.get_state())
        c.close()
    members = [mx.open_context(wl, precision=prec) for wl in wls]
    b = mx.Batch(members)
    b.set_fused(fused)
    b.step(1.0, 8)
    assert b.info()["fused"] == fused
    b.step(1.0, 12)
    b.sync()
    for c, (xa, va, fa, sa) in zip(members, alone):
        x, v, f, s = c.get_state()
        assert s == sa == 20
        assert np.array_equal(x, xa) and np.array_equal(v, va) and np.array_equal(f, fa)
    b.close()


def test_batch_tune_keeps_results(mx):
    wls = _replicas()[:4]
    members = [mx.open_context(wl, precision=1) for wl in wls]
    before = [c.get_state() for c in members]
    b = mx.Batch(members)
    div = b.tune(reps=2)
    assert div in (1, 2, 4, 8, 16)
    for c, st in zip(members, before):
        x, v, f, _ = c.get_state()
        assert np.array_equal(x, st[0]) and np.array_equal(v, st[1]) and np.array_equal(f, st[2])
    b.step(1.0, 10)
    b.sync()
    for wl, c in zip(wls, members):
        a = mx.open_context(wl, precision=1)
        a.step(1.0, 10)
        xa, va, fa, _ = a.get_state()
        x, v, f, _ = c.get_state()
        assert np.array_equal(x, xa) and np.array_equal(f, fa)
    b.close()


def test_context_tune_keeps_state_and_parity(mx):
    wl = I.fe_dumbbell()
    c = mx.open_context(wl)
    x0, v0, f0, _ = c.get_state()
    c.tune(reps=2)
    x1, v1, f1, _ = c.get_state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    assert np.abs(f1 - f0).max() < 1e-13
    info = c.info()
    assert info["exp_grid"] >= 1 and info["gather_grid"] >= 1
    c.step(1.0, 5)
    x, _, F, _ = c.get_state()
    FB, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
    assert np.abs(F[:, :3] - FB[:, :3]).max() < 1e-10


def test_replica_forces_match_oracle(mx):
    for wl in _replicas()[:3]:
        c = mx.open_context(wl, precision=1)
        x, _, F, _ = c.get_state()
        FB, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
        assert np.abs(F[:, :3] - FB[:, :3]).max() <= 1e-3


def _mixed():
    """Si and Fe cells: two groups of the expensive kernel, hot enough that
    lists are rebuilt during the run."""
    ace, spl = I.element_potentials("Si", np.random.default_rng(1), 5.0, 8, 3, 3)
    out = [I.si_replica(70, 900, "vacancy", 1500.0, ace, spl), I.si_replica(71, 2000, "interstitial", 1200.0, ace, spl)]
    for k, seed in enumerate((43, 44)):
        wl = I.small_fe_box(seed, n_rad=5, l_max=4)
        wl.system.v = I.maxwell_boltzmann(np.random.default_rng(seed), wl.system.n, wl.system.mass, 1500.0)
        out.append(wl)
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_fused_mixed_elements_with_rebuilds(mx, prec):
    wls = _mixed()
    alone = []
    for wl in wls:
        c = mx.open_context(wl, precision=prec)
        c.step(1.0, 30)
        alone.append((c.get_state(), c.stats()["rebuilds"]))
        c.close()
    members = [mx.open_context(wl, precision=prec) for wl in wls]
    b = mx.Batch(members)
    b.step(1.0, 11)
    b.step(1.0, 19)
    b.sync()
    inf = b.info()
    assert inf["fused"] and inf["groups"] == 2 and inf["launches"] > 0
    for c, ((xa, va, fa, sa), ra) in zip(members, alone):
        x, v, f, s = c.get_state()
        assert s == sa == 30
        assert c.stats()["rebuilds"] == ra
        assert np.array_equal(x, xa) and np.array_equal(v, va) and np.array_equal(f, fa)
    assert max(r for _, r in alone) > 2     # lists really were rebuilt along the way
    # the oracle on each member's final bits: sets exactly, forces within the
    # precision's tolerance (1e-10 eV/A float64, the 1e-3 eV/A gate float)
    tol = 1e-10 if prec == 0 else 1e-3
    for wl, c in zip(wls, members):
        x, _, f, _ = c.get_state()
        om = oracle.Model(wl)
        fl, _, _ = c.sets()
        assert np.array_equal(fl, om.sets(x))
        FB, _, _ = om.forces(x, oracle.MODE_METHOD)
        assert np.abs(f[:, :3] - FB[:, :3]).max() < tol
    b.close()


def test_fused_batch_falls_back_for_seed_weights(mx):
    wls = _mixed()[:2]
    members = [mx.open_context(wl, precision=1) for wl in wls]
    members[1].set_seeds([3, 4], 2.6, 3.5)
    b = mx.Batch(members)
    b.step(1.0, 5)
    b.sync()
    assert not b.info()["fused"]
    a = mx.open_context(wls[1], precision=1)
    a.set_seeds([3, 4], 2.6, 3.5)
    a.step(1.0, 5)
    xa, va, fa, _ = a.get_state()
    x, v, f, _ = members[1].get_state()
    assert np.array_equal(x, xa) and np.array_equal(f, fa)
    b.close()
