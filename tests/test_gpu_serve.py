"""Serving layer on the GPU (mix_server_*): requests joining and leaving a
running batch give, bit for bit, the trajectories they give alone; admission
waits for device memory; a request that fails (neighbour capacity) leaves
without disturbing the others; argument and state errors."""
import numpy as np
import pytest

import oracle
from paper_2502_19081_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DT = 1.0


@pytest.fixture(scope="module")
def mx():
    from paper_2502_19081_gb300 import build, mix
    build.build()
    return mix


def _alone(mx, wl, nsteps, precision):
    ctx = mx.Context(wl, precision=precision)
    ctx.forces()
    ctx.step(DT, nsteps)
    x, v, f, _ = ctx.get_state()
    ctx.close()
    return x, v, f


def _workloads():
    return [(I.si_vacancy(), 9), (I.small_fe_box(41), 14), (I.si_vacancy(seed=5), 5), (I.small_fe_box(42), 0)]


@pytest.mark.parametrize("precision", [0, 1])
def test_requests_in_the_mix_equal_alone(mx, precision):
    srv = mx.Server(DT)
    wls = _workloads()
    ids = [srv.submit(wls[0][0], wls[0][1], precision=precision)]
    srv.tick(2)
    ids.append(srv.submit(wls[1][0], wls[1][1], precision=precision))
    srv.tick(1)
    ids += [srv.submit(w, n, precision=precision) for w, n in wls[2:]]
    seen_active = 0
    for _ in range(100):
        t = srv.tick(3)
        seen_active = max(seen_active, t["active"])
        if t["active"] == 0 and t["queued"] == 0:
            break
    assert seen_active >= 3
    for rid, (wl, nsteps) in zip(ids, wls):
        info = srv.request(rid)
        assert info["state"] == mx.MIX_REQ_DONE and info["steps_done"] == nsteps
        assert info["t_admit"] >= info["t_submit"] and info["t_done"] >= info["t_admit"]
        x, v, f = srv.fetch(rid)
        xa, va, fa = _alone(mx, wl, nsteps, precision)
        assert np.array_equal(x, xa) and np.array_equal(v, va) and np.array_equal(f, fa)
        # and the oracle on the served request's final bits
        FB, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
        assert np.abs(f[:, :3] - FB[:, :3]).max() < (1e-10 if precision == 0 else 1e-3)
    srv.close()


def test_admission_waits_for_device_memory(mx):
    a, b = I.small_fe_box(43), I.small_fe_box(44)
    probe = mx.Server(DT)
    r = probe.submit(a, 1)
    need = probe.request(r)["device_bytes"]
    probe.close()
    srv = mx.Server(DT, hbm_budget=need + need // 2)       # room for one request only
    ra, rb = srv.submit(a, 4), srv.submit(b, 3)
    t = srv.tick(2)
    assert t["admitted"] == 1 and t["active"] == 1 and t["queued"] == 1 and t["bytes_in_use"] == need
    assert srv.request(rb)["state"] == mx.MIX_REQ_QUEUED
    while srv.request(ra)["state"] != mx.MIX_REQ_DONE:
        srv.tick(2)
    t = srv.tick(1)
    assert srv.request(rb)["state"] in (mx.MIX_REQ_ACTIVE, mx.MIX_REQ_DONE)
    while srv.request(rb)["state"] != mx.MIX_REQ_DONE:
        srv.tick(2)
    ia, ib = srv.request(ra), srv.request(rb)
    assert ib["t_admit"] >= ia["t_done"]
    xb, vb, fb = srv.fetch(rb)
    xa_, va_, fa_ = _alone(mx, b, 3, mx.MIX_FP32)
    assert np.array_equal(xb, xa_) and np.array_equal(fb, fa_)
    srv.close()


def test_a_failing_request_leaves_the_others_alone(mx):
    good, bad = I.si_vacancy(), I.small_fe_box(45)
    srv = mx.Server(DT)
    rg = srv.submit(good, 6)
    rb = srv.submit(bad, 6, nbr_cap=8)          # far below the ~60 neighbours of bcc Fe
    for _ in range(20):
        t = srv.tick(2)
        if t["active"] == 0 and t["queued"] == 0:
            break
    assert srv.request(rb)["state"] == mx.MIX_REQ_FAILED
    assert srv.request(rb)["status"] == mx.MIX_EOVERFLOW
    with pytest.raises(mx.MixError) as e:
        srv.fetch(rb)
    assert e.value.code == mx.MIX_EOVERFLOW
    assert srv.request(rg)["state"] == mx.MIX_REQ_DONE
    x, v, f = srv.fetch(rg)
    xa, va, fa = _alone(mx, good, 6, mx.MIX_FP32)
    assert np.array_equal(x, xa) and np.array_equal(f, fa)
    srv.close()


def test_server_errors(mx):
    srv = mx.Server(DT, hbm_budget=1 << 20)
    with pytest.raises(mx.MixError) as e:
        srv.submit(I.small_fe_box(46), 2)               # needs more than 1 MiB
    assert e.value.code == mx.MIX_ENOMEM
    srv.close()
    srv = mx.Server(DT)
    rid = srv.submit(I.si_vacancy(), 50)
    with pytest.raises(mx.MixError) as e:
        srv.fetch(rid)
    assert e.value.code == mx.MIX_ESTATE
    with pytest.raises(mx.MixError):
        srv.request(rid + 100)
    with pytest.raises(mx.MixError):
        srv.tick(0)
    srv.close()          # releases the unfinished request's memory
