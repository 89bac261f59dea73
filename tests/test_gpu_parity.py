"""GPU path vs the FP64 CPU oracle, through the C ABI (libmix.so).

* cell assignment, neighbour lists, lambda, blend weights and evaluated sets:
  bit-exact;
* FP64 forces: max |dF| < 1e-10 eV/A against the oracle's method and plain
  definitions; site energies likewise;
* FP32 potential arithmetic: max |dF| <= 1e-3 eV/A (the accuracy gate);
* short trajectories, determinism, checkpoint/resume, host-buffer entry point,
  edge cases (empty system, capacity overflow, atom leaving the box), and the
  256,000-atom screw cylinder on sampled atoms.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2502_19081_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
GATE = 1e-3


@pytest.fixture(scope="module")
def mx():
    from paper_2502_19081_gb300 import build, mix
    build.build()
    return mix


def _rlist(wl, skin=None):
    return max(wl.ace.r_cut, wl.spline.r_cut) + (wl.skin if skin is None else skin)


def _cases():
    return {
        "si_vacancy_215": lambda: I.si_vacancy(),
        "fe_box_685": lambda: I.small_fe_box(11, r_core=4.0, ramp=3.0),
        "fe_box_l4": lambda: I.small_fe_box(12, n_rad=5, l_max=4, r_core=3.0, ramp=2.5),
        "cluster_60": lambda: I.cluster_workload(13, n=60, radius=8.0, n_rad=6, l_max=3, r_core=3.5, ramp=2.0),
        "screw_3000": lambda: I.fe_screw(n_atoms=3000, nrep_z=4),
        # n = 11: 6-wide q2 blocks in the float nu = 3 pass, with a ragged last block
        "fe_box_n11": lambda: I.small_fe_box(15, n_rad=11, l_max=3, r_core=3.0, ramp=2.0),
        # the largest shapes the library takes: n = 14 (rows padded to 16) and lmax = 6
        "fe_box_n14_l6": lambda: I.small_fe_box(24, n_rad=14, l_max=6, r_core=3.0, ramp=2.0),
        # the smallest padded rows: n = 4, lmax = 2
        "fe_box_n4_l2": lambda: I.small_fe_box(25, n_rad=4, l_max=2, r_core=3.0, ramp=2.0),
    }


CASES = list(_cases())


def _wl(name):
    wl = _cases()[name]()
    if name == "screw_3000":
        wl.regions = [I.Region(I.REGION_CYLINDER, wl.regions[0].centre, (0, 0, 1), 6.0, 3.0)]
    return wl


def _max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


@pytest.mark.parametrize("name", CASES)
def test_lists_and_cells_bit_exact(mx, name):
    wl = _wl(name)
    ctx = mx.open_context(wl)
    x, _, _, _ = ctx.get_state()
    s = wl.system
    nc, cid = ctx.cells()
    onc, ocid = oracle.cells(x, s.box_lo, s.box_len, s.periodic, _rlist(wl))
    assert np.array_equal(nc, onc) and np.array_equal(cid, ocid)
    nnb, nbr, rev = ctx.neighbours()
    onnb, onbr = oracle.neighbours(x, s.box_lo, s.box_len, s.periodic, _rlist(wl), cap=256)
    assert np.array_equal(nnb, onnb)
    for i in range(s.n):
        assert np.array_equal(nbr[i, :nnb[i]], onbr[i, :onnb[i]]), i
        js = nbr[i, :nnb[i]]
        assert np.all(nbr[js, rev[i, :nnb[i]]] == i)


def _rows_equal(nnb, nbr, onnb, onbr):
    """Sorted rows equal, compared as whole padded arrays."""
    if not np.array_equal(nnb, onnb):
        return False
    w = int(nnb.max()) if len(nnb) else 0
    cols = np.arange(w)[None, :]
    a = np.where(cols < nnb[:, None], nbr[:, :w], -1)
    b = np.where(cols < onnb[:, None], onbr[:, :w], -1)
    return bool(np.array_equal(a, b))


@pytest.mark.parametrize("kind", ["fe_box_40x40x20", "si_12cubed"])
def test_lists_bit_exact_cell_tiled_build(mx, kind):
    """Systems with at least 8 cells an SM take the build that stages each
    cell's stencil in shared memory: a bcc Fe box of 64,000 atoms (3,249
    cells) and the Si 12^3 cell (1,728 cells)."""
    if kind == "fe_box_40x40x20":
        wl = I.small_fe_box(41, nx=40, ny=40, nz=20, r_core=6.0, ramp=3.0)
    else:
        wl = I.si_vacancy(ncell=12, sigma=0.1)
    s = wl.system
    ctx = mx.open_context(wl)
    x, _, _, _ = ctx.get_state()
    nnb, nbr, rev = ctx.neighbours()
    onnb, onbr = oracle.neighbours(x, s.box_lo, s.box_len, s.periodic, _rlist(wl), cap=256)
    assert _rows_equal(nnb, nbr, onnb, onbr)
    for i in range(0, s.n, 97):
        js = nbr[i, :nnb[i]]
        assert np.all(nbr[js, rev[i, :nnb[i]]] == i)
    fl, _, _ = ctx.sets()
    assert np.array_equal(fl, oracle.Model(wl).sets(x))
    ctx.close()


@pytest.mark.parametrize("name", CASES)
def test_lambda_and_sets_bit_exact(mx, name):
    wl = _wl(name)
    ctx = mx.open_context(wl)
    x, _, _, _ = ctx.get_state()
    lam, w = ctx.lam()
    om = oracle.Model(wl)
    olam, ow = om.lam(x)
    assert np.array_equal(lam, olam) and np.array_equal(w, ow)
    fl, ae, ac = ctx.sets()
    ofl = om.sets(x)
    assert np.array_equal(fl, ofl)
    assert np.array_equal(ae, np.nonzero(ofl & 4)[0])
    assert np.array_equal(ac, np.nonzero(ofl & 8)[0])


@pytest.mark.parametrize("name", CASES)
def test_forces_fp64_match_oracle(mx, name):
    wl = _wl(name)
    ctx = mx.open_context(wl)
    x, _, F, _ = ctx.get_state()
    om = oracle.Model(wl)
    FB, Ee, Ec = om.forces(x, oracle.MODE_METHOD)
    FA, _, _ = om.forces(x, oracle.MODE_PLAIN)
    assert _max_abs(F[:, :3], FB[:, :3]) < TOL64
    assert _max_abs(F[:, :3], FA[:, :3]) < TOL64
    ee, ec = ctx.site_energies()
    fl, _, _ = ctx.sets()
    me, mc = (fl & 4) > 0, (fl & 8) > 0
    assert _max_abs(ee[me], Ee[me]) < TOL64 and _max_abs(ec[mc], Ec[mc]) < TOL64
    assert np.all(ee[~me] == 0) and np.all(ec[~mc] == 0)


@pytest.mark.parametrize("name", ["si_vacancy_215", "fe_box_685", "fe_box_l4", "cluster_60", "screw_3000", "fe_box_n11",
                                  "fe_box_n14_l6", "fe_box_n4_l2"])
def test_forces_fp32_within_gate(mx, name):
    wl = _wl(name)
    ctx = mx.open_context(wl, precision=mx.MIX_FP32)
    x, _, F, _ = ctx.get_state()
    FB, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
    err = _max_abs(F[:, :3], FB[:, :3])
    assert err <= GATE, err
    assert err > 0.0   # really the float path
    lam, _ = ctx.lam()
    olam, _ = oracle.Model(wl).lam(x)
    assert np.array_equal(lam, olam)       # weights stay float64


def test_lambda_limits_reduce_to_pure(mx):
    wl = I.small_fe_box(14, n_rad=5, l_max=3)
    s = wl.system
    big = [I.Region(I.REGION_SPHERE, tuple(s.box_len / 2), (0, 0, 1), 1000.0, 1.0)]
    om = oracle.Model(wl)
    ctx = mx.open_context(wl, regions=big)
    x, _, F, _ = ctx.get_state()
    Fe, _, _ = om.forces(x, oracle.MODE_PURE_EXP)
    assert _max_abs(F[:, :3], Fe[:, :3]) < TOL64
    ctx0 = mx.open_context(wl, regions=[])
    x0, _, F0, _ = ctx0.get_state()
    Fc, _, _ = om.forces(x0, oracle.MODE_PURE_CHEAP)
    assert _max_abs(F0[:, :3], Fc[:, :3]) < TOL64


def test_cubic_blend_and_buffer_override(mx):
    wl = I.small_fe_box(15, r_core=4.0, ramp=3.0)
    ctx = mx.open_context(wl, blend=mx.MIX_BLEND_CUBIC)
    x, _, F, _ = ctx.get_state()
    FB, _, _ = oracle.Model(wl, blend=1).forces(x, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], FB[:, :3]) < TOL64
    b = wl.ace.r_cut - 0.5
    ctxn = mx.open_context(wl, buffer_exp=b, buffer_cheap=b)
    xn, _, Fn, _ = ctxn.get_state()
    on = oracle.Model(wl, buf_e=b, buf_c=b)
    FN, _, _ = on.forces(xn, oracle.MODE_METHOD)
    assert _max_abs(Fn[:, :3], FN[:, :3]) < TOL64
    FA, _, _ = on.forces(xn, oracle.MODE_PLAIN)
    assert _max_abs(Fn[:, :3], FA[:, :3]) > 1e-6      # a short buffer is visibly wrong


def test_short_trajectory_matches_oracle(mx):
    wl = I.si_vacancy()
    ctx = mx.open_context(wl)
    x0, v0, F0, _ = ctx.get_state()
    ctx.step(wl.dt, 10)
    x, v, F, step = ctx.get_state()
    assert step == 10
    om = oracle.Model(wl)
    xo, vo, Fo, _ = om.md(x0, v0, F0, wl.dt, 10, oracle.MODE_METHOD)
    d = x[:, :3] - xo[:, :3]
    d -= wl.system.box_len * np.rint(d / wl.system.box_len)
    assert np.abs(d).max() < 1e-10
    assert _max_abs(v[:, :3], vo[:, :3]) < 1e-11
    assert _max_abs(F[:, :3], Fo[:, :3]) < TOL64
    # forces at the GPU's own final positions (re-evaluated on those exact bits)
    Fx, _, _ = om.forces(x, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], Fx[:, :3]) < TOL64


def test_checkpoints_along_a_trajectory(mx):
    wl = I.fe_dumbbell()
    ctx = mx.open_context(wl)
    om = oracle.Model(wl)
    for _ in range(2):
        ctx.step(wl.dt, 25)
        x, _, F, _ = ctx.get_state()
        fl, _, _ = ctx.sets()
        assert np.array_equal(fl, om.sets(x))
        FB, _, _ = om.forces(x, oracle.MODE_METHOD)
        assert _max_abs(F[:, :3], FB[:, :3]) < TOL64
    st = ctx.stats()
    assert st["rebuilds"] >= 1 and st["n_exp"] > 1000


def test_mid_interval_checkpoint_outside_periodic_faces(mx):
    """Between list rebuilds positions are folded only at the last rebuild, so
    atoms sit up to half a skin outside the periodic faces.  Si 12x12x12 with
    a vacancy (L = 65.172 A: the oracle's 13 cells at rc = 5 A are 0.013 A
    wider than rc) at 1500 K: at checkpoints with atoms outside the box the
    oracle re-evaluates sets and forces on the GPU's own bits."""
    wl = I.si_vacancy(ncell=12, sigma=0.1)
    rng = np.random.default_rng(3)
    s = wl.system
    wl.system = dataclasses.replace(s, v=I.maxwell_boltzmann(rng, s.n, s.mass, 1500.0))
    ctx = mx.open_context(wl)
    om = oracle.Model(wl)
    seen = 0
    for _ in range(3):
        ctx.step(wl.dt, 7)
        x, _, F, _ = ctx.get_state()
        out = np.any((x[:, :3] < 0) | (x[:, :3] >= s.box_len), axis=1)
        seen += int(out.sum() > 0)
        fl, _, _ = ctx.sets()
        assert np.array_equal(fl, om.sets(x))
        FB, _, _ = om.forces(x, oracle.MODE_METHOD)
        assert _max_abs(F[:, :3], FB[:, :3]) < TOL64
    assert seen >= 1


def test_deterministic_and_resumable(mx):
    wl = I.small_fe_box(16, r_core=4.0, ramp=3.0, sigma=0.15)
    a = mx.open_context(wl)
    a.step(1.0, 40)
    xa, va, fa, _ = a.get_state()
    b = mx.open_context(wl)
    b.step(1.0, 20)
    xs, vs, fs, st = b.get_state()
    c = mx.open_context(wl)
    c.set_state(xs, vs, fs, st)
    c.step(1.0, 20)
    xc, vc, fc, stc = c.get_state()
    assert stc == 40
    b.step(1.0, 20)
    xb, vb, fb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(fa, fb)
    # resuming rebuilds the lists at the saved positions, so the rebuild schedule
    # (and with it the fold of periodic coordinates) may differ: compare the physics
    d = xc[:, :3] - xa[:, :3]
    d -= wl.system.box_len * np.rint(d / wl.system.box_len)
    assert np.abs(d).max() < 1e-12 and _max_abs(vc, va) < 1e-12 and _max_abs(fc, fa) < 1e-10


@pytest.mark.parametrize("prec", [0, 2])
def test_potential_orders_give_the_same_bits(mx, prec):
    """The two potential kernels write disjoint arrays, so launching them on two
    branches in either order or one after the other on one stream gives the
    same trajectory bit for bit; the autotuner keeps one of the three orders
    and the state it found."""
    wl = I.small_fe_box(16, r_core=4.0, ramp=3.0, sigma=0.15)
    runs = []
    for order in (mx.MIX_ORDER_CHEAP_FIRST, mx.MIX_ORDER_EXP_FIRST, mx.MIX_ORDER_SERIAL):
        c = mx.open_context(wl, precision=prec, order=order)
        assert c.info()["potential_order"] == order
        c.step(1.0, 30)
        runs.append(c.get_state())
        if order == mx.MIX_ORDER_SERIAL:
            c.tune(2)
            assert c.info()["potential_order"] in (0, 1, 2)
            x0, v0, f0, s0 = runs[-1]
            x1, v1, f1, s1 = c.get_state()
            assert s1 == s0 and np.array_equal(x1, x0) and np.array_equal(v1, v0) and np.array_equal(f1, f0)
            c.step(1.0, 5)
            assert c.get_state()[3] == 35
        c.close()
    for x, v, f, st in runs[1:]:
        assert st == runs[0][3]
        assert np.array_equal(x, runs[0][0]) and np.array_equal(v, runs[0][1]) and np.array_equal(f, runs[0][2])
    with pytest.raises(mx.MixError):
        mx.Context(wl, precision=prec, order=3)


def test_tuning_leaves_the_trajectory_unchanged(mx):
    """A non-periodic Fe cylinder keeps warps for its cheap atoms until the
    autotuner, having measured the largest 3-body count, may try half warps;
    whatever shapes it keeps, the trajectory is the untuned one bit for bit."""
    wl = _wl("screw_3000")
    a = mx.open_context(wl, precision=1)
    b = mx.open_context(wl, precision=1)
    assert a.info()["cheap_lanes"] == 32
    a.step(1.0, 10)
    b.step(1.0, 10)
    b.sync()
    b.tune(2)
    assert b.info()["cheap_lanes"] in (16, 32)
    a.step(1.0, 30)
    b.step(1.0, 30)
    xa, va, fa, sa = a.get_state()
    xb, vb, fb, sb = b.get_state()
    assert sa == sb == 40
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(fa, fb)
    a.close()
    b.close()


def test_three_body_lane_groups_narrow_then_widen(mx):
    """A Si bulk: the uniform-density estimate puts the cheap kernel on warps,
    the first evaluation measures at most about 6 three-body neighbours and
    the context narrows to 8-lane groups (16 on-chip slots).  Moving 18 atoms
    into a dense spot 0.9 A apart then overflows those groups: the evaluation
    reports it and widens them to a warp; the repeat matches the oracle."""
    wl = I.si_vacancy(ncell=5)
    s = wl.system
    ctx = mx.open_context(wl, nbr_cap=128)
    assert ctx.info()["cheap_lanes"] == 8
    x, v, _, _ = ctx.get_state()
    _, _, F0, _ = ctx.get_state()
    FB0, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
    assert _max_abs(F0[:, :3], FB0[:, :3]) < TOL64      # the narrow groups give the same forces
    g = np.array([[i, j, k] for i in range(3) for j in range(3) for k in range(2)], float) * 0.9
    spot = s.box_len / 2 + 0.3 + g - g.mean(axis=0)
    far = np.argsort(-np.sum((x[:, :3] - s.box_len / 2) ** 2, axis=1))[:18]
    x2 = x.copy()
    x2[far, :3] = spot
    ctx.set_state(x2, v)
    with pytest.raises(mx.MixError) as e:
        ctx.forces()
        ctx.sync()
    assert e.value.code == mx.MIX_EOVERFLOW and "warp per atom" in str(e.value)
    assert ctx.info()["cheap_lanes"] == 32
    ctx.forces()
    ctx.sync()
    x3, _, F, _ = ctx.get_state()
    FB, _, _ = oracle.Model(wl).forces(x3, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], FB[:, :3]) < 1e-9 * max(1.0, float(np.abs(FB[:, :3]).max()))
    ctx.close()


def test_host_buffer_entry_point_matches_device_path(mx):
    wl = I.small_fe_box(17, r_core=4.0, ramp=3.0)
    a = mx.open_context(wl)
    x0, v0, f0, _ = a.get_state()
    a.step(1.0, 5)
    xa, va, fa, _ = a.get_state()
    b = mx.open_context(wl)
    xh, vh, fh = x0.copy(), v0.copy(), f0.copy()
    for _ in range(5):
        b.step_host(xh, vh, fh, 1.0, 1)
    d = xh[:, :3] - xa[:, :3]
    d -= wl.system.box_len * np.rint(d / wl.system.box_len)
    assert np.abs(d).max() < 1e-12 and _max_abs(vh, va) < 1e-12 and _max_abs(fh, fa) < 1e-10


def test_host_entry_point_with_page_locked_buffers(mx):
    """Page-locked host buffers (with and without forces in and out) give the
    device path's trajectory."""
    torch = pytest.importorskip("torch")
    wl = I.small_fe_box(17, r_core=4.0, ramp=3.0)
    a = mx.open_context(wl)
    x0, v0, f0, _ = a.get_state()
    a.step(1.0, 5)
    xa, va, fa, _ = a.get_state()
    b = mx.open_context(wl)
    hx, hv, hf = (torch.from_numpy(np.ascontiguousarray(t)).pin_memory() for t in (x0, v0, f0))
    xh, vh, fh = hx.numpy(), hv.numpy(), hf.numpy()
    for _ in range(5):
        b.step_host(xh, vh, fh, 1.0, 1)
    d = xh[:, :3] - xa[:, :3]
    d -= wl.system.box_len * np.rint(d / wl.system.box_len)
    assert np.abs(d).max() < 1e-12 and _max_abs(vh, va) < 1e-12 and _max_abs(fh, fa) < 1e-10
    # and the same buffers without forces in or out
    c = mx.open_context(wl)
    hx2, hv2 = (torch.from_numpy(np.ascontiguousarray(t)).pin_memory() for t in (x0, v0))
    c.step_host(hx2.numpy(), hv2.numpy(), None, 1.0, 5)
    d = hx2.numpy()[:, :3] - xa[:, :3]
    d -= wl.system.box_len * np.rint(d / wl.system.box_len)
    assert np.abs(d).max() < 1e-12 and _max_abs(hv2.numpy(), va) < 1e-12


def test_empty_system(mx):
    wl = I.cluster_workload(18, n=4)
    wl.system = I.System(x=np.zeros((0, 4)), v=np.zeros((0, 4)), mass=wl.system.mass,
                         box_lo=wl.system.box_lo, box_len=wl.system.box_len, periodic=(0, 0, 0))
    ctx = mx.Context(wl)
    ctx.forces()
    ctx.step(1.0, 3)
    ctx.sync()
    assert ctx.stats()["n_exp"] == 0


def test_capacity_overflow_is_reported_and_recovered(mx):
    wl = I.small_fe_box(19)
    ctx = mx.Context(wl, nbr_cap=32)
    with pytest.raises(mx.MixError) as e:
        ctx.forces()
        ctx.sync()
    assert e.value.code == mx.MIX_EOVERFLOW
    ok = mx.open_context(wl, nbr_cap=32)
    assert ok.cap > 32
    x, _, F, _ = ok.get_state()
    FB, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], FB[:, :3]) < TOL64


def test_atom_leaving_a_free_dimension_is_reported(mx):
    wl = I.cluster_workload(20, n=10)
    wl.system.x[0, 0] = wl.system.box_lo[0] + wl.system.box_len[0] + 1.0
    ctx = mx.Context(wl)
    with pytest.raises(mx.MixError) as e:
        ctx.forces()
        ctx.sync()
    assert e.value.code == mx.MIX_EBOX


def test_fe_dumbbell_full_size(mx):
    wl = I.fe_dumbbell()
    for prec, tol in ((0, TOL64), (1, GATE)):
        ctx = mx.open_context(wl, precision=prec)
        x, _, F, _ = ctx.get_state()
        om = oracle.Model(wl)
        FB, _, _ = om.forces(x, oracle.MODE_METHOD)
        assert _max_abs(F[:, :3], FB[:, :3]) < tol
        fl, _, _ = ctx.sets()
        assert np.array_equal(fl, om.sets(x))


def test_screw_cylinder_full_size_sampled(mx):
    wl = I.fe_screw()
    ctx = mx.open_context(wl)
    x, _, F, _ = ctx.get_state()
    om = oracle.Model(wl)
    fl, _, _ = ctx.sets()
    assert np.array_equal(fl, om.sets(x))
    lam, _ = ctx.lam()
    rng = np.random.default_rng(0)
    pick = []
    for sel in (lam == 1.0, (lam > 0) & (lam < 1), (lam == 0) & ((fl & 4) > 0), (fl & 4) == 0):
        idx = np.nonzero(sel)[0]
        pick += list(rng.choice(idx, 2, replace=False))
    Fs = om.forces_sampled(x, np.array(pick))
    assert _max_abs(F[pick, :3], Fs[:, :3]) < TOL64


def test_contexts_of_different_capacity_share_kernels(mx):
    """The expensive kernel's shared-memory size grows with the neighbour
    capacity; a context created later with a smaller capacity must not shrink
    the limit an earlier, larger one launches with."""
    wl = I.small_fe_box(16)
    big = mx.open_context(wl, nbr_cap=256)
    small = mx.open_context(wl, nbr_cap=96)
    big.forces()
    big.sync()
    x, _, F, _ = big.get_state()
    FB, _, _ = oracle.Model(wl).forces(x, oracle.MODE_METHOD)
    assert _max_abs(F[:, :3], FB[:, :3]) < TOL64
    xs, _, Fs, _ = small.get_state()
    assert np.array_equal(Fs, F)
