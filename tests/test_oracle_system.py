"""Pins for the oracle's lists, regions, sets, force mixing and integrator (CPU).

* neighbour lists: cell-list result == O(N^2) enumeration;
* weights: closed form of the linear ramp (Alg. 2) at chosen distances, max
  over overlapping regions (Alg. 2 takes the max), cylinder distance;
* sets: brute-force enumeration of Lambda_k and its buffer (buffer-set
  equation, Sec. 4.5; Alg. 3);
* forces: central differences of the total energy, zero net force, rigid
  translation/rotation/permutation invariance for the pure potentials;
* mixing: the method (each potential on its set plus a one-cutoff buffer,
  Alg. 4) equals the plain blend of full forces (buffer sufficiency, Sec. 4.5),
  with a negative control; lambda = 1 and lambda = 0 reduce to the pure forces;
* velocity Verlet: time reversibility and the dt^2 energy-error law.
"""
import dataclasses

import numpy as np
import pytest

import _refmath as RM
from paper_2502_19081_gb300 import inputs as I


def _brute_sets(wl, x, lam, buf_e, buf_c):
    n = x.shape[0]
    L = wl.system.box_len
    per = np.array(wl.system.periodic, dtype=bool)
    d = x[None, :, :3] - x[:, None, :3]
    for k in range(3):
        if per[k]:
            d[:, :, k] = d[:, :, k] - L[k] * np.rint(d[:, :, k] * (1.0 / L[k]))
    r2 = d[:, :, 0] * d[:, :, 0] + d[:, :, 1] * d[:, :, 1] + d[:, :, 2] * d[:, :, 2]
    np.fill_diagonal(r2, np.inf)
    le = lam > 0
    lc = lam < 1
    ae = le | (~le & np.any((r2 < buf_e * buf_e) & le[None, :], axis=1))
    ac = lc | (~lc & np.any((r2 < buf_c * buf_c) & lc[None, :], axis=1))
    return le.astype(np.uint8) | (lc.astype(np.uint8) << 1) | (ae.astype(np.uint8) << 2) | (ac.astype(np.uint8) << 3)


def test_neighbour_cells_equal_brute_force(orc):
    cases = [(I.si_vacancy(), (5.0, 5.3)), (I.small_fe_box(1), (5.3, 5.8)),
             (I.cluster_workload(2, n=40, radius=7.0), (5.3, 5.8)),
             (I.fe_screw(n_atoms=3000, nrep_z=4), (5.5, 5.8))]
    for wl, rls in cases:
        s = wl.system
        for rl in rls:
            a = orc.neighbours(s.x, s.box_lo, s.box_len, s.periodic, rl, cap=256)
            b = orc.neighbours(s.x, s.box_lo, s.box_len, s.periodic, rl, cap=256, brute=True)
            assert np.array_equal(a[0], b[0])
            for i in range(s.n):
                assert np.array_equal(a[1][i, :a[0][i]], b[1][i, :b[0][i]])


def _outside_face_pairs(L, rl, rng):
    """Pairs of atoms whose minimum-image distance is just below rl, one atom of
    each pair 0.01-0.15 A outside a low or a high periodic face, its partner
    across that face; plus scattered atoms, some outside two faces at once."""
    pts = []
    for d in range(3):
        for side in (0, 1):
            for delta in (0.01, 0.05, 0.10, 0.15):
                for r in (rl - 0.10, rl - 0.03, rl - 0.005):
                    a = rng.uniform(0.3 * L, 0.7 * L, 3)
                    b = a + rng.normal(0.0, 0.01, 3)
                    if side == 0:
                        a[d] = -delta            # below the low face
                        b[d] = L - delta - r     # to its left, across the face
                    else:
                        a[d] = L + delta         # above the high face
                        b[d] = delta + r         # to its right, across the face
                    pts += [a, b]
    for _ in range(120):
        a = rng.uniform(0.0, L, 3)
        for d in rng.choice(3, size=int(rng.integers(1, 3)), replace=False):
            a[d] = -rng.uniform(0.01, 0.15) if rng.random() < 0.5 else L + rng.uniform(0.01, 0.15)
        pts.append(a)
    x = np.zeros((len(pts), 4))
    x[:, :3] = np.array(pts)
    return x


def test_neighbour_cells_outside_periodic_faces(orc):
    """Positions up to skin/2 outside a periodic face (the state between list
    rebuilds) in a box whose cell width exceeds the list radius by only
    0.013 A (Si 12x12x12, L = 65.172 A, 13 cells at r = 5.0): the cell-list
    result still equals the O(N^2) enumeration, and the cell ids are those of
    the folded coordinates."""
    L = 12 * 5.431
    box = np.array([L, L, L])
    rng = np.random.default_rng(11)
    x = _outside_face_pairs(L, 5.0, rng)
    outside = np.any((x[:, :3] < 0) | (x[:, :3] >= L), axis=1)
    assert outside.sum() > 150
    for rl in (5.0, 5.0 - 1e-3, 4.9):
        a = orc.neighbours(x, np.zeros(3), box, (1, 1, 1), rl, cap=64)
        b = orc.neighbours(x, np.zeros(3), box, (1, 1, 1), rl, cap=64, brute=True)
        assert b[0].sum() >= 144                     # every planted pair is a neighbour pair
        assert np.array_equal(a[0], b[0])
        for i in range(x.shape[0]):
            assert np.array_equal(a[1][i, :a[0][i]], b[1][i, :b[0][i]])
    nc, cid = orc.cells(x, np.zeros(3), box, (1, 1, 1), 5.0)
    assert list(nc) == [13, 13, 13]
    y = orc.wrap(x, box, (1, 1, 1))
    _, cy = orc.cells(y, np.zeros(3), box, (1, 1, 1), 5.0)
    assert np.array_equal(cid, cy)


def test_forces_and_sets_unchanged_by_periodic_images(orc):
    """Moving the atoms within 0.15 A of a face to their images just outside
    the opposite face (the state between list rebuilds) changes no set and no
    force beyond rounding, since every distance is a minimum image.  Si
    12x12x12 with a vacancy and 0.25 A displacements (so that pairs fall in
    the band a cell list with clamped rather than folded coordinates misses):
    13 cells at rc = 5.0 A, 0.013 A wider than rc."""
    wl = I.si_vacancy(ncell=12, sigma=0.25)
    s = wl.system
    assert abs(s.box_len[0] - 12 * 5.431) < 1e-9
    x0 = orc.wrap(s.x, s.box_len, s.periodic)
    shift = np.zeros_like(x0)
    for d in range(3):
        shift[x0[:, d] < 0.15, d] = s.box_len[d]
        shift[x0[:, d] > s.box_len[d] - 0.15, d] = -s.box_len[d]
    x1 = x0 + shift
    moved = np.any(shift != 0, axis=1)
    assert moved.sum() > 100
    assert np.any(x1[:, :3] >= s.box_len) and np.any(x1[:, :3] < 0)
    # pairs across a face at distances in (h - 0.15, rc): the band at stake
    nnb, nbr = orc.neighbours(x0, s.box_lo, s.box_len, s.periodic, 5.0, cap=64, brute=True)
    h = s.box_len[0] / 13
    band = 0
    for i in np.flatnonzero(moved):
        for j in nbr[i, :nnb[i]]:
            d = x0[j, :3] - x0[i, :3]
            if np.any(np.abs(d) > 0.5 * s.box_len[0]):
                d = d - s.box_len * np.rint(d / s.box_len)
                band += int(np.sqrt(d @ d) > h - 0.15)
    assert band > 10
    om = orc.Model(wl)
    assert np.array_equal(om.sets(x0), om.sets(x1))
    for mode in (orc.MODE_METHOD, orc.MODE_PURE_CHEAP):
        F0, _, _ = om.forces(x0, mode)
        F1, _, _ = om.forces(x1, mode)
        assert float(np.abs(F0[:, :3] - F1[:, :3]).max()) < 1e-10


def test_cells_in_range_and_rejects_small_boxes(orc):
    s = I.si_vacancy().system
    nc, cid = orc.cells(s.x, s.box_lo, s.box_len, s.periodic, 5.3)
    assert list(nc) == [3, 3, 3]
    assert cid.min() >= 0 and cid.max() < 27
    with pytest.raises(ValueError):
        orc.cells(s.x, s.box_lo, s.box_len, s.periodic, 6.0)     # fewer than 3 cells


def test_wrap_folds_into_box(orc):
    rng = np.random.default_rng(1)
    L = np.array([10.0, 12.0, 7.0])
    x = np.zeros((500, 4))
    x[:, :3] = rng.uniform(-30, 30, (500, 3))
    y = orc.wrap(x, L, (1, 1, 0))
    assert np.all(y[:, :2] >= 0) and np.all(y[:, 0] < 10.0) and np.all(y[:, 1] < 12.0)
    assert np.array_equal(y[:, 2], x[:, 2])
    k = (x[:, :2] - y[:, :2]) / L[:2]
    assert np.allclose(k, np.rint(k), atol=1e-9)


def _line_system(dists, axis_kind=I.REGION_SPHERE):
    n = len(dists)
    x = np.zeros((n, 4))
    x[:, 0] = 30.0 + np.asarray(dists)
    x[:, 1] = 30.0
    x[:, 2] = 30.0 + 3.0 * np.arange(n)        # varies along the cylinder axis
    wl = I.cluster_workload(1)
    sysm = I.System(x=x, v=np.zeros_like(x), mass=1.0, box_lo=np.zeros(3),
                    box_len=np.array([60.0, 60.0, 60.0 + 3 * n]), periodic=(0, 0, 0))
    return wl, sysm


@pytest.mark.parametrize("kind", [I.REGION_SPHERE, I.REGION_CYLINDER])
def test_lambda_closed_form(orc, kind):
    rc, w = 6.0, 2.0
    d = np.array([0.0, 3.0, rc - 1e-9, rc, rc + 0.5, rc + 1.0, rc + 1.5, rc + w - 1e-9, rc + w, rc + w + 1.0])
    wl, sysm = _line_system(d)
    centre = (30.0, 30.0, 30.0)
    reg = [I.Region(kind, centre, (0.0, 0.0, 1.0), rc, w)]
    if kind == I.REGION_SPHERE:
        dist = np.linalg.norm(sysm.x[:, :3] - np.array(centre), axis=1)
    else:
        dist = np.abs(d)
    m = orc.Model(system=sysm, ace=wl.ace, spline=wl.spline, regions=reg)
    lam, wgt = m.lam(sysm.x)
    expect = np.clip(1.0 - (dist - rc) / w, 0.0, 1.0)
    expect[dist < rc] = 1.0
    assert np.allclose(lam, expect, atol=1e-14, rtol=0)   # positions carry ~4e-15 A rounding
    assert np.array_equal(wgt, lam)
    if kind == I.REGION_CYLINDER:
        assert lam[3] == 1.0 and lam[4] == 0.75 and lam[5] == 0.5 and lam[8] == 0.0


def test_lambda_max_over_regions_and_cubic_blend(orc):
    d = np.linspace(0, 12, 25)
    wl, sysm = _line_system(d)
    r1 = I.Region(I.REGION_SPHERE, (30.0, 30.0, 30.0), (0, 0, 1), 2.0, 4.0)
    r2 = I.Region(I.REGION_SPHERE, (40.0, 30.0, 60.0), (0, 0, 1), 1.0, 8.0)
    m1 = orc.Model(system=sysm, ace=wl.ace, spline=wl.spline, regions=[r1])
    m2 = orc.Model(system=sysm, ace=wl.ace, spline=wl.spline, regions=[r2])
    m12 = orc.Model(system=sysm, ace=wl.ace, spline=wl.spline, regions=[r1, r2])
    l1, _ = m1.lam(sysm.x)
    l2, _ = m2.lam(sysm.x)
    l12, _ = m12.lam(sysm.x)
    assert np.array_equal(l12, np.maximum(l1, l2))
    mc = orc.Model(system=sysm, ace=wl.ace, spline=wl.spline, regions=[r1], blend=1)
    lc, wc = mc.lam(sysm.x)
    assert np.array_equal(lc, l1)
    assert np.allclose(wc, 3 * l1 ** 2 - 2 * l1 ** 3, atol=1e-15)


@pytest.mark.parametrize("name", ["si", "fe_box", "screw"])
def test_sets_match_brute_force(orc, name):
    if name == "si":
        wl = I.si_vacancy()
    elif name == "fe_box":
        wl = I.small_fe_box(3, r_core=4.0, ramp=3.0)
    else:
        wl = I.fe_screw(n_atoms=3000, nrep_z=4)
        wl.regions = [I.Region(I.REGION_CYLINDER, wl.regions[0].centre, (0, 0, 1), 6.0, 3.0)]
    m = orc.Model(wl)
    x = wl.system.x
    lam, _ = m.lam(x)
    f = m.sets(x)
    ref = _brute_sets(wl, x, lam, wl.ace.r_cut, wl.spline.r_cut)
    assert np.array_equal(f, ref)
    assert (f & 1).sum() > 0 and ((f & 2) > 0).sum() > 0
    assert ((f & 4) > 0).sum() > (f & 1).sum()          # a non-empty buffer


def _energy(m, x, mode):
    _, Ee, Ec = m.forces(x, mode)
    return Ee.sum() + Ec.sum()


@pytest.mark.parametrize("mode", [2, 3])
def test_forces_finite_difference_total_energy(orc, mode):
    wl = I.cluster_workload(8, n=20, radius=4.5, n_rad=5, l_max=3, body_order=4)
    m = orc.Model(wl)
    x = wl.system.x
    F, _, _ = m.forces(x, mode)
    h = 1e-5
    rng = np.random.default_rng(3)
    worst = 0.0
    for i in rng.choice(wl.system.n, 8, replace=False):
        for c in range(3):
            p = x.copy()
            p[i, c] += h
            q = x.copy()
            q[i, c] -= h
            fd = -(_energy(m, p, mode) - _energy(m, q, mode)) / (2 * h)
            worst = max(worst, abs(fd - F[i, c]))
    scale = max(1.0, np.sqrt(np.mean(np.sum(F[:, :3] ** 2, axis=1))))
    assert worst <= 1e-7 * scale


@pytest.mark.parametrize("mode", [2, 3])
def test_pure_forces_invariances(orc, mode):
    wl = I.small_fe_box(4, n_rad=5, l_max=3)
    m = orc.Model(wl)
    s = wl.system
    F, _, _ = m.forces(s.x, mode)
    assert np.abs(F[:, :3].sum(axis=0)).max() < 1e-12 * s.n
    # rigid translation (periodic box)
    xt = s.x.copy()
    xt[:, :3] = xt[:, :3] + np.array([0.37, -1.21, 2.05])
    xt[:, :3] = I.wrap_into_box(xt[:, :3], s.box_len, s.periodic)
    Ft, _, _ = m.forces(xt, mode)
    assert np.abs(Ft - F).max() < 1e-11
    # permutation
    perm = np.random.default_rng(5).permutation(s.n)
    Fp, _, _ = m.forces(s.x[perm], mode)
    assert np.abs(Fp - F[perm]).max() < 1e-11
    # exact symmetry of the cube: axis permutation x->y->z->x
    xr = s.x.copy()
    xr[:, :3] = s.x[:, [2, 0, 1]]
    Fr, _, _ = m.forces(xr, mode)
    assert np.abs(Fr[:, :3] - F[:, [2, 0, 1]]).max() < 1e-11


@pytest.mark.parametrize("mode", [2, 3])
def test_pure_forces_rotation_free_cluster(orc, mode):
    wl = I.cluster_workload(9, n=18, radius=4.5, n_rad=5, l_max=4, body_order=4)
    m = orc.Model(wl)
    x = wl.system.x
    F, _, _ = m.forces(x, mode)
    Q = RM.random_rotation(np.random.default_rng(2))
    xr = x.copy()
    xr[:, :3] = x[:, :3] @ Q.T
    Fr, _, _ = m.forces(xr, mode)
    assert np.abs(Fr[:, :3] - F[:, :3] @ Q.T).max() < 1e-11


@pytest.mark.parametrize("name", ["si", "fe_box"])
def test_method_equals_plain_blend(orc, name):
    wl = I.si_vacancy() if name == "si" else I.small_fe_box(6, r_core=4.0, ramp=3.0)
    m = orc.Model(wl)
    FB, _, _ = m.forces(wl.system.x, 0)
    FA, _, _ = m.forces(wl.system.x, 1)
    assert np.abs(FA - FB).max() < 1e-12
    # negative control: a buffer half an Angstrom short of the cutoff is not enough
    mneg = orc.Model(wl, buf_e=wl.ace.r_cut - 0.5, buf_c=wl.spline.r_cut - 0.5)
    FN, _, _ = mneg.forces(wl.system.x, 0)
    assert np.abs(FA - FN).max() > 1e-6


def test_lambda_limits_reduce_to_pure(orc):
    wl = I.small_fe_box(7, n_rad=5, l_max=3)
    s = wl.system
    big = [I.Region(I.REGION_SPHERE, tuple(s.box_len / 2), (0, 0, 1), 1000.0, 1.0)]
    none = [I.Region(I.REGION_SPHERE, tuple(s.box_len / 2), (0, 0, 1), 0.0, 0.0)]
    mb = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=big)
    mn = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=none)
    F1, _, _ = mb.forces(s.x, 0)
    Fe, _, _ = mb.forces(s.x, 2)
    assert np.abs(F1 - Fe).max() < 1e-12
    F0, _, _ = mn.forces(s.x, 0)
    Fc, _, _ = mn.forces(s.x, 3)
    assert np.abs(F0 - Fc).max() < 1e-12


def test_sampled_forces_equal_full(orc):
    wl = I.small_fe_box(8, r_core=4.0, ramp=3.0)
    m = orc.Model(wl)
    F, _, _ = m.forces(wl.system.x, 0)
    idx = np.array([0, 5, 17, 100, wl.system.n - 1])
    Fs = m.forces_sampled(wl.system.x, idx)
    assert np.abs(Fs - F[idx]).max() < 1e-12


def test_verlet_time_reversible(orc):
    wl = I.si_vacancy()
    m = orc.Model(wl)
    x0 = wl.system.x
    F, _, _ = m.forces(x0, 3)
    x1, v1, F1, _ = m.md(x0, wl.system.v, F, 1.0, 40, 3)
    x2, v2, F2, _ = m.md(x1, -v1, F1, 1.0, 40, 3)
    assert np.abs(x2[:, :3] - x0[:, :3]).max() < 1e-9
    assert np.abs(v2[:, :3] + wl.system.v[:, :3]).max() < 1e-11


def test_verlet_energy_error_dt_squared(orc):
    """Velocity Verlet's energy error scales as dt^2: halving dt over the same
    time shrinks max |E(t) - E(0)| by 4 (+-0.6)."""
    wl = I.si_vacancy()
    m = orc.Model(wl)
    x0, v0 = wl.system.x, wl.system.v
    F, Ee, _ = m.forces(x0, 2)
    e0 = Ee.sum()
    errs = []
    for dt, ns in ((1.0, 60), (0.5, 120)):
        x, v, Fc = x0, v0, F
        worst = 0.0
        xs, vs, Fs, ep = m.md(x, v, Fc, dt, ns, 2)
        # energies along the path: re-run in chunks to read kinetic energy
        x, v, Fc = x0, v0, F
        for s in range(ns):
            x, v, Fc, ep1 = m.md(x, v, Fc, dt, 1, 2)
            ke = 0.5 * wl.system.mass * np.sum(v[:, :3] ** 2) / orc.KAPPA
            worst = max(worst, abs(ep1[0] + ke - e0))
        errs.append(worst)
    ratio = errs[0] / errs[1]
    assert 3.4 <= ratio <= 4.6, (errs, ratio)
