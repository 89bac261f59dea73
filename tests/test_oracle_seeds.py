"""Pins for the oracle's seed-atom weights (Alg. 1-2) and coordination counts
(the neighbour-count defect criterion of the Si vacancy runs, Sec. 4.6).

* coordination within 4 A on a perfect diamond lattice is 16 everywhere; with
  one vacancy exactly the 16 atoms within 4 A of the empty site have 15;
* a single seed with r_core below the nearest-neighbour distance gives the same
  weights, bit for bit, as a geometric sphere of radius 0 and ramp r_blend at
  the seed's position (the atom form of Alg. 2 reduces to the ramp);
* several seeds combine by the maximum (Alg. 2 takes a max);
* every atom within r_core of a seed is a core atom (brute-force distances);
* force mixing with these weights still equals the plain blend (Sec. 4.5).
"""
import numpy as np
import pytest

from paper_2502_19081_gb300 import inputs as I


def _diamond(ncell=3, remove_centre=False):
    a = 5.431
    q = I.diamond_lattice(ncell, ncell, ncell)
    site = None
    if remove_centre:
        ctr = np.array([2 * ncell] * 3)
        k = int(np.argmin(np.sum((q - ctr) ** 2, axis=1)))
        site = q[k] * a / 4.0
        q = np.delete(q, k, axis=0)
    pos = q * a / 4.0
    wl = I.si_vacancy()
    sysm = I.System(x=I._pack(pos), v=np.zeros((pos.shape[0], 4)), mass=I.MASS_SI, box_lo=np.zeros(3),
                    box_len=np.full(3, ncell * a), periodic=(1, 1, 1))
    return wl, sysm, site


def _mic(d, L):
    return d - L * np.rint(d / L)


def test_coordination_perfect_and_vacancy(orc):
    wl, s, _ = _diamond()
    m = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=wl.regions)
    assert np.all(m.coordination(s.x, 4.0) == 16)
    wl, s, site = _diamond(remove_centre=True)
    m = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=wl.regions)
    z = m.coordination(s.x, 4.0)
    d = np.linalg.norm(_mic(s.x[:, :3] - site, s.box_len), axis=1)
    assert np.array_equal(np.nonzero(z == 15)[0], np.nonzero(d < 4.0)[0])
    assert (z == 15).sum() == 16 and np.all(z[d >= 4.0] == 16)


def test_single_seed_small_core_equals_geometric_ramp(orc):
    wl = I.small_fe_box(21)
    s = wl.system
    seed = 123
    rb = 4.5
    m = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=[])
    m.set_atomic([seed], 1.0, rb)
    lam_a, w_a = m.lam(s.x)
    geo = [I.Region(I.REGION_SPHERE, tuple(s.x[seed, :3]), (0, 0, 1), 0.0, rb)]
    mg = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=geo)
    lam_g, _ = mg.lam(s.x)
    assert np.array_equal(lam_a, lam_g)
    assert lam_a[seed] == 1.0 and (lam_a > 0).sum() > 10


def test_seeds_combine_by_max_and_core_radius(orc):
    wl = I.small_fe_box(22)
    s = wl.system
    rcore, rb = 2.6, 3.0
    ma = orc.Model(system=s, ace=wl.ace, spline=wl.spline, regions=[])
    ma.set_atomic([10], rcore, rb)
    la, _ = ma.lam(s.x)
    ma.set_atomic([400], rcore, rb)
    lb, _ = ma.lam(s.x)
    ma.set_atomic([10, 400], rcore, rb)
    lab, _ = ma.lam(s.x)
    assert np.array_equal(lab, np.maximum(la, lb))
    for seed in (10, 400):
        d = np.linalg.norm(_mic(s.x[:, :3] - s.x[seed, :3], s.box_len), axis=1)
        assert np.all(lab[d < rcore - 1e-9] == 1.0)
    core = lab == 1.0
    dmat = np.linalg.norm(_mic(s.x[None, :, :3] - s.x[:, None, :3], s.box_len), axis=2)
    expect = np.where(core, 1.0, np.max(np.where(core[None, :] & (dmat < rb), 1.0 - dmat / rb, 0.0), axis=1))
    assert np.allclose(lab, expect, atol=1e-14, rtol=0)


def test_mixing_identity_with_seed_weights(orc):
    wl = I.small_fe_box(23)
    m = orc.Model(wl)
    m.set_atomic([5, 6, 300], 2.6, 4.0)
    FB, _, _ = m.forces(wl.system.x, 0)
    FA, _, _ = m.forces(wl.system.x, 1)
    assert np.abs(FA - FB).max() < 1e-12
    fl = m.sets(wl.system.x)
    assert (fl & 1).sum() > 0 and ((fl & 4) > 0).sum() > (fl & 1).sum()
