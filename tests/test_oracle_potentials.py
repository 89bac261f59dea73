"""Pins for the oracle's two synthetic potentials (CPU only).

Each check compares the oracle with something other than itself: scipy's
spherical harmonics, quadrature of scipy-built Y products, the addition theorem
plus sphere quadrature for the many-body basis, scipy B-splines for the cheap
potential, central finite differences for the gradients (the force equation of
Sec. 4.5 is a derivative of site energies), and exact invariances.
"""
import math

import numpy as np
import pytest

import _refmath as RM
from paper_2502_19081_gb300 import inputs as I


def _unit(rng, k):
    u = rng.standard_normal((k, 3))
    return u / np.linalg.norm(u, axis=1)[:, None]


def test_ylm_convention_matches_scipy(orc):
    rng = np.random.default_rng(0)
    us = _unit(rng, 40)
    us[0] = [0.0, 0.0, 1.0]
    us[1] = [0.0, 0.0, -1.0]
    us[2] = [1.0, 0.0, 0.0]
    for l in range(7):
        for m in range(-l, l + 1):
            ref = RM.real_ylm_scipy(l, m, us)
            got = np.array([orc.ylm(l, m, u) for u in us])
            assert np.allclose(got, ref, atol=1e-12, rtol=1e-12), (l, m)


def test_gaunt_matches_quadrature(orc):
    # every l up to 6 (the largest lmax the library takes; C3 uses 5): the
    # quadrature integrates products of degree 3 L = 18 exactly
    L = 6
    pts, w = RM.sphere_quadrature(3 * L)
    Y = {(l, m): RM.real_ylm_scipy(l, m, pts) for l in range(L + 1) for m in range(-l, l + 1)}
    worst = 0.0
    for l1 in range(L + 1):
        for l2 in range(l1, L + 1):
            for l3 in range(l2, L + 1):
                for m1 in range(-l1, l1 + 1):
                    for m2 in range(-l2, l2 + 1):
                        for m3 in range(-l3, l3 + 1):
                            q = float(np.dot(w, Y[l1, m1] * Y[l2, m2] * Y[l3, m3]))
                            g = orc.gaunt(l1, m1, l2, m2, l3, m3)
                            worst = max(worst, abs(q - g))
    assert worst < 1e-13


def test_gaunt_special_values(orc):
    # integral of Y_lm Y_lm Y_00 = Y_00 = 1/sqrt(4 pi); odd l-sum vanishes
    for l in range(7):
        for m in range(-l, l + 1):
            assert abs(orc.gaunt(0, 0, l, m, l, m) - 1.0 / math.sqrt(4 * math.pi)) < 1e-14
    assert orc.gaunt(1, 0, 1, 0, 1, 0) == pytest.approx(0.0, abs=1e-15)


def _env(rng, k=14, rmin=2.0, rmax=5.2):
    u = _unit(rng, k)
    r = rng.uniform(rmin, rmax, k)
    return u * r[:, None]


@pytest.mark.parametrize("el,n,L,bo", [("Fe", 4, 2, 4), ("Fe", 6, 3, 4), ("Si", 4, 2, 3), ("Fe", 5, 4, 4),
                                      ("Fe", 12, 5, 4), ("Fe", 4, 6, 4)])
def test_ace_basis_addition_theorem(orc, el, n, L, bo):
    rng = np.random.default_rng(n * 10 + L)
    wl = I.cluster_workload(seed=3, element=el, n_rad=n, l_max=L, body_order=bo)
    m = orc.Model(wl)
    rij = _env(rng)
    E, g, B = m.site(0, rij, want_basis=True)
    Bref = RM.ace_basis_ref(wl.ace, rij)
    assert B.shape == Bref.shape
    scale = max(1.0, np.abs(Bref).max())
    assert np.abs(B - Bref).max() < 1e-11 * scale
    Eref = RM.ace_site_energy_ref(wl.ace, rij)
    assert abs(E - Eref) < 1e-11 * max(1.0, abs(Eref))


def test_ace_basis_count_matches_enumeration(orc):
    for name, expect in (("si_vacancy_215", 152), ("fe_dumbbell_8001", 7895)):
        wl = I.workload(name)
        m = orc.Model(wl)
        assert m.basis_count() == expect == len(RM.ace_labels(wl.ace.n_rad, wl.ace.l_max, wl.ace.nu_max))


def test_ace_basis_rotation_invariant(orc):
    rng = np.random.default_rng(7)
    wl = I.cluster_workload(seed=4, n_rad=6, l_max=4, body_order=4)
    m = orc.Model(wl)
    rij = _env(rng, 18)
    _, _, B = m.site(0, rij, want_basis=True)
    for _ in range(3):
        Q = RM.random_rotation(rng)
        _, _, B2 = m.site(0, rij @ Q.T, want_basis=True)
        assert np.abs(B - B2).max() < 1e-12 * max(1.0, np.abs(B).max())
    # inversion (O(3)): even l-sums make the basis parity-even
    _, _, B3 = m.site(0, -rij, want_basis=True)
    assert np.abs(B - B3).max() < 1e-12 * max(1.0, np.abs(B).max())


def test_cheap_energy_matches_scipy_bsplines(orc):
    rng = np.random.default_rng(11)
    for el in ("Fe", "Si"):
        wl = I.cluster_workload(seed=5, element=el, r_cut=5.5 if el == "Fe" else 5.0)
        m = orc.Model(wl)
        rij = _env(rng, 12, 1.9, 5.4)
        E, _ = m.site(1, rij)
        Eref = RM.cheap_site_energy_ref(wl.spline, rij)
        assert abs(E - Eref) < 1e-12 * max(1.0, abs(Eref))


def test_radial_and_pair_vanish_at_cutoff(orc):
    wl = I.cluster_workload(seed=6)
    m = orc.Model(wl)
    rc = wl.ace.r_cut
    for which in (0, 1):
        rij = np.array([[rc - 1e-9, 0.0, 0.0], [0.0, 2.5, 0.0]])
        E1, g1 = m.site(which, rij)
        rij2 = np.array([[rc + 1e-3, 0.0, 0.0], [0.0, 2.5, 0.0]])
        E2, g2 = m.site(which, rij2)
        assert abs(E1 - E2) < 1e-9
        assert np.abs(g1[0]).max() < 1e-9 and np.abs(g2[0]).max() == 0.0


@pytest.mark.parametrize("which", [0, 1])
def test_site_gradient_finite_difference(orc, which):
    """dE_i/dr_ij from the oracle vs central differences, h = 1e-5 A."""
    rng = np.random.default_rng(21 + which)
    wl = I.cluster_workload(seed=7, n_rad=6, l_max=4, body_order=4)
    m = orc.Model(wl)
    rij = _env(rng, 16, 1.9, 5.3)
    rij[:6] = _env(rng, 6, 1.9, 3.1)   # several inside the 3-body cutoff
    E, g = m.site(which, rij)
    h = 1e-5
    fd = np.zeros_like(g)
    for j in range(rij.shape[0]):
        for c in range(3):
            p = rij.copy()
            p[j, c] += h
            q = rij.copy()
            q[j, c] -= h
            fd[j, c] = (m.site(which, p)[0] - m.site(which, q)[0]) / (2 * h)
    scale = max(1.0, np.sqrt(np.mean(g ** 2)))
    assert np.abs(g - fd).max() <= 1e-7 * scale
