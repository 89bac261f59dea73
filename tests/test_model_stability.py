"""Stability of the synthetic potentials (CPU, oracle MD).

The Si potentials' angular term:

* the expensive potential's stored nu = 2 addition equals, on a random
  environment, the double sum (A/2) sum_{j,k} g_j g_k (cos theta_jk + 1/3)^2
  it encodes through the addition theorem (the j = k part included; the pair
  spline carries its removal);
* with the angular term each pure potential keeps the diamond lattice from
  1500 K over 1000 velocity-Verlet steps (the first shell, 4 bonds near
  2.35 A, stays; without the term the lattice densifies), and without it the
  cheap potential does densify.

The Fe dumbbell cell's potentials (which the serving stream uses for its Fe
requests): a 1,000-atom bcc cell with a vacancy from 900 K keeps its neighbour
count over 200 steps with each pure potential (another random draw of the same
recipe collapses there).
"""
import dataclasses
import math
import os
import sys

import numpy as np
import pytest

from paper_2502_19081_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "oracle"))
import fit_si_angular as F  # noqa: E402  (the script that writes the stored tables)

KAPPA = 9.6485332e-3
KB = 8.617333262e-5


def test_expensive_angular_term_is_the_addition_theorem(orc):
    n, L = 8, 3
    _, c2a, _ = I.si_angular_tables(n, L)
    wl = I.cluster_workload(seed=3, element="Si", r_cut=5.0, n_rad=n, l_max=L, body_order=3)
    ace = dataclasses.replace(wl.ace, c1=np.zeros(n), c2=c2a, c3=np.zeros_like(wl.ace.c3), pair=np.zeros(16))
    m = orc.Model(system=wl.system, ace=ace, spline=wl.spline, regions=wl.regions)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((7, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = rng.uniform(2.0, 3.3, 7)
    E, _ = m.site(0, u * r[:, None])
    rg = np.linspace(0.3, F.RC, 800)
    w = np.where(rg < 1.6, 0.1, np.where(rg < F.G_CUT_EXP, 3.0, 6.0))
    c = np.linalg.lstsq(F.radial_basis(n, rg) * w[:, None], F.taper(rg, F.G_CUT_EXP) * w, rcond=None)[0]
    g = F.radial_basis(n, r) @ c
    ref = 0.5 * F.A_ANG * sum(g[j] * g[k] * (u[j] @ u[k] + 1.0 / 3.0) ** 2 for j in range(7) for k in range(7))
    assert abs(E - ref) < 1e-10 * max(1.0, abs(ref))


def _run(orc, mode, angular=True, temp=1500.0, steps=1000):
    wl = I.si_vacancy(seed=1)
    if not angular:
        c3a, c2a, pa = I.si_angular_tables(wl.ace.n_rad, wl.ace.l_max)
        wl.ace = dataclasses.replace(wl.ace, c2=wl.ace.c2 - c2a, pair=wl.ace.pair - pa)
        wl.spline = dataclasses.replace(wl.spline, c3=wl.spline.c3 - c3a)
    s = wl.system
    v = I.maxwell_boltzmann(np.random.default_rng(1), s.n, s.mass, temp)
    m = orc.Model(wl)
    x = s.x.copy()
    Fx, _, _ = m.forces(x, mode)
    x, v, Fx, _ = m.md(x, v, Fx, 1.0, steps, mode)
    nnb, nbr = orc.neighbours(x, s.box_lo, s.box_len, s.periodic, 3.3, cap=64)
    first = np.mean([np.sum(np.linalg.norm(
        (x[nbr[i, :nnb[i]], :3] - x[i, :3]) - s.box_len * np.rint((x[nbr[i, :nnb[i]], :3] - x[i, :3]) / s.box_len),
        axis=1) < 2.8) for i in range(s.n)])
    within = float(np.mean(nnb))
    return first, within


@pytest.mark.parametrize("which", ["cheap", "exp"])
def test_diamond_stays_with_the_angular_term(orc, which):
    mode = orc.MODE_PURE_CHEAP if which == "cheap" else orc.MODE_PURE_EXP
    first, within = _run(orc, mode)
    assert 3.7 <= first <= 4.2, first        # about 4 bonds (a vacancy and thermal motion)
    assert within < 4.6, within              # nothing but the first shell inside 3.3 A


def test_diamond_densifies_without_it(orc):
    _, within = _run(orc, orc.MODE_PURE_CHEAP, angular=False)
    assert within > 5.5, within


@pytest.mark.parametrize("which", ["cheap", "exp"])
def test_fe_dumbbell_potentials_keep_bcc(orc, which):
    pots = I.serve_potentials()
    wl = I.serve_request(7, "Fe", 1000, 0.08, 900.0, pots)
    s = wl.system
    mode = orc.MODE_PURE_CHEAP if which == "cheap" else orc.MODE_PURE_EXP
    m = orc.Model(wl)
    x, v = s.x.copy(), s.v.copy()
    Fx, _, _ = m.forces(x, mode)
    x, v, Fx, _ = m.md(x, v, Fx, 1.0, 200, mode)
    nnb, _ = orc.neighbours(x, s.box_lo, s.box_len, s.periodic, 5.8, cap=512)
    ke = 0.5 * s.mass * np.sum(v[:, :3] ** 2) / KAPPA
    temp = 2 * ke / (3 * (s.n - 1) * KB)
    assert nnb.max() < 90 and temp < 2000.0, (int(nnb.max()), temp)
