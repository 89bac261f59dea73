"""The seeded generators produce the workloads they describe (CPU)."""
import math

import numpy as np

from paper_2502_19081_gb300 import inputs as I


def test_c1_c2_sizes_and_boxes():
    si = I.si_vacancy()
    assert si.system.n == 215 and np.allclose(si.system.box_len, 3 * 5.431)
    fe = I.fe_dumbbell()
    assert fe.system.n == 8001 and np.allclose(fe.system.box_len, [57.1, 57.1, 28.55])
    assert fe.ace.nu_max == 3 and fe.ace.n_rad == 10 and fe.ace.l_max == 4


def test_screw_cylinder_geometry():
    w = I.fe_screw(n_atoms=5000, nrep_z=4)
    x = w.system.x[:, :3]
    c = w.regions[0].centre
    r = np.hypot(x[:, 0] - c[0], x[:, 1] - c[1])
    assert w.system.n == 5000 and w.system.periodic == (0, 0, 1)
    assert np.all(x[:, 2] >= 0) and np.all(x[:, 2] < w.system.box_len[2])
    assert np.all(x[:, :2] > w.system.box_lo[:2]) and np.all(x[:, :2] < w.system.box_lo[:2] + w.system.box_len[:2])
    assert r.max() < 33.0            # sqrt(N / (rho pi Lz)) = 30.6 A plus thermal noise
    # no two sites closer than a bcc bond shortened by the core strain and noise
    # (sites on the displacement cut must not be pushed onto their column neighbours)
    d = x[:, None, :] - x[None, :, :]
    d[..., 2] -= w.system.box_len[2] * np.rint(d[..., 2] / w.system.box_len[2])
    r2 = np.einsum("ijk,ijk->ij", d, d)
    np.fill_diagonal(r2, 1e9)
    assert np.sqrt(r2.min()) > 1.5


def test_replica_batch_statistics():
    reps = I.si_replicas(256)
    ns = np.array([r.system.n for r in reps])
    assert len(reps) == 256
    assert ns.min() >= 215 and ns.max() <= 21000
    assert abs(ns.mean() - 6342) / 6342 < 0.15          # log-uniform on [1e3, 2e4]: mean 6342
    kinds = {r.extra["defect"] for r in reps}
    assert kinds == {"vacancy", "interstitial"}
    for r in reps[:10]:
        s = r.system
        ke = 0.5 * s.mass * np.sum(s.v[:, :3] ** 2) / 9.6485332e-3
        t = 2 * ke / (3 * (s.n - 1) * 8.617333262e-5)
        assert math.isclose(t, r.extra["temp_k"], rel_tol=1e-9)
        assert np.allclose(s.v[:, :3].sum(axis=0), 0.0, atol=1e-12)
        assert 300.0 <= r.extra["temp_k"] <= 1500.0


def test_interstitial_adds_and_vacancy_removes_an_atom():
    ace, spl = I.element_potentials("Si", np.random.default_rng(1), 5.0, 8, 3, 3)
    v = I.si_replica(1, 1728, "vacancy", 300.0, ace, spl)
    i = I.si_replica(1, 1728, "interstitial", 300.0, ace, spl)
    assert v.system.n == 1727 and i.system.n == 1729
