"""Writes paper_2502_19081_gb300/scales.json: the global scales of the random
parts of the two synthetic potentials, fixed once with the oracle so that on a
reference configuration the many-body part of the expensive potential and the
3-body part of the cheap potential each give a stated RMS force.

Usage:  python -m oracle.calibrate_scales
(Calls only the oracle; the generator reads the file it writes.)
"""
from __future__ import annotations

import dataclasses
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2502_19081_gb300 import inputs as I  # noqa: E402  (seeded generator only)

TARGET_ACE_RMS = 0.3      # eV/Angstrom, many-body part of the expensive potential
TARGET_SPLINE3_RMS = 0.2  # eV/Angstrom, 3-body part of the cheap potential

# (scale key, element, n_rad, l_max, body order, reference workload)
ACE_KEYS = [
    ("Si_n8_l3_b3", "Si", 8, 3, 3, "si"),
    ("Fe_n10_l4_b4", "Fe", 10, 4, 4, "fe"),
    ("Fe_n12_l5_b4", "Fe", 12, 5, 4, "fe"),
    ("Fe_n6_l3_b4", "Fe", 6, 3, 4, "fe"),
    ("Fe_n4_l2_b4", "Fe", 4, 2, 4, "fe"),
    ("Si_n6_l3_b4", "Si", 6, 3, 4, "si"),
    ("Si_n4_l2_b3", "Si", 4, 2, 3, "si"),
    ("Fe_n14_l6_b4", "Fe", 14, 6, 4, "fe"),
]


def _rms(F):
    return float(np.sqrt(np.mean(np.sum(F[:, :3] ** 2, axis=1))))


def _ref(kind):
    return I.si_vacancy() if kind == "si" else I.fe_dumbbell()


def main():
    out = I.load_scales()
    for key, el, n, L, bo, kind in ACE_KEYS:
        wl = _ref(kind)
        if (wl.ace.n_rad, wl.ace.l_max, wl.ace.nu_max + 1) == (n, L, bo):
            ace, spl = wl.ace, wl.spline          # the reference workload's own draw
        else:
            rng = np.random.default_rng(12345)
            ace, spl = I.element_potentials(el, rng, wl.ace.r_cut, n, L, bo, scale_key=key)
        s0 = float(out.get(f"ace:{key}", {}).get("value", 1.0))
        ace0 = dataclasses.replace(ace, pair=np.zeros(16))
        if el == "Si" and ace.nu_max >= 2:      # the random part alone, not the stored angular term
            ace0 = dataclasses.replace(ace0, c2=ace.c2 - I.si_angular_tables(n, L)[1])
        m = oracle.Model(system=wl.system, ace=ace0, spline=spl, regions=wl.regions)
        F, _, _ = m.forces(wl.system.x, oracle.MODE_PURE_EXP)
        rms = _rms(F)
        s = s0 * TARGET_ACE_RMS / rms
        out[f"ace:{key}"] = {"value": s, "reference": wl.name, "rms_target": TARGET_ACE_RMS}
        print(f"ace:{key}: rms {rms:.4g} at scale {s0:.4g} -> {s:.6g}")
    for el, kind in (("Si", "si"), ("Fe", "fe")):
        wl = _ref(kind)
        s0 = float(out.get(f"spline3:{el}", {}).get("value", 0.01))
        spl0 = dataclasses.replace(wl.spline, c2=np.zeros(16))
        if el == "Si":                            # the random 3-body part alone
            spl0 = dataclasses.replace(spl0, c3=wl.spline.c3 - I.si_angular_tables(wl.ace.n_rad, wl.ace.l_max)[0])
        m = oracle.Model(system=wl.system, ace=wl.ace, spline=spl0, regions=wl.regions)
        F, _, _ = m.forces(wl.system.x, oracle.MODE_PURE_CHEAP)
        rms = _rms(F)
        s = s0 * TARGET_SPLINE3_RMS / rms
        out[f"spline3:{el}"] = {"value": s, "reference": wl.name, "rms_target": TARGET_SPLINE3_RMS}
        print(f"spline3:{el}: rms {rms:.4g} at scale {s0:.4g} -> {s:.6g}")
    path = os.path.join(os.path.dirname(I.__file__), "scales.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print("wrote", path)


if __name__ == "__main__":
    main()
