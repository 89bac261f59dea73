"""Writes paper_2502_19081_gb300/si_angular.json: an angular three-body term
A sum_{j<k} g(r_ij) g(r_ik) (cos theta_jik + 1/3)^2 for the two synthetic Si
potentials, so that the diamond lattice is a stable minimum (a pair term with
random many-body terms has no angular stiffness and densifies within a few
hundred steps).  The paper's Si potentials are trained ACE and UF3 fits
(Sec. 2.1) whose angular terms come from DFT; this is a synthetic stand-in in
the spirit of the Stillinger-Weber bond-bending term, matched between the two
potentials as the paper's distillation (Sec. 4.1) matches them.

A = 10 eV in both, and the same g: the first-shell taper
sum_{a <= 4} B_a(r / h3) of the cheap 3-body basis with its cutoff at 3.4 A
(between the first and second shells; the cheap Si potential takes that 3-body
cutoff instead of rc 3.5/6 = 2.9 A, where the bond length would sit on the
steep end of the taper and the expensive potential's basis could not follow
it).  Two angular terms that differ turn force mixing into a heat source, so
they are matched.

* cheap potential (2+3-body cubic B-spline): g as above, and
  the angular factor is a least-squares cubic B-spline in r_jk of
  (4/3 - r_jk^2 / (2 r0^2))^2 (cos theta at the bond length r0), so that
  c3[a][b][c] += A t_c for a, b <= 4;
* expensive potential (linear ACE): g is fitted onto its radial basis,
  g = sum_n c_n R_n, and the addition theorem sum_m Y_lm(u) Y_lm(v) =
  (2l + 1) / (4 pi) P_l(u . v) with (cos + 1/3)^2 = (4/9) P_0 + (2/3) P_1 +
  (2/3) P_2 turns the term into nu = 2 coefficients
  c2[l][n1][n2] += (A/2) f_l 4 pi / (2l + 1) c_n1 c_n2 (twice that for
  n1 < n2); the j = k part this adds, (8A/9) sum_j g(r_ij)^2, is removed from
  the pair spline by a least-squares fit of -(16A/9) g^2.

Usage:  python -m oracle.fit_si_angular
(numpy only; the generator reads the file it writes.)
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
from numpy.polynomial import chebyshev as C
from scipy.interpolate import BSpline

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "paper_2502_19081_gb300", "si_angular.json")

A_ANG = 10.0                           # eV, both potentials
R0 = 5.431 * math.sqrt(3.0) / 4.0      # Si bond length, Angstrom
RC = 5.0                               # Si cutoff of both potentials
RC3 = 3.4                              # 3-body cutoff of the cheap Si potential: between the
                                       # first (2.35 A) and second (3.84 A) shells
G_CUT_EXP = RC3                        # g of the expensive potential ends there too
# (n_rad, l_max) of the Si expensive potentials the workloads use
ACE_SHAPES = [(8, 3), (4, 2), (6, 3)]


def bspline_basis(h: float, x: np.ndarray, nb: int) -> np.ndarray:
    """Cubic B-splines B_c on uniform knots (c - 3) h, c < nb, at x."""
    t = (np.arange(nb + 4) - 3.0) * h
    out = np.zeros((x.size, nb))
    for c in range(nb):
        coef = np.zeros(nb)
        coef[c] = 1.0
        out[:, c] = BSpline(t, coef, 3, extrapolate=False)(x)
    return np.nan_to_num(out)


def taper(r: np.ndarray, cut: float) -> np.ndarray:
    """g(r) = sum_{a <= 4} B_a(r / h), h = cut / 5: the cubic B-spline partition
    of unity with its last three functions (the ones reaching the cut) left out."""
    return bspline_basis(cut / 5.0, r, 8)[:, :5].sum(axis=1)


def radial_basis(n: int, r: np.ndarray) -> np.ndarray:
    """R_q(r) = T_q(2 r / rc - 1) (1 - (r / rc)^2)^3, q < n."""
    s = 2.0 * r / RC - 1.0
    fc = np.where(r < RC, (1.0 - (r / RC) ** 2) ** 3, 0.0)
    return np.stack([C.chebval(s, np.eye(n)[q]) * fc for q in range(n)], axis=1)


def cheap_angular():
    hc = 2.0 * RC3 / 5.0
    x = np.linspace(0.0, 2.0 * RC3, 600)
    f = (4.0 / 3.0 - x * x / (2.0 * R0 * R0)) ** 2
    w = 1.0 + 20.0 * np.exp(-((x - 2.0 * R0 * math.sqrt(2.0 / 3.0)) / 0.5) ** 2)
    B = bspline_basis(hc, x, 8)
    t = np.linalg.lstsq(B * w[:, None], f * w, rcond=None)[0]
    c3 = np.zeros((8, 8, 8))
    c3[:5, :5, :] = A_ANG * t[None, None, :]
    return c3, float(np.abs(B @ t - f)[(x > 3.3) & (x < 4.4)].max())


def ace_angular(n: int, L: int):
    # weights: the bond range, and zero beyond G_CUT_EXP held firmly (no angular
    # term on the second and third shells); below 1.6 A (closer than Si atoms
    # come) loosely
    r = np.linspace(0.3, RC, 800)
    w = np.where(r < 1.6, 0.1, np.where(r < G_CUT_EXP, 3.0, 6.0))
    R = radial_basis(n, r)
    g_t = taper(r, G_CUT_EXP)
    c = np.linalg.lstsq(R * w[:, None], g_t * w, rcond=None)[0]
    g = R @ c
    f = {0: 4.0 / 9.0, 1: 2.0 / 3.0, 2: 2.0 / 3.0}
    c2 = np.zeros((L + 1, n, n))
    for l, fl in f.items():
        if l > L:
            continue
        k = 0.5 * A_ANG * fl * 4.0 * math.pi / (2 * l + 1)
        for a in range(n):
            for b in range(a, n):
                c2[l, a, b] = k * c[a] * c[b] * (1.0 if a == b else 2.0)
    # the j = k part of the double sum, as a pair term 1/2 sum_j V(r_ij): V = (16 A / 9) g^2
    h = RC / 13.0
    rp = np.linspace(1.6, RC, 1000)
    Rp = radial_basis(n, rp)
    vself = 16.0 * A_ANG / 9.0 * (Rp @ c) ** 2
    Bp = bspline_basis(h, rp, 16)[:, :13]
    wp = np.where((rp > 2.0) & (rp < 3.0), 10.0, 1.0)    # the bond range first
    p = np.linalg.lstsq(Bp * wp[:, None], vself * wp, rcond=None)[0]
    pair = np.zeros(16)
    pair[:13] = -p
    bond = (rp > 2.0) & (rp < 3.0)
    return c2, pair, float(np.abs(g - g_t)[r > G_CUT_EXP].max()), float(np.abs(Bp @ p - vself)[bond].max())


def main():
    c3, ferr = cheap_angular()
    out = {"A_eV": A_ANG, "g_cut": G_CUT_EXP, "r0": R0, "note": "angular term A sum_{j<k} g g (cos + 1/3)^2 of the Si potentials",
           "cheap_c3_add": c3.tolist(), "cheap_fit_err_near_bond": ferr, "ace": {}}
    for n, L in ACE_SHAPES:
        c2, pair, gres, perr = ace_angular(n, L)
        out["ace"][f"n{n}_l{L}"] = {"c2_add": c2.tolist(), "pair_add": pair.tolist(),
                                    "g_residual_beyond_cut": gres, "pair_fit_err_2_3A": perr}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"wrote {OUT}: cheap fit err {ferr:.2e}; " +
          ", ".join(f"{k}: g residual {v['g_residual_beyond_cut']:.3f}, pair err (2-3 A) {v['pair_fit_err_2_3A']:.2e}"
                    for k, v in out["ace"].items()))


if __name__ == "__main__":
    main()
