"""Independent test-side mathematics used to pin the oracle.

Nothing here re-types the oracle's formulas: spherical harmonics come from
scipy's complex Y_l^m, Chebyshev polynomials from numpy, B-splines from scipy,
Legendre polynomials from scipy, and the many-body basis is rebuilt through the
addition theorem and sphere quadrature instead of Gaunt coefficients.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp
from numpy.polynomial import chebyshev as C
from scipy.interpolate import BSpline


def real_ylm_scipy(l: int, m: int, u: np.ndarray) -> np.ndarray:
    """Real orthonormal Y_lm without Condon-Shortley phase, from scipy's complex
    Y_l^m (which carries the phase): m>0: sqrt2 (-1)^m Re Y_l^m;
    m<0: sqrt2 (-1)^|m| Im Y_l^|m|; m=0: Y_l^0."""
    u = np.atleast_2d(u)
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    mu = abs(m)
    y = sp.sph_harm_y(l, mu, theta, phi)
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * y.real
    if m < 0:
        return math.sqrt(2.0) * (-1) ** mu * y.imag
    return y.real


def sphere_quadrature(degree: int):
    """Nodes (K,3) and weights (K,) integrating polynomials up to `degree`
    exactly over the unit sphere (Gauss-Legendre in cos(theta) x uniform phi)."""
    nt = degree // 2 + 2
    npf = degree + 2
    z, wz = np.polynomial.legendre.leggauss(nt)
    phi = 2.0 * np.pi * np.arange(npf) / npf
    Z, P = np.meshgrid(z, phi, indexing="ij")
    W = np.outer(wz, np.full(npf, 2.0 * np.pi / npf))
    s = np.sqrt(1.0 - Z ** 2)
    pts = np.stack([s * np.cos(P), s * np.sin(P), Z], axis=-1).reshape(-1, 3)
    return pts, W.reshape(-1)


def radial_ref(n_rad: int, rc: float, r: np.ndarray) -> np.ndarray:
    """R_n(r) = T_n(2r/rc - 1) (1 - (r/rc)^2)^3 for r < rc (0 beyond); (len(r), n)."""
    r = np.asarray(r, dtype=np.float64)
    s = 2.0 * r / rc - 1.0
    fc = np.where(r < rc, (1.0 - (r / rc) ** 2) ** 3, 0.0)
    out = np.zeros((r.size, n_rad))
    for n in range(n_rad):
        e = np.zeros(n + 1)
        e[n] = 1.0
        out[:, n] = C.chebval(s, e) * fc
    return out


def uniform_bspline(coef: np.ndarray, h: float) -> BSpline:
    """Cubic spline sum_a c_a B_a with knots t_a = (a - 3) h."""
    nb = len(coef)
    t = (np.arange(nb + 4) - 3.0) * h
    return BSpline(t, np.asarray(coef, dtype=np.float64), 3, extrapolate=False)


def _nan0(v):
    v = np.asarray(v, dtype=np.float64)
    return np.where(np.isfinite(v), v, 0.0)


def pair_energy_ref(coef: np.ndarray, rc: float, r: np.ndarray) -> float:
    """1/2 sum_j V(r_j) over r_j < rc."""
    spl = uniform_bspline(coef, rc / 13.0)
    r = np.asarray(r)
    r = r[r < rc]
    return 0.5 * float(np.sum(_nan0(spl(r))))


def cheap_site_energy_ref(spline, rij: np.ndarray) -> float:
    """E_i = 1/2 sum_j V2(r_ij) + sum_{j<k, r_ij, r_ik < rc3} V3(r_ij, r_ik, r_jk),
    V3 a tensor product of scipy B-splines."""
    rij = np.asarray(rij).reshape(-1, 3)
    r = np.linalg.norm(rij, axis=1)
    E = pair_energy_ref(spline.c2, spline.r_cut, r)
    h3 = spline.r_cut3 / 5.0
    hc = 2.0 * spline.r_cut3 / 5.0
    ta = (np.arange(12) - 3.0) * h3
    tc = (np.arange(12) - 3.0) * hc

    def basis(t, x):
        out = np.zeros(8)
        for a in range(8):
            e = np.zeros(8)
            e[a] = 1.0
            out[a] = float(_nan0(BSpline(t, e, 3, extrapolate=False)(x)))
        return out

    idx = np.where(r < spline.r_cut3)[0]
    for p in range(len(idx)):
        for q in range(p + 1, len(idx)):
            j, k = idx[p], idx[q]
            r3 = np.linalg.norm(rij[k] - rij[j])
            E += float(np.einsum("abc,a,b,c->", spline.c3, basis(ta, r[j]), basis(ta, r[k]),
                                 basis(tc, r3)))
    return E


def ace_labels(n_rad: int, l_max: int, nu_max: int):
    """Canonical basis enumeration: nu=1 (n); nu=2 (l, n1<=n2); nu=3 labels
    sorted by (l, n) with l1+l2+l3 even and l3 <= l1+l2."""
    labels = [((n, 0),) for n in range(n_rad)]
    if nu_max >= 2:
        for l in range(l_max + 1):
            for n1 in range(n_rad):
                for n2 in range(n1, n_rad):
                    labels.append(((n1, l), (n2, l)))
    if nu_max >= 3:
        for l1 in range(l_max + 1):
            for l2 in range(l1, l_max + 1):
                for l3 in range(l2, l_max + 1):
                    if (l1 + l2 + l3) % 2 or l3 > l1 + l2:
                        continue
                    for n1 in range(n_rad):
                        for n2 in range(n1 if l2 == l1 else 0, n_rad):
                            for n3 in range(n2 if l3 == l2 else 0, n_rad):
                                labels.append(((n1, l1), (n2, l2), (n3, l3)))
    return labels


def ace_basis_ref(ace, rij: np.ndarray) -> np.ndarray:
    """Basis values through the addition theorem and sphere quadrature:
    rho_nl(u) = sum_j R_n(r_j) (2l+1)/(4pi) P_l(u . u_j) is the degree-l part of
    the density; nu=1: A_n00 = sum_j R_n / sqrt(4pi); nu=2 and nu=3: the sphere
    integral of the product of the rho's (exact by quadrature of degree 3L)."""
    rij = np.asarray(rij).reshape(-1, 3)
    r = np.linalg.norm(rij, axis=1)
    keep = r < ace.r_cut
    rij, r = rij[keep], r[keep]
    u = rij / r[:, None]
    R = radial_ref(ace.n_rad, ace.r_cut, r)                  # (J, n)
    pts, wts = sphere_quadrature(3 * ace.l_max)
    cosg = pts @ u.T                                          # (K, J)
    rho = np.zeros((ace.l_max + 1, ace.n_rad, pts.shape[0]))
    for l in range(ace.l_max + 1):
        Pl = sp.eval_legendre(l, np.clip(cosg, -1.0, 1.0))   # (K, J)
        rho[l] = (2 * l + 1) / (4 * np.pi) * (R.T @ Pl.T)   # (n, K)
    out = []
    for lab in ace_labels(ace.n_rad, ace.l_max, ace.nu_max):
        if len(lab) == 1:
            out.append(R[:, lab[0][0]].sum() / math.sqrt(4 * np.pi))
        else:
            prod = np.ones(pts.shape[0])
            for (n, l) in lab:
                prod = prod * rho[l, n]
            out.append(float(np.dot(wts, prod)))
    return np.array(out)


def ace_coeffs_ref(ace) -> np.ndarray:
    """Coefficient of each canonical basis function, read from the dense tables."""
    cs = []
    for lab in ace_labels(ace.n_rad, ace.l_max, ace.nu_max):
        if len(lab) == 1:
            cs.append(ace.c1[lab[0][0]])
        elif len(lab) == 2:
            (n1, l), (n2, _) = lab
            cs.append(ace.c2[l, n1, n2])
        else:
            (n1, l1), (n2, l2), (n3, l3) = lab
            cs.append(ace.c3[l1, l2, l3, n1, n2, n3])
    return np.array(cs)


def ace_site_energy_ref(ace, rij: np.ndarray) -> float:
    r = np.linalg.norm(np.asarray(rij).reshape(-1, 3), axis=1)
    return pair_energy_ref(ace.pair, ace.r_cut, r) + float(np.dot(ace_coeffs_ref(ace), ace_basis_ref(ace, rij)))


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, rr = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(rr))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q
