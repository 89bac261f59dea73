"""Seeded synthetic inputs for the spatially mixed MD step.

This module builds the workloads both sides consume: lattices with their
defects and thermal displacements, region shapes, and the coefficient tables of
the two synthetic potentials.  It holds none of the force-mixing arithmetic
(no distances, no basis functions, no energies or forces); a random coefficient
here is a raw normal draw times a label-dependent decay, and the pair shape is a
control polygon sampled from a closed-form target curve.

The paper (arXiv 2502.19081) fixes neither potential; it only names the
families (linear ACE, Sec. 2.1 and Table 1; UF3 2+3-body splines, Sec. 2.1).
The concrete forms these tables parameterise are:

* expensive ("ACE"): R_n(r) = T_n(2r/rc - 1) (1 - (r/rc)^2)^3, real orthonormal
  Y_lm, A_nlm = sum_j R_n Y_lm, product basis of correlation order nu <= 3 with
  real Gaunt coupling at nu = 3, linear readout, plus a cubic B-spline pair term
  (linear ACE fits carry a pair basis beside the many-body basis);
* cheap ("UF3-like"): cubic B-spline 2-body term on 16 uniform knots and
  3-body term on an 8x8x8 tensor-product basis.

Coefficient layouts (shared with the C interface):

* ace.c1[n]                         nu = 1 label (n, l=0)
* ace.c2[l, n1, n2]                 nu = 2, used for n1 <= n2
* ace.c3[l1, l2, l3, n1, n2, n3]    nu = 3, used for labels sorted by (l, n):
                                    l1 <= l2 <= l3, n1 <= n2 when l1 == l2,
                                    n2 <= n3 when l2 == l3, l1+l2+l3 even,
                                    l3 <= l1 + l2
* ace.pair[16], spline.c2[16]       B-spline pair coefficients, knots (a-3)h,
                                    h = rc/13; entries 13..15 are zero
* spline.c3[a, b, c]                symmetric in (a, b); zero for a >= 5 or b >= 5

Random draws use numpy's PCG64 generator with the seed recorded per workload.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

REGION_SPHERE = 0
REGION_CYLINDER = 1

PRECISION_FP64 = 0
PRECISION_FP32 = 1
PRECISION_BF16 = 2

MASS_SI = 28.0855
MASS_FE = 55.845

_SCALES_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scales.json")


@dataclass
class Region:
    """A core region: points closer than r_core get weight 1, a ramp of width
    `ramp` follows (Sec. 4.4, Alg. 2 in its geometric reading)."""
    kind: int
    centre: Tuple[float, float, float]
    axis: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    r_core: float = 0.0
    ramp: float = 0.0


@dataclass
class System:
    x: np.ndarray            # (N, 4) float64 positions in Angstrom; column 3 unused (0)
    v: np.ndarray            # (N, 4) float64 velocities in Angstrom/fs; column 3 unused
    mass: float              # amu, one species
    box_lo: np.ndarray       # (3,) float64; 0 in periodic dimensions
    box_len: np.ndarray      # (3,) float64
    periodic: Tuple[int, int, int]

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


@dataclass
class Ace:
    r_cut: float
    n_rad: int
    l_max: int
    nu_max: int
    c1: np.ndarray           # (n,)
    c2: np.ndarray           # (L+1, n, n)
    c3: np.ndarray           # (L+1, L+1, L+1, n, n, n)
    pair: np.ndarray         # (16,)


@dataclass
class Spline:
    r_cut: float
    r_cut3: float
    c2: np.ndarray           # (16,)
    c3: np.ndarray           # (8, 8, 8)


@dataclass
class Workload:
    name: str
    system: System
    regions: List[Region]
    ace: Ace
    spline: Spline
    skin: float = 0.3
    dt: float = 1.0
    steps: int = 100
    precision: int = PRECISION_FP64
    seed: int = 0
    description: str = ""
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# lattices


def diamond_lattice(nx: int, ny: int, nz: int) -> np.ndarray:
    """Integer coordinates (units of a/4) of a diamond supercell, z-major order."""
    fcc = np.array([[0, 0, 0], [0, 2, 2], [2, 0, 2], [2, 2, 0]])
    basis = np.concatenate([fcc, fcc + 1])
    return (basis[None, :, :] + 4 * _cell_grid(nx, ny, nz)[:, None, :]).reshape(-1, 3).astype(np.int64)


def _cell_grid(nx: int, ny: int, nz: int) -> np.ndarray:
    """Cell indices (ix, iy, iz), ix slowest and iz fastest."""
    g = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return np.stack(g, axis=-1).reshape(-1, 3)


def bcc_lattice(nx: int, ny: int, nz: int) -> np.ndarray:
    """Integer coordinates (units of a/2) of a bcc supercell."""
    basis = np.array([[0, 0, 0], [1, 1, 1]])
    return (basis[None, :, :] + 2 * _cell_grid(nx, ny, nz)[:, None, :]).reshape(-1, 3).astype(np.int64)


def _pack(pos3: np.ndarray) -> np.ndarray:
    x = np.zeros((pos3.shape[0], 4), dtype=np.float64)
    x[:, :3] = pos3
    return x


def wrap_into_box(pos3: np.ndarray, box_len, periodic) -> np.ndarray:
    """Fold coordinates of periodic dimensions into [0, L).  Input preparation
    only (the step itself folds positions when it rebuilds its lists)."""
    out = pos3.copy()
    for d in range(3):
        if periodic[d]:
            out[:, d] = np.mod(out[:, d], box_len[d])
            out[:, d] = np.where(out[:, d] >= box_len[d], 0.0, out[:, d])
    return out


def maxwell_boltzmann(rng: np.random.Generator, n: int, mass: float, temp_k: float) -> np.ndarray:
    """Velocities (Angstrom/fs) at temperature T: zero total momentum, rescaled to
    exactly T with 3N-3 degrees of freedom."""
    kb = 8.617333262e-5            # eV/K
    kappa = 9.6485332e-3           # (eV/Angstrom/amu) -> Angstrom/fs^2
    if n < 2 or temp_k <= 0:
        return np.zeros((n, 4))
    sig = math.sqrt(kb * temp_k / mass * kappa)
    v = rng.standard_normal((n, 3)) * sig
    v -= v.mean(axis=0)
    ke = 0.5 * mass * np.sum(v * v) / kappa
    t_now = 2.0 * ke / (3.0 * (n - 1) * kb)
    v *= math.sqrt(temp_k / t_now)
    out = np.zeros((n, 4))
    out[:, :3] = v
    return out


# ----------------------------------------------------------------------------
# potentials


def _morse_target(r: np.ndarray, depth: float, alpha: float, r0: float, r_taper: float) -> np.ndarray:
    """Closed-form target pair shape: Morse well at r0, tapered to zero at r_taper."""
    rr = np.maximum(r, 0.0)
    e = np.exp(-alpha * (rr - r0))
    phi = depth * (e * e - 2.0 * e)
    t = np.clip(rr / r_taper, 0.0, 1.0)
    taper = (1.0 - t * t) ** 3
    return phi * taper


def pair_control_polygon(r_cut: float, depth: float, alpha: float, r0: float,
                         r_taper: Optional[float] = None) -> np.ndarray:
    """Sixteen B-spline coefficients sampled from the target shape at the knot
    averages (a-1)h of the uniform cubic basis, h = rc/13; the last three are zero
    so that the pair term and its first two derivatives vanish at rc.  The
    target is tapered to zero at r_taper (default 11 h)."""
    h = r_cut / 13.0
    grev = (np.arange(16) - 1.0) * h
    c = _morse_target(grev, depth, alpha, r0, 11.0 * h if r_taper is None else r_taper)
    c[13:] = 0.0
    return c


def ace_decay(n_rad: int, l_max: int):
    """Label decay factors (n + l + 1)^-2 for each (n, l)."""
    n = np.arange(n_rad)[:, None]
    l = np.arange(l_max + 1)[None, :]
    return (n + l + 1.0) ** -2.0           # (n, L+1)


def make_ace(rng: np.random.Generator, r_cut: float, n_rad: int, l_max: int, body_order: int,
             scale: float, pair: np.ndarray) -> Ace:
    """Random linear-ACE coefficients: c = scale * xi * prod_t (n_t + l_t + 1)^-2,
    xi ~ N(0, 1), drawn densely over every label (unused entries are ignored by
    the evaluators)."""
    nu_max = body_order - 1
    f = ace_decay(n_rad, l_max)            # f[n, l]
    L1 = l_max + 1
    c1 = scale * rng.standard_normal(n_rad) * f[:, 0]
    xi2 = rng.standard_normal((L1, n_rad, n_rad))
    c2 = scale * xi2 * np.einsum("al,bl->lab", f, f)
    if nu_max >= 3:
        xi3 = rng.standard_normal((L1, L1, L1, n_rad, n_rad, n_rad))
        dec = np.einsum("ai,bj,ck->ijkabc", f, f, f)
        c3 = scale * xi3 * dec
    else:
        c3 = np.zeros((L1, L1, L1, n_rad, n_rad, n_rad))
    if nu_max < 2:
        c2[:] = 0.0
    return Ace(r_cut=r_cut, n_rad=n_rad, l_max=l_max, nu_max=nu_max, c1=c1, c2=c2, c3=c3,
               pair=np.asarray(pair, dtype=np.float64).copy())


def make_spline(rng: np.random.Generator, r_cut: float, r_cut3: float, scale3: float,
                pair: np.ndarray) -> Spline:
    """Cheap 2+3-body spline: pair control polygon plus a small random part, and
    random 3-body coefficients symmetrised in their first two indices and zeroed
    where the first or second index is >= 5."""
    c2 = np.asarray(pair, dtype=np.float64).copy()
    c3 = rng.standard_normal((8, 8, 8))
    c3 = 0.5 * (c3 + c3.transpose(1, 0, 2))
    c3[5:, :, :] = 0.0
    c3[:, 5:, :] = 0.0
    return Spline(r_cut=r_cut, r_cut3=r_cut3, c2=c2, c3=scale3 * c3)


def load_scales() -> dict:
    if os.path.exists(_SCALES_FILE):
        with open(_SCALES_FILE) as fh:
            return json.load(fh)
    return {}


def _scale(key: str, default: float) -> float:
    return float(load_scales().get(key, {}).get("value", default))


# element pair targets (depth eV, alpha 1/Angstrom, r0 Angstrom = nearest-neighbour distance)
# 3-body cutoff of the cheap Si potential: between the first (2.35 A) and second
# (3.84 A) shells, so that the angular term's taper is gentle at the bond length
# (rc 3.5/6 = 2.9 A would put the bond on its steep end)
SI_RC3 = 3.4
# Si: a short-ranged well (tapered to zero at 3.4 A, between the first and second
# shells), so that with the angular term the diamond lattice is a minimum
PAIR_SI = dict(depth=1.5, alpha=2.0, r0=5.431 * math.sqrt(3.0) / 4.0, r_taper=3.4)
PAIR_FE = dict(depth=0.5, alpha=1.7, r0=2.855 * math.sqrt(3.0) / 2.0)


_SI_ANGULAR_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "si_angular.json")


def si_angular_tables(n_rad: int, l_max: int):
    """The stored angular term of the Si potentials (written by
    oracle/fit_si_angular.py): additions to the cheap 3-body coefficients
    [8][8][8], to the expensive nu = 2 coefficients [l_max+1][n][n] and to its
    pair spline [16].  Zero tables where the file or the shape is absent."""
    c3 = np.zeros((8, 8, 8))
    c2 = np.zeros((l_max + 1, n_rad, n_rad))
    pair = np.zeros(16)
    if os.path.exists(_SI_ANGULAR_FILE):
        with open(_SI_ANGULAR_FILE) as fh:
            tab = json.load(fh)
        c3 = np.asarray(tab["cheap_c3_add"], dtype=np.float64)
        ent = tab["ace"].get(f"n{n_rad}_l{l_max}")
        if ent is not None:
            c2 = np.asarray(ent["c2_add"], dtype=np.float64)
            pair = np.asarray(ent["pair_add"], dtype=np.float64)
    return c3, c2, pair


def element_potentials(element: str, rng: np.random.Generator, r_cut: float, n_rad: int, l_max: int,
                       body_order: int, scale_key: Optional[str] = None, angular: bool = True):
    """Expensive and cheap potentials for one element.  Both pair terms follow
    the same target shape with independent small perturbations, so the two
    potentials agree in the bulk the way a distilled cheap potential does.
    Si (angular=True) also carries the stored angular term of both potentials
    (si_angular_tables), without which the diamond lattice densifies."""
    tgt = PAIR_SI if element == "Si" else PAIR_FE
    base = pair_control_polygon(r_cut, **tgt)
    pert_e = 0.02 * rng.standard_normal(16)
    pert_c = 0.02 * rng.standard_normal(16)
    pe = base + pert_e
    pc = base + pert_c
    pe[13:] = 0.0
    pc[13:] = 0.0
    key = scale_key or f"{element}_n{n_rad}_l{l_max}_b{body_order}"
    s_e = _scale(f"ace:{key}", 1.0)
    r_cut3 = SI_RC3 if element == "Si" else r_cut * 3.5 / 6.0
    s_3 = _scale(f"spline3:{element}", 0.01)
    ace = make_ace(rng, r_cut, n_rad, l_max, body_order, s_e, pe)
    spl = make_spline(rng, r_cut, r_cut3, s_3, pc)
    if element == "Si" and angular:
        c3a, c2a, pa = si_angular_tables(n_rad, l_max)
        spl = Spline(r_cut=spl.r_cut, r_cut3=spl.r_cut3, c2=spl.c2, c3=spl.c3 + c3a)
        if ace.nu_max >= 2:
            ace = Ace(r_cut=ace.r_cut, n_rad=ace.n_rad, l_max=ace.l_max, nu_max=ace.nu_max, c1=ace.c1,
                      c2=ace.c2 + c2a, c3=ace.c3, pair=ace.pair + pa)
    return ace, spl


# ----------------------------------------------------------------------------
# the three single-system workloads


def si_vacancy(seed: int = 1, ncell: int = 3, sigma: float = 0.05) -> Workload:
    """Si diamond 3x3x3 conventional cells (a = 5.431 A) minus the atom nearest
    the box centre (ties broken by lowest index), periodic, Gaussian displacements
    sigma = 0.05 A; core sphere 6 A about the vacant site, ramp 2 A, rc = 5 A;
    expensive n = 8, lmax = 3, body order 3."""
    a = 5.431
    rng = np.random.default_rng(seed)
    q = diamond_lattice(ncell, ncell, ncell)
    ctr = np.array([2 * ncell] * 3)            # box centre in a/4 units
    d2 = np.sum((q - ctr) ** 2, axis=1)
    vac = int(np.argmin(d2))                   # argmin returns the lowest index on ties
    site = q[vac] * (a / 4.0)
    q = np.delete(q, vac, axis=0)
    pos = q * (a / 4.0) + rng.normal(0.0, sigma, (q.shape[0], 3))
    L = np.array([ncell * a] * 3)
    pos = wrap_into_box(pos, L, (1, 1, 1))
    sysm = System(x=_pack(pos), v=np.zeros((pos.shape[0], 4)), mass=MASS_SI,
                  box_lo=np.zeros(3), box_len=L, periodic=(1, 1, 1))
    ace, spl = element_potentials("Si", rng, 5.0, 8, 3, 3)
    reg = [Region(REGION_SPHERE, tuple(site), (0.0, 0.0, 1.0), 6.0, 2.0)]
    return Workload("si_vacancy_215", sysm, reg, ace, spl, skin=0.3, dt=1.0, steps=100,
                    precision=PRECISION_FP64, seed=seed,
                    description="Si diamond 3x3x3 minus one vacancy (215 atoms), FP64")


def fe_dumbbell(seed: int = 2, nx: int = 20, ny: int = 20, nz: int = 10, sigma: float = 0.08,
                sep: float = 1.0) -> Workload:
    """bcc Fe 20x20x10 (a = 2.855 A, 8000 sites): the site at the box centre is
    replaced by a <110> dumbbell, two atoms at site +- sep (1,1,0)/sqrt2 with
    sep = 1.0 A; thermal sigma = 0.08 A; core sphere 8 A about the site, ramp
    3 A, rc = 5.5 A; expensive n = 10, lmax = 4, body order 4."""
    a = 2.855
    rng = np.random.default_rng(seed)
    q = bcc_lattice(nx, ny, nz)
    ctr = np.array([nx, ny, nz])               # box centre in a/2 units
    d2 = np.sum((q - ctr) ** 2, axis=1)
    c = int(np.argmin(d2))
    site = q[c] * (a / 2.0)
    q = np.delete(q, c, axis=0)
    pos = q * (a / 2.0)
    u = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    dumb = np.stack([site + sep * u, site - sep * u])
    pos = np.concatenate([pos, dumb])
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    L = np.array([nx * a, ny * a, nz * a])
    pos = wrap_into_box(pos, L, (1, 1, 1))
    sysm = System(x=_pack(pos), v=np.zeros((pos.shape[0], 4)), mass=MASS_FE,
                  box_lo=np.zeros(3), box_len=L, periodic=(1, 1, 1))
    ace, spl = element_potentials("Fe", rng, 5.5, 10, 4, 4)
    reg = [Region(REGION_SPHERE, tuple(site), (0.0, 0.0, 1.0), 8.0, 3.0)]
    return Workload("fe_dumbbell_8001", sysm, reg, ace, spl, skin=0.3, dt=1.0, steps=1000,
                    precision=PRECISION_FP64, seed=seed,
                    description="bcc Fe 20x20x10 + <110> dumbbell (8001 atoms)")


def fe_screw(seed: int = 3, n_atoms: int = 256000, nrep_z: int = 26, sigma: float = 0.08,
             pad: float = 12.0) -> Workload:
    """bcc Fe cylinder about a 1/2<111> screw dislocation: z || [111],
    x || [1-10], y || [11-2]; Lz = 26 a sqrt3 (periodic), free in x and y; the
    n_atoms sites nearest the line (ties by index) are kept; the line passes
    through the centroid of three neighbouring [111] columns; u_z = b atan2/2pi,
    b = 2.47 A.  Core cylinder 15 A, ramp 4 A, rc = 5.5 A; expensive n = 12,
    lmax = 5, body order 4."""
    a = 2.855
    b = 2.47
    rng = np.random.default_rng(seed)
    ex = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    ey = np.array([1.0, 1.0, -2.0]) / math.sqrt(6.0)
    ez = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    rot = np.stack([ex, ey, ez])
    lz = nrep_z * a * math.sqrt(3.0)
    rho = 2.0 / a ** 3
    r_need = math.sqrt(n_atoms / (rho * lz * math.pi)) + 3.0
    reach = math.sqrt(2.0 * r_need ** 2 + lz ** 2) + 2 * a
    m = int(math.ceil(reach / a)) + 1
    ii = np.arange(-m, m + 1)
    g = np.stack(np.meshgrid(ii, ii, ii, indexing="ij"), axis=-1).reshape(-1, 3)
    pts = np.concatenate([g, g + 0.5]) * a
    pr = pts @ rot.T
    eps = 1e-6
    keep = (pr[:, 2] >= -eps) & (pr[:, 2] < lz - eps)
    pr = pr[keep]
    pr[:, 2] = np.maximum(pr[:, 2], 0.0)
    x0 = a / (3.0 * math.sqrt(2.0))
    y0 = a / math.sqrt(6.0)
    dxy = np.hypot(pr[:, 0] - x0, pr[:, 1] - y0)
    near = dxy < r_need
    pr = pr[near]
    dxy = dxy[near]
    order = np.lexsort((np.arange(pr.shape[0]), np.round(dxy, 9)))
    pr = pr[order[:n_atoms]]
    # sites on the cut (dy = 0 up to rounding, dx < 0) all take the +pi branch:
    # the sign of the rounding noise must not pick the branch, or two sites of
    # one column are displaced towards each other
    dyc = pr[:, 1] - y0
    dyc = np.where(np.abs(dyc) < 1e-9, 0.0, dyc)
    theta = np.arctan2(dyc, pr[:, 0] - x0)
    pr[:, 2] = pr[:, 2] + b * theta / (2.0 * math.pi)
    pr = pr + rng.normal(0.0, sigma, pr.shape)
    rmax = float(np.max(np.hypot(pr[:, 0] - x0, pr[:, 1] - y0)))
    half = rmax + pad
    lo = np.array([x0 - half, y0 - half, 0.0])
    L = np.array([2 * half, 2 * half, lz])
    pr = wrap_into_box(pr, L, (0, 0, 1))
    sysm = System(x=_pack(pr), v=np.zeros((pr.shape[0], 4)), mass=MASS_FE,
                  box_lo=lo, box_len=L, periodic=(0, 0, 1))
    ace, spl = element_potentials("Fe", rng, 5.5, 12, 5, 4)
    reg = [Region(REGION_CYLINDER, (x0, y0, 0.0), (0.0, 0.0, 1.0), 15.0, 4.0)]
    return Workload("fe_screw_256000", sysm, reg, ace, spl, skin=0.3, dt=1.0, steps=500,
                    precision=PRECISION_BF16, seed=seed,
                    description="bcc Fe screw-dislocation cylinder (256000 atoms)")


def si_replica(seed: int, n_target: int, defect: str, temp_k: float, ace: Ace = None,
               spline: Spline = None) -> Workload:
    """One Si defect cell of a batch: the diamond k1 x k2 x k3 box (k >= 3) whose
    atom count is nearest n_target, then a vacancy (atom nearest the centre
    removed) or a tetrahedral interstitial (atom added at the empty (1/2,1/2,1/2)a
    site nearest the centre); Maxwell-Boltzmann velocities at temp_k; core sphere
    6 A + ramp 2 A at the defect with the C1 potentials (shared when given)."""
    a = 5.431
    rng = np.random.default_rng(seed)
    k = max(3, int(round((n_target / 8.0) ** (1.0 / 3.0))))
    k3 = max(3, int(round(n_target / (8.0 * k * k))))
    q = diamond_lattice(k, k, k3)                          # a/4 units
    ctr = np.array([2 * k, 2 * k, 2 * k3])
    if defect == "vacancy":
        d2 = np.sum((q - ctr) ** 2, axis=1)
        idx = int(np.argmin(d2))
        site = q[idx] * (a / 4.0)
        q = np.delete(q, idx, axis=0)
        pos = q * (a / 4.0)
    else:
        # empty tetrahedral sites: (1/2,1/2,1/2)a + fcc translations, i.e. 2 + 4*cell + fcc offsets
        cell = np.array([k // 2, k // 2, k3 // 2])
        site = ((cell * 4 + np.array([2, 2, 2])) * (a / 4.0))
        pos = np.concatenate([q * (a / 4.0), site[None, :]])
    pos = pos + rng.normal(0.0, 0.05, pos.shape)
    L = np.array([k * a, k * a, k3 * a])
    pos = wrap_into_box(pos, L, (1, 1, 1))
    v = maxwell_boltzmann(rng, pos.shape[0], MASS_SI, temp_k)
    sysm = System(x=_pack(pos), v=v, mass=MASS_SI, box_lo=np.zeros(3), box_len=L, periodic=(1, 1, 1))
    if ace is None or spline is None:
        c1 = si_vacancy()
        ace, spline = c1.ace, c1.spline
    reg = [Region(REGION_SPHERE, tuple(site), (0.0, 0.0, 1.0), 6.0, 2.0)]
    return Workload(f"si_replica_{seed}", sysm, reg, ace, spline, skin=0.3, dt=1.0, steps=200,
                    precision=PRECISION_FP32, seed=seed, extra={"defect": defect, "temp_k": temp_k})


def si_replicas(n_replicas: int = 256, seed: int = 4, n_min: int = 1000, n_max: int = 20000):
    """The batch of independent Si defect cells: sizes log-uniform on
    [n_min, n_max], vacancy or interstitial with equal probability,
    temperatures uniform on [300, 1500] K; the Si vacancy cell's potentials."""
    rng = np.random.default_rng(seed)
    c1 = si_vacancy()                       # the Si vacancy cell's potentials
    ace, spl = c1.ace, c1.spline
    out = []
    for r in range(n_replicas):
        n_t = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        defect = "vacancy" if rng.uniform() < 0.5 else "interstitial"
        temp = float(rng.uniform(300.0, 1500.0))
        out.append(si_replica(seed * 100000 + r, n_t, defect, temp, ace, spl))
    return out


def serve_potentials():
    """The two potential pairs of the request stream: those of the silicon
    vacancy cell (rc 5 A, n 8, lmax 3, body order 3) and of the Fe dumbbell cell
    (rc 5.5 A, n 10, lmax 4, body order 4) themselves.  (Each random draw of
    the many-body terms is a different potential; another draw of the Fe
    recipe collapses the bcc lattice within 200 steps.)"""
    si, fe = si_vacancy(), fe_dumbbell()
    return {"Si": (si.ace, si.spline), "Fe": (fe.ace, fe.spline)}


def serve_request(seed: int, element: str, n_target: int, core_frac: float, temp_k: float, pots) -> Workload:
    """One request: the periodic diamond (Si, 8 atoms per cell) or bcc (Fe, 2
    per cell) box of k x k x k3 cells (k >= 3) whose atom count is nearest
    n_target, minus the site nearest the centre (a vacancy), thermal sigma
    0.05 A, Maxwell-Boltzmann velocities at temp_k; a core sphere at the
    vacancy holding the fraction core_frac of the atoms,
    r_core = (3 f N / (4 pi rho))^(1/3), ramp 2 A (Si) or 3 A (Fe)."""
    rng = np.random.default_rng(seed)
    if element == "Si":
        a, per_cell, unit, mass, ramp = 5.431, 8, 4.0, MASS_SI, 2.0
    else:
        a, per_cell, unit, mass, ramp = 2.855, 2, 2.0, MASS_FE, 3.0
    k = max(3, int(round((n_target / per_cell) ** (1.0 / 3.0))))
    k3 = max(3, int(round(n_target / (per_cell * k * k))))
    q = diamond_lattice(k, k, k3) if element == "Si" else bcc_lattice(k, k, k3)
    ctr = np.array([k, k, k3]) * (unit / 2.0)
    idx = int(np.argmin(np.sum((q - ctr) ** 2, axis=1)))
    site = q[idx] * (a / unit)
    pos = np.delete(q, idx, axis=0) * (a / unit)
    pos = pos + rng.normal(0.0, 0.05, pos.shape)
    L = np.array([k * a, k * a, k3 * a])
    pos = wrap_into_box(pos, L, (1, 1, 1))
    n = pos.shape[0]
    rho = n / float(np.prod(L))
    r_core = (3.0 * core_frac * n / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    sysm = System(x=_pack(pos), v=maxwell_boltzmann(rng, n, mass, temp_k), mass=mass, box_lo=np.zeros(3),
                  box_len=L, periodic=(1, 1, 1))
    ace, spl = pots[element]
    reg = [Region(REGION_SPHERE, tuple(site), (0.0, 0.0, 1.0), r_core, ramp)]
    return Workload(f"request_{element}_{n}_{seed}", sysm, reg, ace, spl, skin=0.3, dt=1.0, steps=0,
                    precision=PRECISION_FP32, seed=seed,
                    extra={"core_frac": core_frac, "temp_k": temp_k, "element": element})


def serve_stream(seed: int = 5, rate: float = 20.0, duration: float = 600.0, n_min: float = 1e3,
                 n_max: float = 5e5, len_min: float = 100.0, len_max: float = 2000.0):
    """Request specifications of a Poisson arrival process: exponential gaps of
    mean 1/rate seconds up to `duration`; Si or Fe with equal probability; atom
    counts and trajectory lengths log-uniform on [n_min, n_max] and
    [len_min, len_max]; core fraction uniform on [1 %, 10 %]; temperature
    uniform on [300, 1500] K.  Yields dicts (t, seed, element, n_target,
    core_frac, temp_k, nsteps); serve_request builds the system."""
    rng = np.random.default_rng(seed)
    t = 0.0
    k = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            return
        yield {"t": t, "seed": seed * 1000003 + k, "element": "Si" if rng.uniform() < 0.5 else "Fe",
               "n_target": int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))),
               "core_frac": float(rng.uniform(0.01, 0.10)), "temp_k": float(rng.uniform(300.0, 1500.0)),
               "nsteps": int(round(math.exp(rng.uniform(math.log(len_min), math.log(len_max)))))}
        k += 1


WORKLOADS = {
    "si_vacancy_215": si_vacancy,
    "fe_dumbbell_8001": fe_dumbbell,
    "fe_screw_256000": fe_screw,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)


# ----------------------------------------------------------------------------
# small systems for tests


def random_cluster(rng: np.random.Generator, n: int, radius: float, dmin: float = 1.8) -> np.ndarray:
    """n points in a ball of given radius with pairwise separation >= dmin
    (rejection sampling); returns (n, 3)."""
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("cluster packing failed")
        p = rng.uniform(-radius, radius, 3)
        if np.dot(p, p) > radius * radius:
            continue
        if pts and np.min(np.sum((np.array(pts) - p) ** 2, axis=1)) < dmin * dmin:
            continue
        pts.append(p)
    return np.array(pts)


def cluster_workload(seed: int, n: int = 24, radius: float = 5.0, element: str = "Fe",
                     r_cut: float = 5.5, n_rad: int = 6, l_max: int = 3, body_order: int = 4,
                     r_core: float = 3.0, ramp: float = 2.0, pad: float = 20.0) -> Workload:
    """A free cluster in a non-periodic box with small potentials, for checks
    that need arbitrary rotations or many evaluations."""
    rng = np.random.default_rng(seed)
    pos = random_cluster(rng, n, radius)
    lo = np.full(3, -radius - pad)
    L = np.full(3, 2 * (radius + pad))
    sysm = System(x=_pack(pos), v=np.zeros((n, 4)), mass=MASS_FE if element == "Fe" else MASS_SI,
                  box_lo=lo, box_len=L, periodic=(0, 0, 0))
    ace, spl = element_potentials(element, rng, r_cut, n_rad, l_max, body_order)
    reg = [Region(REGION_SPHERE, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), r_core, ramp)]
    return Workload(f"cluster_{n}_{seed}", sysm, reg, ace, spl, skin=0.3, seed=seed)


def small_fe_box(seed: int, nx: int = 7, ny: int = 7, nz: int = 7, sigma: float = 0.1,
                 n_rad: int = 6, l_max: int = 3, body_order: int = 4, r_core: float = 3.0,
                 ramp: float = 2.0, vacancy: bool = True) -> Workload:
    """A small periodic bcc Fe box (optionally with a vacancy), rc = 5.5 A."""
    a = 2.855
    rng = np.random.default_rng(seed)
    q = bcc_lattice(nx, ny, nz)
    site = np.array([nx, ny, nz]) * (a / 2.0)
    if vacancy:
        d2 = np.sum((q - np.array([nx, ny, nz])) ** 2, axis=1)
        q = np.delete(q, int(np.argmin(d2)), axis=0)
    pos = q * (a / 2.0) + rng.normal(0.0, sigma, (q.shape[0], 3))
    L = np.array([nx * a, ny * a, nz * a])
    pos = wrap_into_box(pos, L, (1, 1, 1))
    sysm = System(x=_pack(pos), v=np.zeros((pos.shape[0], 4)), mass=MASS_FE,
                  box_lo=np.zeros(3), box_len=L, periodic=(1, 1, 1))
    ace, spl = element_potentials("Fe", rng, 5.5, n_rad, l_max, body_order)
    reg = [Region(REGION_SPHERE, tuple(site), (0.0, 0.0, 1.0), r_core, ramp)]
    return Workload(f"fe_box_{nx}{ny}{nz}_{seed}", sysm, reg, ace, spl, skin=0.3, seed=seed)
