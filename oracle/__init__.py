"""Plain FP64 CPU oracle for the spatially mixed MD step (arXiv 2502.19081).

TEST INFRASTRUCTURE ONLY.  The tests, the package's smoke check and the
benchmark's CPU-baseline leg may call it; the product path never does, and it
shares no code with the CUDA library (it reads the seeded workload objects by
attribute and imports nothing from the package).

The C source (oracle.c) follows the paper's steps: region weights (Sec. 4.4,
Alg. 2 in its geometric reading), evaluated sets with one-cutoff buffers
(Sec. 4.5 buffer-set equation, Alg. 3), forces as sums of site-energy
derivatives (Sec. 4.5 force equation) per potential on its evaluated set,
scaled by the blend weight and summed (Alg. 4), and velocity-Verlet steps.

The two potentials are synthetic, since the paper fixes neither:

* expensive, a linear atomic cluster expansion:
  R_n(r) = T_n(2r/rc - 1) (1 - (r/rc)^2)^3 (Chebyshev T_n), real orthonormal
  Y_lm without Condon-Shortley phase, A_nlm(i) = sum_j R_n(r_ij) Y_lm(r_ij/r_ij),
  basis nu=1: A_n00; nu=2: sum_m A_n1lm A_n2lm (n1 <= n2);
  nu=3: sum_m G^{l1 l2 l3}_{m1 m2 m3} A A A over labels sorted by (l, n), with
  G the real Gaunt coefficient (integral of three real Y over the sphere);
  E_i = 1/2 sum_j Vpair(r_ij) + sum_k c_k B_k(i);
* cheap, a 2+3-body cubic B-spline: E_i = 1/2 sum_j V2(r_ij) +
  sum_{j<k; r_ij, r_ik < rc3} V3(r_ij, r_ik, r_jk).

Pins (tests/test_oracle_*.py) tie every function here to something other than
itself: scipy's spherical harmonics and B-splines, quadrature identities for
the basis, central finite differences for forces, brute-force enumeration for
lists and sets, closed forms for the weights, invariances, and the
dt^2 energy-error law of velocity Verlet.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_OK = 0
OR_EINVAL = -1
OR_ENOMEM = -2
OR_EOVERFLOW = -4

MODE_METHOD = 0
MODE_PLAIN = 1
MODE_PURE_EXP = 2
MODE_PURE_CHEAP = 3

KAPPA = 9.6485332e-3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.or_model_new.restype = P
            L.or_model_new.argtypes = [i64, dp, dp, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double,
                                       ctypes.c_double, dp, dp, ctypes.c_int, dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double]
            L.or_model_free.argtypes = [P]
            L.or_model_basis_count.argtypes = [P]
            L.or_cells.argtypes = [i64, dp, dp, dp, ip, ctypes.c_double, ip, ip]
            L.or_neighbours.argtypes = [i64, dp, dp, dp, ip, ctypes.c_double, ctypes.c_int, ip, ip]
            L.or_neighbours_brute.argtypes = [i64, dp, dp, dp, ip, ctypes.c_double, ctypes.c_int, ip, ip]
            L.or_wrap.argtypes = [i64, dp, dp, ip]
            L.or_ylm.restype = ctypes.c_double
            L.or_ylm.argtypes = [ctypes.c_int, ctypes.c_int, dp]
            L.or_gaunt_real.restype = ctypes.c_double
            L.or_gaunt_real.argtypes = [ctypes.c_int] * 6
            L.or_lambda.argtypes = [P, dp, dp, dp]
            L.or_sets.argtypes = [P, dp, ctypes.POINTER(ctypes.c_uint8)]
            L.or_forces.argtypes = [P, dp, ctypes.c_int, dp, dp, dp]
            L.or_forces_sampled.argtypes = [P, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp]
            L.or_site.restype = ctypes.c_double
            L.or_site.argtypes = [P, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.or_density.argtypes = [P, ctypes.c_int, dp, dp]
            L.or_md.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
            L.or_set_atomic.argtypes = [P, ctypes.POINTER(ctypes.c_uint8), ctypes.c_double, ctypes.c_double]
            L.or_coordination.argtypes = [P, dp, ctypes.c_double, ip]
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_get_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def ylm(l: int, m: int, u) -> float:
    """Real orthonormal Y_lm (no Condon-Shortley phase) at a unit vector."""
    uu = _c64(u)
    return float(lib().or_ylm(l, m, _d(uu)))


def gaunt(l1, m1, l2, m2, l3, m3) -> float:
    """Integral over the sphere of Y_l1m1 Y_l2m2 Y_l3m3 (real Y of this oracle),
    from the Racah formula for Wigner 3j symbols and the complex-to-real map."""
    return float(lib().or_gaunt_real(l1, m1, l2, m2, l3, m3))


def _pos(x) -> np.ndarray:
    x = _c64(x)
    if x.ndim != 2 or x.shape[1] != 4:
        raise ValueError("positions must be (N, 4) float64")
    return x


def cells(x, box_lo, box_len, periodic, rlist):
    x = _pos(x)
    n = x.shape[0]
    lo, L = _c64(box_lo), _c64(box_len)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    nc = np.zeros(3, dtype=np.int32)
    cid = np.zeros(max(n, 1), dtype=np.int32)
    st = lib().or_cells(n, _d(x), _d(lo), _d(L), _i(per), float(rlist), _i(nc), _i(cid))
    if st:
        raise ValueError(f"or_cells status {st}")
    return nc, cid[:n]


def neighbours(x, box_lo, box_len, periodic, rlist, cap=256, brute=False):
    """Full neighbour lists (sorted rows) at radius rlist; returns (nnb, nbr)."""
    x = _pos(x)
    n = x.shape[0]
    lo, L = _c64(box_lo), _c64(box_len)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    nnb = np.zeros(max(n, 1), dtype=np.int32)
    nbr = np.full((max(n, 1), cap), -1, dtype=np.int32)
    fn = lib().or_neighbours_brute if brute else lib().or_neighbours
    st = fn(n, _d(x), _d(lo), _d(L), _i(per), float(rlist), int(cap), _i(nnb), _i(nbr))
    if st == OR_EOVERFLOW:
        raise OverflowError("neighbour capacity exceeded")
    if st:
        raise ValueError(f"neighbour status {st}")
    if brute:
        for i in range(n):
            nbr[i, :nnb[i]] = np.sort(nbr[i, :nnb[i]])
    return nnb[:n], nbr[:n]


def wrap(x, box_len, periodic) -> np.ndarray:
    x = _pos(x).copy()
    L = _c64(box_len)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    lib().or_wrap(x.shape[0], _d(x), _d(L), _i(per))
    return x


class Model:
    """A system with both potentials and its regions, held by the C oracle."""

    def __init__(self, workload=None, *, system=None, ace=None, spline=None, regions=None,
                 blend: int = 0, buf_e: float = 0.0, buf_c: float = 0.0):
        if workload is not None:
            system = workload.system
            ace = workload.ace
            spline = workload.spline
            regions = workload.regions
        self.system, self.ace, self.spline, self.regions = system, ace, spline, regions
        self.n = int(system.x.shape[0])
        self._keep = []
        lo, L = _c64(system.box_lo), _c64(system.box_len)
        per = np.ascontiguousarray(system.periodic, dtype=np.int32)
        c1, c2, c3, pair = _c64(ace.c1), _c64(ace.c2), _c64(ace.c3), _c64(ace.pair)
        s2, s3 = _c64(spline.c2), _c64(spline.c3)
        regs = np.zeros((max(len(regions), 1), 9))
        for k, r in enumerate(regions):
            regs[k] = [r.kind, *r.centre, *r.axis, r.r_core, r.ramp]
        self._keep += [lo, L, per, c1, c2, c3, pair, s2, s3, regs]
        self._h = lib().or_model_new(self.n, _d(lo), _d(L), _i(per), float(system.mass),
                                     float(ace.r_cut), int(ace.n_rad), int(ace.l_max), int(ace.nu_max),
                                     _d(c1), _d(c2), _d(c3), _d(pair), float(spline.r_cut),
                                     float(spline.r_cut3), _d(s2), _d(s3), len(regions), _d(regs),
                                     int(blend), float(buf_e), float(buf_c))
        if not self._h:
            raise ValueError("oracle model rejected its parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_model_free(h)
            self._h = None

    def set_atomic(self, seeds=None, r_core: float = 0.0, r_blend: float = 0.0):
        """Weights from seed atoms (Alg. 1-2); seeds: indices or a [N] mask, None
        returns to the geometric regions."""
        if seeds is None:
            lib().or_set_atomic(self._h, None, 0.0, 0.0)
            return
        mask = np.zeros(max(self.n, 1), dtype=np.uint8)
        s = np.asarray(seeds)
        if s.dtype == bool or (s.size == self.n and set(np.unique(s)) <= {0, 1} and s.dtype != np.int64):
            mask[:self.n] = s.astype(np.uint8)
        else:
            mask[s.astype(np.int64)] = 1
        self._keep.append(mask)
        st = lib().or_set_atomic(self._h, mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), float(r_core),
                                 float(r_blend))
        if st:
            raise ValueError(f"or_set_atomic status {st}")

    def coordination(self, x, r: float) -> np.ndarray:
        """Number of neighbours closer than r of every atom."""
        x = _pos(x)
        z = np.zeros(max(self.n, 1), dtype=np.int32)
        st = lib().or_coordination(self._h, _d(x), float(r), _i(z))
        if st:
            raise ValueError(f"or_coordination status {st}")
        return z[:self.n]

    def basis_count(self) -> int:
        return int(lib().or_model_basis_count(self._h))

    def lam(self, x):
        x = _pos(x)
        lam = np.zeros(self.n)
        w = np.zeros(self.n)
        lib().or_lambda(self._h, _d(x), _d(lam), _d(w))
        return lam, w

    def sets(self, x) -> np.ndarray:
        x = _pos(x)
        f = np.zeros(max(self.n, 1), dtype=np.uint8)
        st = lib().or_sets(self._h, _d(x), f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        if st:
            raise ValueError(f"or_sets status {st}")
        return f[:self.n]

    def forces(self, x, mode: int = MODE_METHOD):
        """Returns (F (N,4), Ee (N,), Ec (N,))."""
        x = _pos(x)
        F = np.zeros((max(self.n, 1), 4))
        Ee = np.zeros(max(self.n, 1))
        Ec = np.zeros(max(self.n, 1))
        st = lib().or_forces(self._h, _d(x), int(mode), _d(F), _d(Ee), _d(Ec))
        if st:
            raise ValueError(f"or_forces status {st}")
        return F[:self.n], Ee[:self.n], Ec[:self.n]

    def forces_sampled(self, x, idx):
        x = _pos(x)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        Fs = np.zeros((max(len(idx), 1), 4))
        st = lib().or_forces_sampled(self._h, _d(x), len(idx),
                                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _d(Fs))
        if st:
            raise ValueError(f"or_forces_sampled status {st}")
        return Fs[:len(idx)]

    def site(self, which: int, rij, want_basis: bool = False):
        """Site energy and pair gradients dE_i/dr_ij for one environment
        (rows of rij = x_j - x_i).  which 0 = expensive, 1 = cheap."""
        rij = _c64(rij).reshape(-1, 3)
        nn = rij.shape[0]
        g = np.zeros((max(nn, 1), 3))
        nb = self.basis_count() if (want_basis and which == 0) else 1
        basis = np.zeros(nb)
        E = lib().or_site(self._h, int(which), nn, _d(rij), _d(g),
                          _d(basis) if (want_basis and which == 0) else None)
        if want_basis:
            return E, g[:nn], basis
        return E, g[:nn]

    def density(self, rij):
        rij = _c64(rij).reshape(-1, 3)
        A = np.zeros((self.ace.n_rad, (self.ace.l_max + 1) ** 2))
        lib().or_density(self._h, rij.shape[0], _d(rij), _d(A))
        return A

    def md(self, x, v, F, dt: float, nsteps: int, mode: int = MODE_METHOD):
        """Velocity Verlet in place on copies; returns (x, v, F, epot[nsteps])."""
        x = _pos(x).copy()
        v = _pos(v).copy()
        F = _pos(F).copy()
        ep = np.zeros(max(nsteps, 1))
        st = lib().or_md(self._h, _d(x), _d(v), _d(F), float(dt), int(nsteps), int(mode), _d(ep))
        if st:
            raise ValueError(f"or_md status {st}")
        return x, v, F, ep[:nsteps]
