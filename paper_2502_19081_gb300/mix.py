"""Python binding of the C ABI in include/mix.h (ctypes; marshalling only).

Every step of the mixed MD path runs in the CUDA library libmix.so built from
csrc/; this module only converts arguments, owns the torch device buffers the
library borrows (positions, velocities, forces, workspace) and turns status
codes into exceptions.  There is no CPU fallback: if the library is missing
or no CUDA device is present, constructing a Context raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmix.so")

MIX_OK = 0
MIX_EINVAL = -1
MIX_ENOMEM = -2
MIX_ECUDA = -3
MIX_EOVERFLOW = -4
MIX_ETIMEOUT = -5
MIX_ENUMERIC = -6
MIX_ESTATE = -7
MIX_EBOX = -8

MIX_FP64 = 0
MIX_FP32 = 1
MIX_BF16 = 2          # float path, nu = 3 readout on the tensor cores (bf16 operands, float accumulation)
MIX_BF16_SPLIT = 3    # the same with hi/lo bf16 operand splits (three MMAs per product)
PREC_NAMES = {MIX_FP64: "f64", MIX_FP32: "f32", MIX_BF16: "bf16", MIX_BF16_SPLIT: "bf16x3"}
MIX_BLEND_LINEAR = 0
MIX_BLEND_CUBIC = 1
MIX_ORDER_CHEAP_FIRST = 0   # the two potential kernels on two branches, the cheap one launched first
MIX_ORDER_EXP_FIRST = 1     # two branches, the expensive one launched first
MIX_ORDER_SERIAL = 2        # one stream: the expensive kernel, then the cheap one

# functions declared in include/mix.h
EXPORTS = [
    "mix_init", "mix_workspace_bytes", "mix_bind", "mix_set_regions", "mix_forces", "mix_step",
    "mix_step_host", "mix_sync", "mix_get_stats", "mix_get_cells", "mix_get_neighbours",
    "mix_get_lambda", "mix_get_sets", "mix_get_site_energies", "mix_get_state", "mix_set_state",
    "mix_destroy", "mix_strerror", "mix_last_error", "mix_get_info", "mix_profile", "mix_get_profile",
    "mix_fma_peak", "mix_tune", "mix_batch_create", "mix_batch_step", "mix_batch_sync", "mix_batch_tune",
    "mix_batch_destroy", "mix_batch_last_error", "mix_set_seeds", "mix_set_seed_rule", "mix_get_seeds",
    "mix_server_create", "mix_server_submit", "mix_server_tick", "mix_server_request", "mix_server_fetch",
    "mix_server_destroy", "mix_server_last_error", "mix_admission_plan", "mix_batch_set_fused", "mix_batch_info",
    "mix_tc_selftest",
]

MIX_PHASES = 6
PHASE_NAMES = ["disp", "lists", "sets", "exp", "cheap", "gather"]


class MixError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class mix_system(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("box_lo", ctypes.c_double * 3), ("box_len", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("mass", ctypes.c_double)]


class mix_ace(ctypes.Structure):
    _fields_ = [("r_cut", ctypes.c_double), ("n_rad", ctypes.c_int), ("l_max", ctypes.c_int),
                ("nu_max", ctypes.c_int), ("c1", ctypes.POINTER(ctypes.c_double)),
                ("c2", ctypes.POINTER(ctypes.c_double)), ("c3", ctypes.POINTER(ctypes.c_double)),
                ("pair", ctypes.POINTER(ctypes.c_double))]


class mix_spline(ctypes.Structure):
    _fields_ = [("r_cut", ctypes.c_double), ("r_cut3", ctypes.c_double),
                ("c2", ctypes.POINTER(ctypes.c_double)), ("c3", ctypes.POINTER(ctypes.c_double))]


class mix_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skin", ctypes.c_double), ("blend", ctypes.c_int),
                ("buffer_exp", ctypes.c_double), ("buffer_cheap", ctypes.c_double), ("nbr_cap", ctypes.c_int),
                ("no_graphs", ctypes.c_int), ("potential_order", ctypes.c_int)]


class mix_region(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("centre", ctypes.c_double * 3), ("axis", ctypes.c_double * 3),
                ("r_core", ctypes.c_double), ("ramp", ctypes.c_double)]


class mix_stats(ctypes.Structure):
    _fields_ = [("n_core", ctypes.c_int64), ("n_ramp", ctypes.c_int64), ("n_exp", ctypes.c_int64),
                ("n_cheap", ctypes.c_int64), ("rebuilds", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("max_neighbours", ctypes.c_int), ("status_bits", ctypes.c_int)]


class mix_info(ctypes.Structure):
    _fields_ = [("nbr_cap", ctypes.c_int), ("n_tau", ctypes.c_int), ("gaunt_nnz", ctypes.c_int64),
                ("tau_dim3_sum", ctypes.c_int64), ("basis_size", ctypes.c_int64),
                ("nu3_flops_per_atom", ctypes.c_double),
                ("workspace_bytes", ctypes.c_size_t), ("exp_smem_bytes", ctypes.c_size_t),
                ("exp_grid", ctypes.c_int), ("exp_threads", ctypes.c_int), ("cheap_smem_bytes", ctypes.c_size_t),
                ("cheap_grid", ctypes.c_int), ("launches_per_evaluation", ctypes.c_int),
                ("launches", ctypes.c_int64), ("gather_grid", ctypes.c_int), ("build_grid", ctypes.c_int),
                ("buffer_grid", ctypes.c_int), ("exp_tensor_cores", ctypes.c_int),
                ("tc_flops_per_atom", ctypes.c_double), ("cheap_lanes", ctypes.c_int),
                ("nu3_flops_ref_per_atom", ctypes.c_double), ("potential_order", ctypes.c_int)]


class mix_server_options(ctypes.Structure):
    _fields_ = [("dt_fs", ctypes.c_double), ("hbm_budget", ctypes.c_size_t), ("hbm_reserve", ctypes.c_size_t),
                ("max_active_atoms", ctypes.c_int64), ("max_active", ctypes.c_int), ("fifo", ctypes.c_int)]


class mix_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("n_atoms", ctypes.c_int64),
                ("steps_done", ctypes.c_int64), ("steps_total", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class mix_tick_info(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int), ("retired", ctypes.c_int), ("failed", ctypes.c_int),
                ("active", ctypes.c_int), ("queued", ctypes.c_int), ("active_atoms", ctypes.c_int64),
                ("steps", ctypes.c_int), ("bytes_in_use", ctypes.c_size_t), ("step_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("rebuild_ms", ctypes.c_double), ("t", ctypes.c_double)]


MIX_REQ_QUEUED, MIX_REQ_ACTIVE, MIX_REQ_DONE, MIX_REQ_FAILED = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def lib():
    """Load libmix.so (built by build() / __graft_entry__.build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run python -m paper_2502_19081_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i64p = ctypes.POINTER(ctypes.c_int64)
            L.mix_init.argtypes = [ctypes.POINTER(mix_system), ctypes.POINTER(mix_ace), ctypes.POINTER(mix_spline),
                                   ctypes.POINTER(mix_options), P, ctypes.POINTER(P)]
            L.mix_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
            L.mix_bind.argtypes = [P, P, P, P, P]
            L.mix_set_regions.argtypes = [P, ctypes.POINTER(mix_region), ctypes.c_int]
            L.mix_set_seeds.argtypes = [P, ip, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.mix_set_seed_rule.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double]
            L.mix_get_seeds.argtypes = [P, ctypes.POINTER(ctypes.c_uint8), i64p]
            L.mix_forces.argtypes = [P]
            L.mix_server_create.argtypes = [ctypes.POINTER(mix_server_options), P, ctypes.POINTER(P)]
            L.mix_server_submit.argtypes = [P, ctypes.POINTER(mix_system), ctypes.POINTER(mix_ace),
                                            ctypes.POINTER(mix_spline), ctypes.POINTER(mix_options),
                                            ctypes.POINTER(mix_region), ctypes.c_int, dp, dp, ctypes.c_int64, i64p]
            L.mix_server_tick.argtypes = [P, ctypes.c_int, ctypes.POINTER(mix_tick_info)]
            L.mix_server_request.argtypes = [P, ctypes.c_int64, ctypes.POINTER(mix_request_info)]
            L.mix_server_fetch.argtypes = [P, ctypes.c_int64, dp, dp, dp]
            L.mix_server_destroy.argtypes = [P]
            L.mix_server_last_error.restype = ctypes.c_char_p
            L.mix_server_last_error.argtypes = [P]
            L.mix_admission_plan.argtypes = [ctypes.POINTER(ctypes.c_size_t), i64p, ctypes.c_int, ctypes.c_size_t,
                                             ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip]
            L.mix_step.argtypes = [P, ctypes.c_double, ctypes.c_int]
            L.mix_step_host.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_int]
            L.mix_sync.argtypes = [P]
            L.mix_get_stats.argtypes = [P, ctypes.POINTER(mix_stats)]
            L.mix_get_cells.argtypes = [P, ip, ip]
            L.mix_get_neighbours.argtypes = [P, ip, ip, ip, ip]
            L.mix_get_lambda.argtypes = [P, dp, dp]
            L.mix_get_sets.argtypes = [P, ctypes.POINTER(ctypes.c_uint8), ip, i64p, ip, i64p]
            L.mix_get_site_energies.argtypes = [P, dp, dp]
            L.mix_get_state.argtypes = [P, dp, dp, dp, i64p]
            L.mix_set_state.argtypes = [P, dp, dp, dp, ctypes.c_int64, ctypes.c_int]
            L.mix_destroy.argtypes = [P]
            L.mix_strerror.restype = ctypes.c_char_p
            L.mix_strerror.argtypes = [ctypes.c_int]
            L.mix_last_error.restype = ctypes.c_char_p
            L.mix_last_error.argtypes = [P]
            L.mix_get_info.argtypes = [P, ctypes.POINTER(mix_info)]
            L.mix_profile.argtypes = [P, ctypes.c_int]
            L.mix_get_profile.argtypes = [P, dp, dp, i64p]
            L.mix_fma_peak.argtypes = [ctypes.c_int, P, dp]
            L.mix_tc_selftest.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
            L.mix_neighbours_noalloc.argtypes = [ctypes.c_int64, P, dp, dp, ip, ctypes.c_double, ctypes.c_int,
                                                 P, P, P, P]
            L.mix_tune.argtypes = [P, ctypes.c_int]
            L.mix_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.POINTER(P)]
            L.mix_batch_step.argtypes = [P, ctypes.c_double, ctypes.c_int]
            L.mix_batch_sync.argtypes = [P]
            L.mix_batch_tune.argtypes = [P, ctypes.c_int, ip]
            L.mix_batch_destroy.argtypes = [P]
            L.mix_batch_set_fused.argtypes = [P, ctypes.c_int]
            L.mix_batch_info.argtypes = [P, ip, ip, i64p]
            L.mix_batch_last_error.restype = ctypes.c_char_p
            L.mix_batch_last_error.argtypes = [P]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _init_structs(workload, precision, nbr_cap=0, blend=MIX_BLEND_LINEAR, buffer_exp=0.0, buffer_cheap=0.0,
                  skin=None, graphs=True, order=MIX_ORDER_CHEAP_FIRST):
    """mix_init arguments for a workload; the returned list keeps the arrays alive."""
    s = workload.system
    keep = []
    sysd = mix_system(int(s.n), (ctypes.c_double * 3)(*s.box_lo), (ctypes.c_double * 3)(*s.box_len),
                      (ctypes.c_int * 3)(*[int(p) for p in s.periodic]), float(s.mass))
    a = workload.ace
    c1, c2, c3, pair = _f64(a.c1), _f64(a.c2), _f64(a.c3), _f64(a.pair)
    sp = workload.spline
    s2, s3 = _f64(sp.c2), _f64(sp.c3)
    keep += [c1, c2, c3, pair, s2, s3]
    aced = mix_ace(float(a.r_cut), int(a.n_rad), int(a.l_max), int(a.nu_max), _dp(c1), _dp(c2), _dp(c3),
                   _dp(pair))
    spld = mix_spline(float(sp.r_cut), float(sp.r_cut3), _dp(s2), _dp(s3))
    opt = mix_options(int(precision), float(workload.skin if skin is None else skin), int(blend),
                      float(buffer_exp), float(buffer_cheap), int(nbr_cap), 0 if graphs else 1, int(order))
    return sysd, aced, spld, opt, keep


def _regions_array(regions):
    arr = (mix_region * max(len(regions), 1))()
    for k, r in enumerate(regions):
        arr[k] = mix_region(int(r.kind), (ctypes.c_double * 3)(*r.centre), (ctypes.c_double * 3)(*r.axis),
                            float(r.r_core), float(r.ramp))
    return arr


class Context:
    """One mixed-MD trajectory on one CUDA device, backed by libmix.so.

    Positions, velocities, forces ([N, 4] float64) and the workspace are torch
    tensors owned here and lent to the library."""

    def __init__(self, workload: "I.Workload", precision: int = MIX_FP64, device: str = "cuda:0",
                 nbr_cap: int = 0, blend: int = MIX_BLEND_LINEAR, buffer_exp: float = 0.0,
                 buffer_cheap: float = 0.0, skin: Optional[float] = None, regions: Optional[Sequence] = None,
                 stream=None, graphs: bool = True, order: int = MIX_ORDER_CHEAP_FIRST):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the mixed-MD path runs only on the GPU")
        self._torch = torch
        self.L = lib()
        self.device = torch.device(device)
        self.wl = workload
        s = workload.system
        self.n = int(s.n)
        self.precision = precision
        sysd, aced, spld, opt, self._keep = _init_structs(workload, precision, nbr_cap, blend, buffer_exp,
                                                          buffer_cheap, skin, graphs, order)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            st = self.L.mix_init(ctypes.byref(sysd), ctypes.byref(aced), ctypes.byref(spld), ctypes.byref(opt),
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
            if st != MIX_OK:
                raise MixError(st, "mix_init: " + self.L.mix_strerror(st).decode())
            self.h = h
            nb = ctypes.c_size_t()
            self._check(self.L.mix_workspace_bytes(self.h, ctypes.byref(nb)), "mix_workspace_bytes")
            self.ws_bytes = int(nb.value)
            self.x = torch.zeros((max(self.n, 1), 4), dtype=torch.float64, device=self.device)
            self.v = torch.zeros_like(self.x)
            self.f = torch.zeros_like(self.x)
            self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)
            if self.n:
                self.x[:self.n].copy_(torch.from_numpy(_f64(s.x)))
                self.v[:self.n].copy_(torch.from_numpy(_f64(s.v)))
            torch.cuda.synchronize(self.device)
            self._check(self.L.mix_bind(self.h, ctypes.c_void_p(self.x.data_ptr()), ctypes.c_void_p(self.v.data_ptr()),
                                        ctypes.c_void_p(self.f.data_ptr()), ctypes.c_void_p(self.ws.data_ptr())),
                        "mix_bind")
            self.set_regions(workload.regions if regions is None else regions)
        cap = ctypes.c_int()
        self.L.mix_get_neighbours(self.h, ctypes.byref(cap), None, None, None)
        self.cap = int(cap.value)

    # -- plumbing -----------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != MIX_OK:
            msg = self.L.mix_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise MixError(st, f"{what}: {self.L.mix_strerror(st).decode()}: {msg}")

    def close(self):
        h = getattr(self, "h", None)
        if h:
            self.L.mix_destroy(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls --------------------------------------------------------------
    def set_regions(self, regions):
        arr = _regions_array(regions)
        self._check(self.L.mix_set_regions(self.h, arr, len(regions)), "mix_set_regions")

    def set_seeds(self, seeds, r_core: float, r_blend: float):
        """Weights from explicit seed atoms (Alg. 1-2)."""
        idx = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32).reshape(-1))
        buf = idx if idx.size else np.zeros(1, dtype=np.int32)
        self._check(self.L.mix_set_seeds(self.h, _ip(buf), int(idx.size), float(r_core), float(r_blend)),
                    "mix_set_seeds")

    def set_seed_rule(self, r_coord: float, z_lo: float, z_hi: float, period: int, r_core: float,
                      r_blend: float):
        """Seeds from the (period-averaged) coordination number, then Alg. 1-2."""
        self._check(self.L.mix_set_seed_rule(self.h, float(r_coord), float(z_lo), float(z_hi), int(period),
                                             float(r_core), float(r_blend)), "mix_set_seed_rule")

    def seeds(self):
        m = np.zeros(max(self.n, 1), dtype=np.uint8)
        k = ctypes.c_int64()
        self._check(self.L.mix_get_seeds(self.h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(k)),
                    "mix_get_seeds")
        return m[:self.n], k.value

    def forces(self):
        self._check(self.L.mix_forces(self.h), "mix_forces")
        return self.f[:self.n]

    def step(self, dt: float, nsteps: int = 1):
        self._check(self.L.mix_step(self.h, float(dt), int(nsteps)), "mix_step")

    def step_host(self, x: np.ndarray, v: np.ndarray, f: Optional[np.ndarray], dt: float, nsteps: int = 1):
        """End-to-end call with host arrays ([N,4] float64, C-contiguous; updated in place)."""
        self._check(self.L.mix_step_host(self.h, _dp(x), _dp(v), _dp(f) if f is not None else None, float(dt),
                                         int(nsteps)), "mix_step_host")

    def sync(self):
        self._check(self.L.mix_sync(self.h), "mix_sync")

    def stats(self, check: bool = True) -> dict:
        s = mix_stats()
        st = self.L.mix_get_stats(self.h, ctypes.byref(s))
        if check:
            self._check(st, "mix_get_stats")
        return {k: getattr(s, k) for k, _ in mix_stats._fields_}

    def cells(self):
        nc = np.zeros(3, dtype=np.int32)
        cid = np.zeros(max(self.n, 1), dtype=np.int32)
        self._check(self.L.mix_get_cells(self.h, _ip(nc), _ip(cid)), "mix_get_cells")
        return nc, cid[:self.n]

    def neighbours(self):
        nnb = np.zeros(max(self.n, 1), dtype=np.int32)
        nbr = np.zeros((max(self.n, 1), self.cap), dtype=np.int32)
        rev = np.zeros((max(self.n, 1), self.cap), dtype=np.int32)
        cap = ctypes.c_int()
        self._check(self.L.mix_get_neighbours(self.h, ctypes.byref(cap), _ip(nnb), _ip(nbr), _ip(rev)),
                    "mix_get_neighbours")
        return nnb[:self.n], nbr[:self.n], rev[:self.n]

    def lam(self):
        lam = np.zeros(max(self.n, 1))
        w = np.zeros(max(self.n, 1))
        self._check(self.L.mix_get_lambda(self.h, _dp(lam), _dp(w)), "mix_get_lambda")
        return lam[:self.n], w[:self.n]

    def sets(self):
        fl = np.zeros(max(self.n, 1), dtype=np.uint8)
        ae = np.zeros(max(self.n, 1), dtype=np.int32)
        ac = np.zeros(max(self.n, 1), dtype=np.int32)
        ne = ctypes.c_int64()
        nc = ctypes.c_int64()
        self._check(self.L.mix_get_sets(self.h, fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _ip(ae),
                                        ctypes.byref(ne), _ip(ac), ctypes.byref(nc)), "mix_get_sets")
        return fl[:self.n], ae[:ne.value], ac[:nc.value]

    def site_energies(self):
        ee = np.zeros(max(self.n, 1))
        ec = np.zeros(max(self.n, 1))
        self._check(self.L.mix_get_site_energies(self.h, _dp(ee), _dp(ec)), "mix_get_site_energies")
        return ee[:self.n], ec[:self.n]

    def get_state(self):
        x = np.zeros((max(self.n, 1), 4))
        v = np.zeros_like(x)
        f = np.zeros_like(x)
        st = ctypes.c_int64()
        self._check(self.L.mix_get_state(self.h, _dp(x), _dp(v), _dp(f), ctypes.byref(st)), "mix_get_state")
        return x[:self.n], v[:self.n], f[:self.n], int(st.value)

    def tune(self, reps: int = 3):
        """Autotune the launch shapes on the current positions (state unchanged)."""
        self._check(self.L.mix_tune(self.h, int(reps)), "mix_tune")

    def info(self) -> dict:
        s = mix_info()
        self._check(self.L.mix_get_info(self.h, ctypes.byref(s)), "mix_get_info")
        return {k: getattr(s, k) for k, _ in mix_info._fields_}

    def profile(self, enable: bool = True):
        self._check(self.L.mix_profile(self.h, 1 if enable else 0), "mix_profile")

    def get_profile(self):
        """(total ms per phase, last-evaluation ms per phase, evaluations)."""
        tot = np.zeros(MIX_PHASES)
        last = np.zeros(MIX_PHASES)
        ev = ctypes.c_int64()
        self._check(self.L.mix_get_profile(self.h, _dp(tot), _dp(last), ctypes.byref(ev)), "mix_get_profile")
        return tot, last, int(ev.value)

    def set_state(self, x, v, f=None, step: int = 0):
        x = _f64(x)
        v = _f64(v)
        fa = _f64(f) if f is not None else None
        self._check(self.L.mix_set_state(self.h, _dp(x), _dp(v), _dp(fa) if fa is not None else None, int(step),
                                         1 if fa is not None else 0), "mix_set_state")


class Batch:
    """Independent trajectories advanced together: one CUDA graph launch per
    step, one child graph per member (mix_batch_*).  Members are Contexts
    created on the same stream; the batch keeps them alive."""

    def __init__(self, contexts: Sequence[Context]):
        if not contexts:
            raise ValueError("empty batch")
        self.L = lib()
        self.members = list(contexts)
        stream = self.members[0].stream
        arr = (ctypes.c_void_p * len(self.members))(*[c.h.value for c in self.members])
        h = ctypes.c_void_p()
        st = self.L.mix_batch_create(arr, len(self.members), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != MIX_OK:
            raise MixError(st, "mix_batch_create (members must be bound and share one stream)")
        self.h = h

    def _check(self, st: int, what: str):
        if st != MIX_OK:
            raise MixError(st, f"{what}: {self.L.mix_strerror(st).decode()}: "
                               f"{self.L.mix_batch_last_error(self.h).decode()}")

    def step(self, dt: float, nsteps: int = 1):
        self._check(self.L.mix_batch_step(self.h, float(dt), int(nsteps)), "mix_batch_step")

    def sync(self):
        self._check(self.L.mix_batch_sync(self.h), "mix_batch_sync")

    def tune(self, reps: int = 3) -> int:
        out = ctypes.c_int()
        self._check(self.L.mix_batch_tune(self.h, int(reps), ctypes.byref(out)), "mix_batch_tune")
        return int(out.value)

    def set_fused(self, on: bool = True):
        """Fused step (one launch per kernel for all members) when the members
        allow it (one precision, geometric regions); else one child graph per member."""
        self._check(self.L.mix_batch_set_fused(self.h, 1 if on else 0), "mix_batch_set_fused")

    def info(self) -> dict:
        fused = ctypes.c_int()
        groups = ctypes.c_int()
        launches = ctypes.c_int64()
        self._check(self.L.mix_batch_info(self.h, ctypes.byref(fused), ctypes.byref(groups), ctypes.byref(launches)),
                    "mix_batch_info")
        return {"fused": bool(fused.value), "groups": int(groups.value), "launches": int(launches.value)}

    def close(self):
        h = getattr(self, "h", None)
        if h:
            self.L.mix_batch_destroy(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fma_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput (flop/s) of the current device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double()
    st = lib().mix_fma_peak(int(precision), ctypes.c_void_p(s.cuda_stream), ctypes.byref(out))
    if st != MIX_OK:
        raise MixError(st, "mix_fma_peak")
    return float(out.value)


def tc_selftest(a, b, d, status, stream=None) -> None:
    """mix_tc_selftest on torch device tensors: a [m, k] (m = 128 or 64) and
    b [n, k] bfloat16, d [128, n] float32 (written: TMEM lane l of a @ b.T on
    the tensor cores in row l), status [1] int32 (bit 0 set if the wait for the
    MMAs gave up).  Asynchronous on `stream`."""
    import torch
    for t, dt, shp in ((a, torch.bfloat16, None), (b, torch.bfloat16, None), (d, torch.float32, None),
                       (status, torch.int32, (1,))):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError("tc_selftest: a, b bfloat16, d float32, status int32, contiguous CUDA tensors")
    n, k, m = int(b.shape[0]), int(b.shape[1]), int(a.shape[0])
    if a.dim() != 2 or int(a.shape[1]) != k or tuple(d.shape) != (128, n) or status.numel() < 1:
        raise ValueError("tc_selftest: shapes a [m, k], b [n, k], d [128, n]")
    s = stream if stream is not None else torch.cuda.current_stream(a.device)
    st = lib().mix_tc_selftest(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), m, n, k,
                               ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                               ctypes.c_void_p(s.cuda_stream))
    if st != MIX_OK:
        raise MixError(st, "mix_tc_selftest: " + lib().mix_strerror(st).decode())


def neighbours_noalloc(x, box_lo, box_len, periodic, r_list: float, cap: int, nnb, nbr, rev, stream=None) -> int:
    """mix_neighbours_noalloc on torch device tensors: x [N, 4] float64 (read),
    nnb [N], nbr [N, cap], rev [N, cap] int32 (written).  For callers that may
    not allocate device memory; returns the status code."""
    import torch
    n = int(x.shape[0])
    dev = x.device
    if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 4:
        raise ValueError("neighbours_noalloc: x must be a [N, 4] float64 tensor")
    for t, name in ((x, "x"), (nnb, "nnb"), (nbr, "nbr"), (rev, "rev")):
        if not t.is_cuda or t.device != dev or not t.is_contiguous():
            raise ValueError(f"neighbours_noalloc: {name} must be a contiguous tensor on {dev}")
    for t, need, name in ((nnb, n, "nnb"), (nbr, n * int(cap), "nbr"), (rev, n * int(cap), "rev")):
        if t.dtype != torch.int32 or t.numel() < need:
            raise ValueError(f"neighbours_noalloc: {name} must be int32 with at least {need} entries")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    lo = _f64(box_lo)
    ln = _f64(box_len)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    return int(lib().mix_neighbours_noalloc(n, ctypes.c_void_p(x.data_ptr()), _dp(lo), _dp(ln), _ip(per),
                                            float(r_list), int(cap), ctypes.c_void_p(nnb.data_ptr()),
                                            ctypes.c_void_p(nbr.data_ptr()), ctypes.c_void_p(rev.data_ptr()),
                                            ctypes.c_void_p(s.cuda_stream)))


def admission_plan(need, atoms, bytes_free: int, atoms_free: int = -1, active: int = 0, max_active: int = 0,
                   fifo: bool = True):
    """The server's admission rule alone (host only): admit flags per queued request."""
    L = lib()
    k = len(need)
    nd = (ctypes.c_size_t * max(k, 1))(*[int(v) for v in need])
    at = np.ascontiguousarray(np.asarray(atoms, dtype=np.int64).reshape(-1)) if k else np.zeros(1, np.int64)
    out = np.zeros(max(k, 1), dtype=np.int32)
    cnt = L.mix_admission_plan(nd, at.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), k, int(bytes_free),
                               int(atoms_free), int(active), int(max_active), 1 if fifo else 0, _ip(out))
    if cnt < 0:
        raise MixError(cnt, "mix_admission_plan")
    return out[:k].astype(bool)


class Server:
    """A request queue served by continuous batching on one device (libmix.so's
    mix_server_*): requests are admitted while their device memory fits the
    budget, stepped together, and retired with their final state on the host."""

    def __init__(self, dt: float, hbm_budget: int = 0, hbm_reserve: int = 0, max_active_atoms: int = 0,
                 max_active: int = 0, fifo: bool = True, device: str = "cuda:0", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the serving path runs only on the GPU")
        self.L = lib()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o = mix_server_options(float(dt), int(hbm_budget), int(hbm_reserve), int(max_active_atoms),
                               int(max_active), 1 if fifo else 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.L.mix_server_create(ctypes.byref(o), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != MIX_OK:
            raise MixError(st, "mix_server_create: " + self.L.mix_strerror(st).decode())
        self.h = h
        self.n = {}

    def _check(self, st: int, what: str):
        if st != MIX_OK:
            msg = self.L.mix_server_last_error(self.h).decode() if self.h else ""
            raise MixError(st, f"{what}: {self.L.mix_strerror(st).decode()}: {msg}")

    def submit(self, workload, nsteps: int, precision: int = MIX_FP32, nbr_cap: int = 0,
               blend: int = MIX_BLEND_LINEAR, skin: Optional[float] = None, regions=None) -> int:
        sysd, aced, spld, opt, keep = _init_structs(workload, precision, nbr_cap, blend, 0.0, 0.0, skin, True)
        regs = workload.regions if regions is None else regions
        arr = _regions_array(regs)
        s = workload.system
        x = np.ascontiguousarray(np.asarray(s.x, dtype=np.float64).reshape(-1, 4)) if s.n else np.zeros((1, 4))
        v = np.ascontiguousarray(np.asarray(s.v, dtype=np.float64).reshape(-1, 4)) if s.n else np.zeros((1, 4))
        rid = ctypes.c_int64()
        self._check(self.L.mix_server_submit(self.h, ctypes.byref(sysd), ctypes.byref(aced), ctypes.byref(spld),
                                             ctypes.byref(opt), arr, len(regs), _dp(x), _dp(v), int(nsteps),
                                             ctypes.byref(rid)), "mix_server_submit")
        self.n[int(rid.value)] = int(s.n)
        return int(rid.value)

    def tick(self, max_steps: int = 1) -> dict:
        t = mix_tick_info()
        self._check(self.L.mix_server_tick(self.h, int(max_steps), ctypes.byref(t)), "mix_server_tick")
        return {k: getattr(t, k) for k, _ in mix_tick_info._fields_}

    def request(self, rid: int) -> dict:
        r = mix_request_info()
        self._check(self.L.mix_server_request(self.h, int(rid), ctypes.byref(r)), "mix_server_request")
        return {k: getattr(r, k) for k, _ in mix_request_info._fields_}

    def fetch(self, rid: int):
        n = self.n.get(int(rid), 0)
        x = np.zeros((max(n, 1), 4))
        v = np.zeros_like(x)
        f = np.zeros_like(x)
        self._check(self.L.mix_server_fetch(self.h, int(rid), _dp(x), _dp(v), _dp(f)), "mix_server_fetch")
        self.n.pop(int(rid), None)
        return x[:n], v[:n], f[:n]

    def close(self):
        if getattr(self, "h", None):
            self.L.mix_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def open_context(workload, precision: int = MIX_FP64, retries: int = 2, **kw) -> Context:
    """Create a context and evaluate forces once; if the neighbour capacity
    overflows, recreate it with room for the observed maximum.  A three-body
    overflow of the cheap kernel's narrow lane groups (the neighbour rows fit)
    has already widened them inside the context: the evaluation is repeated on
    the same context."""
    cap = kw.pop("nbr_cap", 0)
    for _ in range(retries + 1):
        ctx = Context(workload, precision=precision, nbr_cap=cap, **kw)
        for _ in range(2):
            try:
                ctx.forces()
                ctx.sync()
                return ctx
            except MixError as e:
                if e.code != MIX_EOVERFLOW:
                    raise
                st = ctx.stats(check=False)
                if int(st["max_neighbours"]) <= ctx.cap:
                    continue
                break
        need = max(int(st["max_neighbours"]), ctx.cap + 1)
        ctx.close()
        cap = min(256, ((int(need * 1.25) + 31) // 32) * 32)
    raise MixError(MIX_EOVERFLOW, "neighbour capacity could not be sized")
