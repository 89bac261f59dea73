#!/usr/bin/env python
"""Throughput of the spatially mixed MD step (arXiv 2502.19081 force mixing)
on GB300, in atom-steps/s.

A step is one velocity-Verlet step of the whole hot path: skin test and (when
needed) cell/neighbour-list rebuild, blend weights, evaluated sets with their
buffers, expensive potential on its set, cheap potential on its set, atomics-free
gather + blend, second half-kick.  Default workload: the 256,000-atom bcc Fe
screw-dislocation cylinder (the largest single-GPU configuration), with the
8,001-atom Fe dumbbell reported beside it; seeded synthetic positions and
potentials.

Timing: W untimed warm-up steps, then K steps; before every timed step a 512 MB
buffer is written to flush L2 (129 MB), outside the timed interval; each step is
timed on the device with CUDA events the library records on its stream around
its kernel groups.  Multi-GPU (torchrun): independent replicas, one per rank,
no collective on the data path; value = atoms x steps x ranks / max rank time.

--impl reference times the FP64 CPU oracle (the program the GPU path is checked
against) on the host cores, on the same workload, for a bounded time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "mixed-MD atom-steps/s, FP64 plain vs FP32/BF16 at ≤1e-3 eV/Å; p50/p99 step ms"
UNIT = "atom-steps/s"
GATE = 1e-3


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="fe_screw_256000")
    p.add_argument("--precision", default="auto", choices=["auto", "fp32", "fp64", "bf16", "bf16x3"])
    p.add_argument("--secondary-steps", type=int, default=20)
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--ncu", action="store_true",
                   help="profiling mode: W warm-up and K steps of the workload at one precision, nothing else")
    p.add_argument("--ref-seconds", type=float, default=90.0)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-rate", type=float, default=20.0)
    p.add_argument("--serve-atoms", type=int, default=2_000_000)
    p.add_argument("--serve-queue", type=int, default=8)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, rank: int):
    """Replica `rank` of the workload: same system, its own thermal draw."""
    from paper_2502_19081_gb300 import inputs as I
    base = {"si_vacancy_215": 1, "fe_dumbbell_8001": 2, "fe_screw_256000": 3}[name]
    return I.workload(name, seed=base + 1000 * rank)


def max_over_ranks(total_ms: float, device=None) -> float:
    """Largest per-rank timed total (the job ends when the slowest replica does)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_atoms: int, steps: int, world: int, total_ms_max: float) -> float:
    """Whole-job atom-steps/s: every rank advanced its own replica `steps` steps."""
    return n_atoms * steps * world / (total_ms_max * 1e-3)


# ---------------------------------------------------------------------------
# algorithmic work model (per evaluated atom)


def exp_flops_per_atom(wl, info, nnb_rc: float, executed: bool = False) -> float:
    """Linear ACE: density 2 n nlm Nnb; pair gradients (4 n nlm + 8 nlm) Nnb;
    nu=2 readout + adjoint 4 n^2 nlm; nu=3 readout + adjoint as counted by the
    library from its l-triples (U = W A3 and omega3 = W^T Z, Z, E, and the
    omega1/omega2 terms that coinciding l's do not make redundant), with each
    triple's factors in the potential's own ascending order
    (mix_info.nu3_flops_ref_per_atom: the fixed algorithmic count), or, with
    executed=True, in the order the kernel contracts them (smallest l dense,
    mix_info.nu3_flops_per_atom: less work)."""
    a = wl.ace
    n, nlm = a.n_rad, (a.l_max + 1) ** 2
    f = 2.0 * n * nlm * nnb_rc + (4.0 * n * nlm + 8.0 * nlm) * nnb_rc
    if a.nu_max >= 2:
        f += 4.0 * n * n * nlm
    if a.nu_max >= 3:
        f += float(info["nu3_flops_per_atom" if executed else "nu3_flops_ref_per_atom"])
    return f


def cheap_flops_per_atom(nnb2: float, n3: float) -> float:
    """2+3-body spline: about 40 flops per pair and 650 per triplet."""
    return 40.0 * nnb2 + 650.0 * n3 * (n3 - 1) / 2.0


def neighbour_stats(ctx, wl):
    """Mean neighbours inside each cutoff over the evaluated sets (host-side
    analysis of the device lists, outside any timed region)."""
    x, _, _, _ = ctx.get_state()
    nnb, nbr, _ = ctx.neighbours()
    fl, ae, ac = ctx.sets()
    L = wl.system.box_len
    per = np.array(wl.system.periodic, dtype=bool)

    def counts(idx, rc):
        if len(idx) == 0:
            return 0.0
        out = []
        for i in idx:
            js = nbr[i, :nnb[i]]
            d = x[js, :3] - x[i, :3]
            d[:, per] -= L[per] * np.rint(d[:, per] / L[per])
            out.append(int(np.sum(np.sum(d * d, axis=1) < rc * rc)))
        return float(np.mean(out))

    se = ae if len(ae) <= 4000 else ae[:: max(1, len(ae) // 4000)]
    sc = ac if len(ac) <= 4000 else ac[:: max(1, len(ac) // 4000)]
    return {"n_exp": int(len(ae)), "n_cheap": int(len(ac)), "nnb_exp_rc": counts(se, wl.ace.r_cut),
            "nnb_cheap_rc": counts(sc, wl.spline.r_cut), "n3_cheap": counts(sc, wl.spline.r_cut3)}


# ---------------------------------------------------------------------------
# clocks


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm


def run_precision(mix, torch, wl, precision, steps, warmup, flush, regions=None):
    """Open a context, warm it up, let the library's autotuner pick its launch
    shapes (mix_tune: force evaluations at the current positions, the state
    unchanged), then time `steps` steps with the L2 flushed before each."""
    ctx = mix.open_context(wl, precision=precision, regions=regions)
    for _ in range(warmup):
        ctx.step(wl.dt, 1)
    ctx.sync()
    ctx.tune(3)
    ctx.sync()
    launches0 = ctx.info()["launches"]
    rebuilds0 = ctx.stats()["rebuilds"]
    ctx.profile(True)
    per_step = []
    for _ in range(steps):
        flush()
        ctx.step(wl.dt, 1)
        _, last, _ = ctx.get_profile()
        per_step.append(float(np.sum(last)))
    tot, _, nev = ctx.get_profile()
    ctx.profile(False)
    ctx.sync()
    launches = ctx.info()["launches"] - launches0
    rebuilds = ctx.stats()["rebuilds"] - rebuilds0
    return ctx, np.array(per_step), tot, nev, launches, rebuilds


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_leg(wl, x0, seconds: float):
    """The oracle as it stands (C, OpenMP over sites) on this host's cores: its
    forces and site energies at x0 (the GPU contexts' first positions), then
    consecutive mixed velocity-Verlet steps for about `seconds` (at least one)."""
    import oracle
    cores = host_cores()
    oracle.set_threads(cores)
    m = oracle.Model(wl)
    t0 = time.perf_counter()
    F, Ee, Ec = m.forces(x0, oracle.MODE_METHOD)
    t_force = time.perf_counter() - t0
    x, v, Fs = x0, np.array(wl.system.v, dtype=np.float64), F
    done = 0
    t0 = time.perf_counter()
    while True:
        x, v, Fs, _ = m.md(x, v, Fs, wl.dt, 1, oracle.MODE_METHOD)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds or done >= 50:
            break
    base = {"value": wl.system.n * done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} mixed velocity-Verlet step(s) of {wl.name} ({wl.system.n} atoms), FP64, "
                      f"OpenMP over sites on {cores} threads, {el:.1f} s (after one {t_force:.1f} s force "
                      f"evaluation at the starting positions, not timed)"}
    return base, F, Ee, Ec


def oracle_single_thread(names, seconds: float = 4.0):
    """Single-thread oracle throughput on the small workloads (one core)."""
    import oracle
    from paper_2502_19081_gb300 import inputs as I
    out = {}
    oracle.set_threads(1)
    try:
        for name in names:
            wl = I.workload(name)
            m = oracle.Model(wl)
            x, v = wl.system.x, wl.system.v
            F, _, _ = m.forces(x, oracle.MODE_METHOD)
            done = 0
            t0 = time.perf_counter()
            while True:
                x, v, F, _ = m.md(x, v, F, wl.dt, 1, oracle.MODE_METHOD)
                done += 1
                el = time.perf_counter() - t0
                if el >= seconds or done >= 200:
                    break
            out[name] = {"value": wl.system.n * done / el, "unit": UNIT, "cores": 1, "steps": done}
    finally:
        oracle.set_threads(host_cores())
    return out


def errors_against(ctx_F, ctx_E, F_ref, E_ref, flags):
    """max |dF| over atoms, max |dE_i| over each potential's evaluated sites and
    the error of each potential's total energy over its evaluated set."""
    dF = float(np.abs(ctx_F[:, :3] - F_ref[:, :3]).max()) if len(F_ref) else 0.0
    out = {"force_max_abs_eV_per_A": dF}
    for k, (e, er, bit) in enumerate(zip(ctx_E, E_ref, (4, 8))):
        sel = (flags & bit) > 0
        name = "exp" if k == 0 else "cheap"
        out[f"site_energy_{name}_max_abs_eV"] = float(np.abs(e[sel] - er[sel]).max()) if sel.any() else 0.0
        out[f"energy_{name}_total_abs_eV"] = float(abs(np.sum(e[sel]) - np.sum(er[sel])))
    return out


def phase_bytes(name: str, n: int, nst: dict, rebuild_frac: float) -> float:
    """Algorithmic DRAM bytes per step of a memory-bound phase (atom-major
    float64 rows of 32 B, int32 lists): disp reads x, v, f and writes x, v;
    lists (rebuild steps only) read x and write cell ids, nnb and the sorted
    rows and reverse slots; sets read x and the list and write weights and
    flags; gather reads both potentials' own and incoming slot rows (16 B a
    slot in float) and writes f, v."""
    nb = nst["nnb_list"]
    if name == "disp":
        return n * 96.0
    if name == "lists":
        return rebuild_frac * n * (32.0 + 4.0 + 4.0 + 8.0 * nb)
    if name == "sets":
        return n * (32.0 + 4.0 * nb + 9.0 + 4.0)
    if name == "gather":
        return nst["n_exp"] * 2 * 16.0 * nst["nnb_exp_rc"] + nst["n_cheap"] * 2 * 16.0 * nst["nnb_cheap_rc"] + n * 72.0
    return 0.0


def profiled_traffic(profile: str, sources) -> "int | None":
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel's sources changed since the capture (hash recorded in the summary)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.split(":", 1)[0] in ("traffic_bytes_per_launch", "kernel_source_sha256_16"):
            k, v = line.split(":", 1)
            vals[k] = v.strip()
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, "paper_2502_19081_gb300", "csrc", src), "rb").read())
    if vals.get("kernel_source_sha256_16") != h.hexdigest()[:16] or "traffic_bytes_per_launch" not in vals:
        return None
    return int(vals["traffic_bytes_per_launch"])


def gpu_leg(mix, torch, wl, prec, args, flush, peaks, hbm, oracle_seconds, e2e=True, timed_steps=None,
            secondary_steps=None, candidates=None):
    """Everything the line reports for one workload on the GPU (and, unless
    --no-cpu, the oracle beside it).  prec None: the first of `candidates`
    whose force error against the FP64 path at the starting positions is
    within the gate (else FP32) is the headline precision; every candidate
    and the FP64 path are timed beside it."""
    steps = args.steps if timed_steps is None else timed_steps
    sec = args.secondary_steps if secondary_steps is None else secondary_steps
    names = mix.PHASE_NAMES
    candidates = list(candidates or [])
    # FP64 path at the starting positions: reference bits for the other precisions
    c64 = mix.open_context(wl, precision=mix.MIX_FP64)
    x0, _, F64, _ = c64.get_state()
    E64 = c64.site_energies()
    flags, _, _ = c64.sets()
    nst = neighbour_stats(c64, wl)
    nnb, _, _ = c64.neighbours()
    nst["nnb_list"] = float(np.mean(nnb)) if len(nnb) else 0.0
    info = c64.info()
    c64.close()
    firsts = {mix.MIX_FP64: (F64, E64)}
    for p in [mix.MIX_FP32] + candidates + ([prec] if prec is not None else []):
        if p in firsts:
            continue
        cp = mix.open_context(wl, precision=p)
        _, _, Fp, _ = cp.get_state()
        firsts[p] = (Fp, cp.site_energies())
        cp.close()
    if prec is None:
        prec = mix.MIX_FP32
        for p in candidates:
            if float(np.abs(firsts[p][0][:, :3] - F64[:, :3]).max()) <= GATE:
                prec = p
                break

    ctx, per, tot, nev, launches, rebuilds = run_precision(mix, torch, wl, prec, steps, args.warmup, flush)
    hinfo = ctx.info()
    total_ms = float(per.sum())
    e2e_blk = None
    if e2e:
        n = wl.system.n
        hx = torch.empty((n, 4), dtype=torch.float64, pin_memory=True)
        hv = torch.empty_like(hx, pin_memory=True)
        hf = torch.empty_like(hx, pin_memory=True)
        xs, vs, fs, _ = ctx.get_state()
        hx.numpy()[:] = xs
        hv.numpy()[:] = vs
        hf.numpy()[:] = fs
        e2e_s = []
        for _ in range(max(1, args.e2e_steps)):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.step_host(hx.numpy(), hv.numpy(), hf.numpy(), wl.dt, 1)
            e2e_s.append(time.perf_counter() - t0)
        e2e_blk = {"value": n / float(np.mean(e2e_s)), "unit": UNIT, "h2d_bytes_per_step": 3 * n * 32,
                   "d2h_bytes_per_step": 3 * n * 32, "steps": len(e2e_s),
                   "entry": "mix_step_host (x, v, f in and out, pinned host memory)"}
    ctx.close()

    # the FP64 path (or FP32 when FP64 is the headline), shorter
    other = mix.MIX_FP64 if prec != mix.MIX_FP64 else mix.MIX_FP32
    c2, per2, tot2, nev2, _, _ = run_precision(mix, torch, wl, other, sec, 3, flush)
    c2.close()
    # the other reduced precisions, as long as the FP64 path's run
    others = {}
    for p in firsts:
        if p in (prec, other):
            continue
        cq, perq, totq, nevq, _, _ = run_precision(mix, torch, wl, p, sec, 3, flush)
        cq.close()
        others[p] = {"value": wl.system.n * len(perq) / (perq.sum() * 1e-3), "ms_per_step": float(perq.mean()),
                     "p50_ms": float(np.percentile(perq, 50)), "p99_ms": float(np.percentile(perq, 99)),
                     "kernels_ms": {names[k]: float(totq[k] / max(nevq, 1)) for k in range(len(names))}}

    # pure potentials on every atom, same arithmetic: the measured speed ratio
    # S_C/E and the zero-overhead bound (paper SI, load balancing)
    centre = tuple(float(v) for v in np.asarray(wl.system.box_lo) + 0.5 * np.asarray(wl.system.box_len))
    from paper_2502_19081_gb300 import inputs as I
    everywhere = [I.Region(I.REGION_SPHERE, centre, (0.0, 0.0, 1.0), 1.0e4, 1.0)]
    pure = {}
    for key, regs in (("exp", everywhere), ("cheap", [])):
        cx, perx, _, _, _, _ = run_precision(mix, torch, wl, prec, max(3, sec // 2), 3, flush, regions=regs)
        cx.close()
        pure[key] = float(np.mean(perx))

    n = wl.system.n
    ms_step = total_ms / steps
    phase_ms = tot / max(nev, 1)
    pe = exp_flops_per_atom(wl, info, nst["nnb_exp_rc"])
    pe_run = exp_flops_per_atom(wl, info, nst["nnb_exp_rc"], executed=True)
    pc = cheap_flops_per_atom(nst["nnb_cheap_rc"], nst["n3_cheap"])
    rf = rebuilds / max(steps, 1)
    kern = {}
    for p, nm in enumerate(names):
        kb = {"ms": float(phase_ms[p]), "share": float(phase_ms[p] / phase_ms.sum())}
        if nm == "exp":
            kb["algorithmic_flops"] = pe * nst["n_exp"]
            kb["executed_flops"] = pe_run * nst["n_exp"]
            kb["tflops"] = kb["algorithmic_flops"] / (phase_ms[p] * 1e-3) / 1e12 if phase_ms[p] > 0 else 0.0
        elif nm == "cheap":
            kb["algorithmic_flops"] = pc * nst["n_cheap"]
            if hinfo["potential_order"] == mix.MIX_ORDER_SERIAL:
                # one stream: the phase is the cheap kernel's own duration
                kb["tflops"] = kb["algorithmic_flops"] / (phase_ms[p] * 1e-3) / 1e12 if phase_ms[p] > 0 else 0.0
                kb["note"] = "after exp on the same stream (order chosen by mix_tune); ms = its own duration"
            else:
                # on a second stream beside the expensive kernel: its phase time
                # is only the part not hidden behind it; its own throughput
                # comes from the pure-cheap step below
                first = "cheap" if hinfo["potential_order"] == mix.MIX_ORDER_CHEAP_FIRST else "exp"
                kb["note"] = (f"concurrent with exp on a second stream, {first} launched first (order chosen by "
                              "mix_tune); ms = the part after exp ends")
        else:
            kb["algorithmic_bytes"] = phase_bytes(nm, n, nst, rf)
            kb["gbs"] = kb["algorithmic_bytes"] / (phase_ms[p] * 1e-3) / 1e9 if phase_ms[p] > 0 else 0.0
            kb["hbm_frac"] = kb["gbs"] / hbm
        kern[nm] = kb
    kern["cheap"]["pure_cheap_step_tflops"] = pc * n / (pure["cheap"] * 1e-3) / 1e12
    s_ce = pure["exp"] / pure["cheap"]
    s_ul = n * s_ce / (nst["n_exp"] * s_ce + nst["n_cheap"])
    speedup = pure["exp"] / ms_step
    blk = {
        "value": n * steps / (total_ms * 1e-3), "ms_per_step": ms_step,
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "per_step_ms": per, "total_ms": total_ms, "phase_ms": phase_ms, "launches": int(launches),
        "kernels": kern, "nstat": nst, "info": info, "hinfo": hinfo, "pe": pe, "pc": pc, "rebuilds": int(rebuilds),
        "other": {"precision": other, "value": n * len(per2) / (per2.sum() * 1e-3),
                  "ms_per_step": float(per2.mean()), "p50_ms": float(np.percentile(per2, 50)),
                  "p99_ms": float(np.percentile(per2, 99)),
                  "kernels_ms": {names[p]: float(tot2[p] / max(nev2, 1)) for p in range(len(names))}},
        "mixing": {"pure_expensive_ms_per_step": pure["exp"], "pure_cheap_ms_per_step": pure["cheap"],
                   "s_ce_measured": s_ce, "speedup": speedup, "s_ul": s_ul, "speedup_over_s_ul": speedup / s_ul,
                   "note": "speedup = pure-expensive step / mixed step, same arithmetic; s_ul = N S / (N_E S + N_C) "
                           "with S = S_C/E the measured ratio of the pure-expensive to the pure-cheap step time "
                           "(paper SI, load balancing); N_E, N_C = evaluated set sizes"},
        "e2e": e2e_blk, "x0": x0, "flags": flags, "firsts": firsts, "prec": prec, "others": others,
    }
    blk["errors_vs_gpu_fp64"] = {mix.PREC_NAMES[p]: errors_against(F, E, F64, E64, flags)
                                 for p, (F, E) in firsts.items() if p != mix.MIX_FP64}
    if not args.no_cpu:
        cpu, Fo, Eeo, Eco = oracle_leg(wl, x0, oracle_seconds)
        blk["cpu_baseline"] = cpu
        blk["errors_vs_oracle"] = {mix.PREC_NAMES[p]: errors_against(F, E, Fo, (Eeo, Eco), flags)
                                   for p, (F, E) in firsts.items()}
    return blk


def profile_run(args):
    """The command the committed ncu summaries were taken with: one context of
    the workload (precision auto: bf16 for the screw cylinder, else fp32), W
    warm-up steps, the library's autotuner (as the timed runs use it), and K
    steps between cudaProfilerStart and cudaProfilerStop (ncu
    --profile-from-start off captures those alone), synchronised, and a
    one-line summary."""
    import torch
    from paper_2502_19081_gb300 import build as B
    from paper_2502_19081_gb300 import mix
    torch.cuda.set_device(0)
    B.build()
    if args.workload == "si_replicas_256":
        from paper_2502_19081_gb300 import inputs as I
        wls = I.si_replicas(256, seed=4)
        ctxs = [mix.open_context(w, precision=mix.MIX_FP32) for w in wls]
        b = mix.Batch(ctxs)
        b.step(1.0, args.warmup)
        b.sync()
        t0 = time.perf_counter()
        b.step(1.0, args.steps)
        b.sync()
        print(json.dumps({"mode": "ncu", "workload": "si_replicas_256", "precision": "f32", "steps": args.steps,
                          "wall_s": time.perf_counter() - t0, "batch": b.info()}), flush=True)
        b.close()
        return
    wl = make_workload(args.workload, 0)
    pmap = {"fp32": mix.MIX_FP32, "fp64": mix.MIX_FP64, "bf16": mix.MIX_BF16, "bf16x3": mix.MIX_BF16_SPLIT}
    prec = pmap.get(args.precision, mix.MIX_BF16 if args.workload == "fe_screw_256000" else mix.MIX_FP32)
    ctx = mix.open_context(wl, precision=prec)
    ctx.step(wl.dt, args.warmup)
    ctx.sync()
    ctx.tune(3)
    ctx.sync()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    ctx.step(wl.dt, args.steps)
    ctx.sync()
    el = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    print(json.dumps({"mode": "ncu", "workload": wl.name, "precision": mix.PREC_NAMES[prec], "steps": args.steps,
                      "wall_s": el, "info": ctx.info()}), flush=True)
    ctx.close()


def blended_energy(ctx, mass: float) -> float:
    """KE + sum_i [w_i E_exp,i + (1 - w_i) E_cheap,i] of a context's current
    state (eV): the energy force mixing would conserve if it were the gradient
    of one function (it is not; the drift measures the difference)."""
    x, v, _, _ = ctx.get_state()
    ee, ec = ctx.site_energies()
    _, w = ctx.lam()
    ke = 0.5 * mass * float(np.sum(v[:, :3] ** 2)) / 9.6485332e-3
    return ke + float(np.sum(w * ee + (1.0 - w) * ec))


def nve_drift(mix, wl, precision, steps, regions=None):
    """Drift of the blended energy over an NVE run, per atom and as the
    temperature it amounts to (3/2 k_B per atom), per picosecond."""
    ctx = mix.open_context(wl, precision=precision, regions=regions)
    h0 = blended_energy(ctx, wl.system.mass)
    ctx.step(wl.dt, steps)
    h1 = blended_energy(ctx, wl.system.mass)
    ctx.close()
    n = wl.system.n
    ps = steps * wl.dt * 1e-3
    de = (h1 - h0) / n
    return {"steps": steps, "dt_fs": wl.dt, "dE_per_atom_eV": de, "eV_per_atom_per_ps": de / ps,
            "K_per_ps": de / (1.5 * 8.617333262e-5) / ps}


def drift_block(mix):
    """Mixed-NVE drift of the Si vacancy cell (100 steps, float64) and the Fe
    dumbbell cell (1000 steps, float), each beside the same run with the pure
    cheap potential (no regions): the integrator's own error."""
    from paper_2502_19081_gb300 import inputs as I
    out = {}
    for name, prec, steps in (("si_vacancy_215", mix.MIX_FP64, 100), ("fe_dumbbell_8001", mix.MIX_FP32, 1000)):
        wl = I.workload(name)
        out[name] = {"precision": mix.PREC_NAMES[prec], "mixed": nve_drift(mix, wl, prec, steps),
                     "pure_cheap": nve_drift(mix, wl, prec, steps, regions=[])}
    return out


def ours(args):
    import torch
    import torch.distributed as dist
    from paper_2502_19081_gb300 import build as B
    from paper_2502_19081_gb300 import mix

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    B.build()
    wl = make_workload(args.workload, rank)
    pmap = {"fp32": mix.MIX_FP32, "fp64": mix.MIX_FP64, "bf16": mix.MIX_BF16, "bf16x3": mix.MIX_BF16_SPLIT}
    # auto: the 256,000-atom cylinder's readout runs on the tensor cores in bf16,
    # the hi/lo split when plain bf16 misses the force gate; FP32 elsewhere
    prec = pmap.get(args.precision)
    cands = [mix.MIX_BF16, mix.MIX_BF16_SPLIT] if args.precision == "auto" and args.workload == "fe_screw_256000" \
        else []
    if args.precision == "auto" and not cands:
        prec = mix.MIX_FP32
    flush_buf = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def flush():
        flush_buf.zero_()

    peaks = {p: mix.fma_peak(p) for p in (mix.MIX_FP64, mix.MIX_FP32)}
    peaks_file = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = json.load(open(peaks_file))["hbm_gbs"] if os.path.exists(peaks_file) else 6800.0

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    main = gpu_leg(mix, torch, wl, prec, args, flush, peaks, hbm, args.cpu_seconds if rank == 0 else 0.0,
                   candidates=cands)
    prec = main["prec"]
    clk = clocks.stop()
    total_max = max_over_ranks(main["total_ms"], device="cuda")
    value = job_throughput(wl.system.n, args.steps, world, total_max)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    names = mix.PHASE_NAMES
    phase_ms = main["phase_ms"]
    dom = int(np.argmax(phase_ms))
    peak = peaks[mix.MIX_FP64 if prec == mix.MIX_FP64 else mix.MIX_FP32]
    kern = main["kernels"]
    if names[dom] in ("exp", "cheap"):
        fl = kern[names[dom]]["algorithmic_flops"]
        ach = fl / (phase_ms[dom] * 1e-3)
        roof = {"kernel": "k_ace" if names[dom] == "exp" else "k_spline", "bound": "alu",
                "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": (profiled_traffic(f"k_ace_{mix.PREC_NAMES[prec]}_{wl.name}.md",
                                             ("k_ace.cuh", "k_ace_f32.cu") if prec == mix.MIX_FP32 else
                                             ("k_ace.cuh", "k_ace_tc.cuh", "k_ace_tc1.cu", "tc.cuh"))
                            if names[dom] == "exp" and prec != mix.MIX_FP64 else None),
                "algorithmic_flops_per_launch": fl,
                "peak_source": "measured FMA microbenchmark "
                               f"({'fp64' if prec == mix.MIX_FP64 else 'fp32'}), mix_fma_peak (of measured)"}
        if names[dom] == "exp":
            # the work the kernel does with the smallest l of each triple dense
            fx = kern["exp"]["executed_flops"]
            roof["executed_flops_per_launch"] = fx
            roof["frac_executed"] = fx / (phase_ms[dom] * 1e-3) / peak
        if names[dom] == "exp" and prec in (mix.MIX_BF16, mix.MIX_BF16_SPLIT):
            # the part of the kernel on the tensor cores: V = Z W per l-triple,
            # 2 d3 n^2 n flops per atom (three products with the split)
            tfl = main["hinfo"]["tc_flops_per_atom"] * main["nstat"]["n_exp"]
            tpk = json.load(open(peaks_file))["bf16_tflops"] * 1e12 if os.path.exists(peaks_file) else 1.9e15
            roof["tensor_part"] = {"flops_per_launch": tfl, "achieved": tfl / (phase_ms[dom] * 1e-3) / 1e12,
                                   "peak": tpk / 1e12, "unit": "TFLOP/s",
                                   "frac": tfl / (phase_ms[dom] * 1e-3) / tpk,
                                   "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)"}
    else:
        byts = kern[names[dom]]["algorithmic_bytes"]
        ach = byts / (phase_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None, "algorithmic_bytes_per_launch": byts,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    n = wl.system.n
    pname = mix.PREC_NAMES[prec]
    other = main["other"]
    nst = main["nstat"]
    errs = main.get("errors_vs_oracle", main["errors_vs_gpu_fp64"])
    ferr = errs[pname]["force_max_abs_eV_per_A"] if pname in errs else 0.0
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_max / args.steps,
        "p50_ms": main["p50_ms"],
        "p99_ms": main["p99_ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": pname,
        "data": "synthetic (seeded lattice, defect, thermal displacements and potential coefficients)",
        "config": {"workload": wl.name, "n_atoms": n, "potential_arithmetic": pname, "integration": "f64",
                   "expensive": f"linear ACE n={wl.ace.n_rad} lmax={wl.ace.l_max} body order {wl.ace.nu_max + 1}",
                   "cheap": "2+3-body cubic B-spline", "l2": "flushed before every timed step (512 MB write)",
                   "parallelism": f"replicas x{world}", "evaluated_exp": nst["n_exp"],
                   "evaluated_cheap": nst["n_cheap"]},
        "force_err_vs_oracle_eV_per_A": ferr,
        "gate_eV_per_A": GATE,
        "within_gate": bool(ferr <= GATE),
        "errors": errs,
        "errors_reference": "oracle (FP64 CPU) at the starting positions" if "errors_vs_oracle" in main
                            else "GPU FP64 path at the starting positions",
        mix.PREC_NAMES[other["precision"]] + "_path": {k: v for k, v in other.items() if k != "precision"},
        "precisions": {mix.PREC_NAMES[p]: dict(v, force_err_eV_per_A=errs.get(mix.PREC_NAMES[p], {}).get(
            "force_max_abs_eV_per_A"), within_gate=bool(errs.get(mix.PREC_NAMES[p], {}).get(
                "force_max_abs_eV_per_A", 1.0) <= GATE)) for p, v in main["others"].items()},
        "roofline": roof,
        "kernels": kern,
        "launch": {k: main["hinfo"][k] for k in ("potential_order", "exp_grid", "exp_threads", "exp_smem_bytes",
                                                 "cheap_grid", "cheap_lanes", "gather_grid", "buffer_grid")},
        "mixing": main["mixing"],
        "fma_peak_tflops": {"fp64": peaks[mix.MIX_FP64] / 1e12, "fp32": peaks[mix.MIX_FP32] / 1e12},
        "e2e": main["e2e"],
        "gpu_launches": main["launches"],
        "rebuilds_in_timed_steps": main["rebuilds"],
        "clocks": clk,
    }
    if "cpu_baseline" in main:
        out["cpu_baseline"] = main["cpu_baseline"]
    # the 8,001-atom Fe dumbbell beside it: the configuration the paper's ~11x
    # mixing speedup at ~8,000 atoms is comparable with
    if args.workload != "fe_dumbbell_8001" and not args.no_secondary:
        wl2 = make_workload("fe_dumbbell_8001", 0)
        sec = gpu_leg(mix, torch, wl2, mix.MIX_FP32, args, flush, peaks, hbm, 8.0, e2e=True,
                      timed_steps=max(10, args.steps), secondary_steps=args.secondary_steps)
        e2 = sec.get("errors_vs_oracle", sec["errors_vs_gpu_fp64"])
        out["fe_dumbbell_8001"] = {
            "value": sec["value"], "ms_per_step": sec["ms_per_step"], "p50_ms": sec["p50_ms"],
            "p99_ms": sec["p99_ms"], "dtype": "f32", "errors": e2, "f64_path": sec["other"],
            "mixing": sec["mixing"], "kernels": sec["kernels"], "e2e": sec["e2e"],
            "cpu_baseline": sec.get("cpu_baseline"),
            "evaluated_exp": sec["nstat"]["n_exp"], "evaluated_cheap": sec["nstat"]["n_cheap"]}
    if not args.no_secondary:
        out["nve_drift"] = drift_block(mix)
    if not args.no_cpu:
        out["oracle_single_thread"] = oracle_single_thread(["si_vacancy_215", "fe_dumbbell_8001"])
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def batch_bench(args):
    """256 independent Si defect cells (1.59 M atoms in total), FP32 potentials
    and FP64 integration, advanced by one graph launch per step (mix_batch);
    launch shapes autotuned first.  The batch's working set (lists and slot
    gradients, ~1 GB) exceeds L2, so no flush is needed between steps."""
    import torch
    from paper_2502_19081_gb300 import build as B
    from paper_2502_19081_gb300 import inputs as I
    from paper_2502_19081_gb300 import mix
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    wls = I.si_replicas(256, seed=4 + 1000 * rank)
    ctxs = [mix.open_context(wl, precision=mix.MIX_FP32) for wl in wls]
    b = mix.Batch(ctxs)
    div = b.tune(reps=3)
    for _ in range(args.warmup):
        b.step(1.0, 1)
    b.sync()
    s = ctxs[0].stream
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    for k in range(args.steps):
        e0[k].record(s)
        b.step(1.0, 1)
        e1[k].record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    b.sync()
    per = np.array([a.elapsed_time(c) for a, c in zip(e0, e1)])
    natoms = sum(wl.system.n for wl in wls)
    binfo = b.info()
    # the same batch stepped as one child graph per member, for comparison
    b.set_fused(False)
    b.step(1.0, 2)
    torch.cuda.synchronize()
    ch0, ch1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nch = max(3, min(10, args.steps))
    ch0.record(s)
    b.step(1.0, nch)
    ch1.record(s)
    torch.cuda.synchronize()
    child_ms = ch0.elapsed_time(ch1) / nch
    b.set_fused(True)
    out = {"metric": METRIC, "value": natoms * args.steps / (per.sum() * 1e-3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(per.mean()),
           "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
           "higher_is_better": True, "dtype": "f32",
           "config": {"workload": "si_replicas_256", "n_atoms": natoms, "replicas": len(wls),
                      "potential_arithmetic": "f32", "integration": "f64", "grid_divisor": div,
                      "step": "fused: one launch per kernel for all replicas" if binfo["fused"]
                      else "one child graph per replica",
                      "l2": "working set > L2 (no flush)"},
           "gpu_launches": binfo["launches"],
           "child_graph_ms_per_step": child_ms,
           "clocks": clk}
    b.close()
    print(json.dumps(out), flush=True)


def serve_window(mix, I, stream, pots, seconds, precision, max_active_atoms, queue, clocks=None):
    """Serve the arrival stream for `seconds` of wall clock with one server:
    requests are generated when they arrive (a client-side backlog holds them
    while the server's queue is full), the server admits, batches and steps
    them (one step a tick).  Returns the served throughput and the latencies:
    per-request per-step (each active request waits one batched step per tick:
    the step's device time and the tick's wall time, over all (request, step)
    pairs) and queueing delay (admission minus arrival)."""
    import collections
    srv = mix.Server(1.0, max_active_atoms=max_active_atoms)
    pending = collections.deque(stream)
    backlog = collections.deque()
    arrival = {}
    step_dev, step_wall, atoms_per_step, qdelay, done = [], [], [], [], []
    served = 0.0
    server_queued = 0
    t0 = time.perf_counter()
    while True:
        t_now = time.perf_counter() - t0
        if t_now >= seconds:
            break
        while pending and pending[0]["t"] <= t_now:
            backlog.append(pending.popleft())
        while backlog and server_queued < queue:
            r = backlog.popleft()
            wl = I.serve_request(r["seed"], r["element"], r["n_target"], r["core_frac"], r["temp_k"], pots)
            rid = srv.submit(wl, r["nsteps"], precision=precision, nbr_cap=128 if r["element"] == "Si" else 0)
            arrival[rid] = r["t"]
            server_queued += 1
        tw = time.perf_counter()
        t = srv.tick(1)
        tw = time.perf_counter() - tw
        server_queued = t["queued"]
        if t["steps"]:
            step_dev += [t["step_ms"]] * t["active"]
            step_wall += [tw * 1e3] * t["active"]
            atoms_per_step.append(t["active_atoms"])
            served += t["active_atoms"] * t["steps"]
        for rid in list(arrival):
            info = srv.request(rid)
            if info["state"] in (mix.MIX_REQ_DONE, mix.MIX_REQ_FAILED):
                qdelay.append(info["t_admit"] - arrival[rid] if info["t_admit"] >= 0 else float("nan"))
                done.append((rid, info["state"], info["steps_done"], info["status"]))
                try:
                    srv.fetch(rid)
                except mix.MixError:
                    pass
                del arrival[rid]
        if t["active"] == 0 and t["queued"] == 0 and not backlog and pending:
            time.sleep(max(0.0, min(pending[0]["t"] - (time.perf_counter() - t0), 0.05)))
    wall = time.perf_counter() - t0
    active_delay = []
    for rid, ta in arrival.items():
        info = srv.request(rid)
        if info["t_admit"] >= 0:
            active_delay.append(info["t_admit"] - ta)
    srv.close()
    dev = np.array(step_dev) if step_dev else np.zeros(1)
    wal = np.array(step_wall) if step_wall else np.zeros(1)
    qd = np.array([q for q in qdelay + active_delay if q == q]) if (qdelay or active_delay) else np.zeros(1)
    return {
        "value": served / wall, "wall_s": wall, "ticks": len(atoms_per_step),
        "per_request_step_ms": {"device_p50": float(np.percentile(dev, 50)), "device_p99": float(np.percentile(dev, 99)),
                                "wall_p50": float(np.percentile(wal, 50)), "wall_p99": float(np.percentile(wal, 99)),
                                "pairs": len(step_dev)},
        "arrived": len(stream) - len(pending), "completed": sum(1 for d in done if d[1] == mix.MIX_REQ_DONE),
        "failed": sum(1 for d in done if d[1] == mix.MIX_REQ_FAILED),
        "failed_by_status": dict(collections.Counter(
            mix.lib().mix_strerror(d[3]).decode() for d in done if d[1] == mix.MIX_REQ_FAILED)),
        "admitted": len(done) + len(active_delay),
        "queue_delay_s": {"p50": float(np.percentile(qd, 50)), "p99": float(np.percentile(qd, 99))},
        "mean_active_atoms": float(np.mean(atoms_per_step)) if atoms_per_step else 0.0,
    }


def serve_bench(args):
    """Serving: a Poisson stream of requests (20 per second; Si or Fe cells of
    1e3 to 5e5 atoms, log-uniform; 100 to 2000 steps, log-uniform; core 1 to
    10 % of the atoms) served for a bounded wall-clock window by the library's
    server (mix_server_*): admission by device memory and an active-atom cap,
    continuous batching, one step per tick, FP32 potentials with FP64
    integration.  The same stream is then served by the plain FP64 unbatched
    path (every request alone, float64 potentials) for a shorter window, as the
    comparator.  value = atom-steps served per second of the window."""
    import torch
    from paper_2502_19081_gb300 import build as B
    from paper_2502_19081_gb300 import inputs as I
    from paper_2502_19081_gb300 import mix
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    pots = I.serve_potentials()
    stream = list(I.serve_stream(seed=5 + 1000 * rank, rate=args.serve_rate, duration=args.serve_seconds))
    offered = sum(r["n_target"] * r["nsteps"] for r in stream) / args.serve_seconds
    clocks = Clocks(local)
    clocks.start()
    main = serve_window(mix, I, stream, pots, args.serve_seconds, mix.MIX_FP32, args.serve_atoms, args.serve_queue)
    clk = clocks.stop()
    base_s = max(10.0, args.serve_seconds / 3.0)
    base = serve_window(mix, I, [r for r in stream if r["t"] < base_s], pots, base_s, mix.MIX_FP64, 1,
                        args.serve_queue)
    out = {"metric": "served atom-steps/s, Poisson request stream (continuous batching)",
           "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": main["ticks"], "warmup": 0,
           "p50_ms": main["per_request_step_ms"]["device_p50"], "p99_ms": main["per_request_step_ms"]["device_p99"],
           "higher_is_better": True, "dtype": "f32",
           "config": {"workload": "serve_poisson", "rate_per_s": args.serve_rate, "window_s": args.serve_seconds,
                      "max_active_atoms": args.serve_atoms, "server_queue": args.serve_queue,
                      "potential_arithmetic": "f32", "integration": "f64",
                      "l2": "working set > L2 (no flush)"},
           "offered_atom_steps_per_s": offered,
           "served": {k: v for k, v in main.items() if k != "value"},
           "fp64_unbatched": dict(base, window_s=base_s,
                                  note="the plain FP64 path: float64 potentials, one request at a time "
                                       "(active-atom cap 1), the same arrival stream"),
           "speedup_over_fp64_unbatched": main["value"] / base["value"] if base["value"] > 0 else None,
           "clocks": clk}
    print(json.dumps(out), flush=True)


def reference(args):
    """The oracle arm: FP64 C oracle on the host cores, same workload and
    metric.  One oracle step of the 256,000-atom cylinder takes seconds, so
    the arm times at most K steps within --ref-seconds (at least one) after
    one untimed force evaluation (its warm-up), and says so in the line."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = make_workload(args.workload, 0)
    cores = host_cores()
    oracle.set_threads(cores)
    m = oracle.Model(wl)
    x, v = wl.system.x, wl.system.v
    F, _, _ = m.forces(x, oracle.MODE_METHOD)
    per = []
    t_all = time.perf_counter()
    while len(per) < args.steps:
        t0 = time.perf_counter()
        x, v, F, _ = m.md(x, v, F, wl.dt, 1, oracle.MODE_METHOD)
        per.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all >= args.ref_seconds:
            break
    per = np.array(per)
    value = wl.system.n * len(per) / per.sum()
    sample = (f"{len(per)} of the {args.steps} requested mixed velocity-Verlet steps of {wl.name} "
              f"({wl.system.n} atoms), FP64, OpenMP over sites on {cores} threads, bounded at "
              f"{args.ref_seconds:.0f} s; warm-up: one untimed force evaluation")
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": len(per),
        "steps_requested": args.steps,
        "warmup": args.warmup,
        "ms_per_step": float(per.mean() * 1e3),
        "p50_ms": float(np.percentile(per, 50) * 1e3),
        "p99_ms": float(np.percentile(per, 99) * 1e3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "n_atoms": wl.system.n, "potential_arithmetic": "f64",
                   "integration": "f64", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
    elif args.ncu:
        profile_run(args)
    elif args.workload == "si_replicas_256":
        batch_bench(args)
    elif args.workload == "serve_poisson":
        serve_bench(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
