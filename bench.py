"""Benchmark: spacetime unknowns relaxed per second of the least-action propagator on one GB300.

Default line: the 3D workload's forward propagation (128^3 points, K = 4 Legendre time functions,
4 x 4 x 4-point subvolumes of 256 unknowns, 4-level V(1,2) cycles with a (1,0) Galerkin cycle, FP64
residual, action and refinement with complex64 local solves, tolerance 1e-10 on N/N(0)).  A "step"
is one least-action time step: time matrices, right-hand side, subvolume factorisation on every
level, V-cycles to tolerance from the trial extrapolated from the last three steps, step advance.
Metric = (finest-level unknowns) x (finest-level sweeps) / time.  The same JSON line carries clocked
sub-records: the same 3D problem in plain FP64, the 2D workload's whole 200-step propagation in FP64
and in mixed precision, and the 512-grid batch in FP64 and mixed precision, each with its speed-up
at the same tolerance, plus the FMA peaks of this GPU measured in the run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision -1|0|1]
                  [--workload 3d|3d-small|3d-mid|2d|2d-small|1d|2d-square|batched|3d-adjoint|lfa]
                  [--trial -1|0..3] [--headline-only]

N > 1 runs N independent replicas (one propagation per rank, no collective: the path does not
shard).  ``--impl reference`` times the CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1111_4363_gb300 import workloads as wl  # noqa: E402

METRIC = "spacetime unknowns relaxed/s"
# (kernel class, precision) -> DRAM bytes (read + write) per finest-level subvolume of the current kernels,
# from one-pass ncu captures of full-size launches, scaled to a launch by the subvolumes it processes
# (set to None when a kernel changes):
# - 2D 256x256 FP64: the finest k_factor launch (4096 subvolumes) and one full k_sweep_fine sweep (four
#   colour launches), profiles/dram_2d_softcore_256x256_fp64.md
# - 3D 128^3 complex64: one k_factor_wide launch (32768 subvolumes of 256 unknowns) and one full wide
#   sweep (eight colour launches of 4096), profiles/dram_3d_hydrogen_128x128x128_mixed.md
NCU_BYTES_PER_SUBVOLUME = {("factor", 0): (867072 + 287257600) / 4096,
                           ("sweep", 0): (390778880 + 216064) / 4096,
                           ("factor_wide", 1): (33378560 + 9068625920) / 32768,
                           ("sweep_wide", 1): (10943546368 + 56069376) / 32768}
FP64_PEAK_TFLOPS = 152 * 4 * 2070e6 / 1e12   # 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz (derived)
FP32_PEAK_TFLOPS = 152 * 256 * 2070e6 / 1e12  # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz (derived)
L2_BYTES = 129 * 2 ** 20


# production schedule of the 2D workload: 4-level cycles, V(1,2) on the finest level and one
# pre-sweep on the Galerkin levels, started from the quadratic trial (2 cycles per step to 1e-10,
# against 5 for V(1,1) from c = 0); --trial 0 gives the plain start
PRODUCTION_2D = dict(nu1=1, nu2=2, coarse_nu=(1, 0), trial=3)
# the same shape for the 3D workload (4 levels): 2 cycles per step instead of 3 for V(1,1)
PRODUCTION_3D = dict(nu1=1, nu2=2, coarse_nu=(1, 0), trial=3)


def workload(name: str) -> wl.Workload:
    if name == "2d":
        return dataclasses.replace(wl.softcore_2d(n=256, levels=4, nsteps=200), **PRODUCTION_2D)
    if name == "2d-small":          # the same problem on 128 x 128, for ncu captures of single kernels
        return dataclasses.replace(wl.softcore_2d(n=128, levels=4, nsteps=200), **PRODUCTION_2D)
    if name == "1d":
        return wl.harmonic_1d()
    if name == "3d":                # the 3D workload's forward propagation: 128^3, K = 4, 4x4x4 subvolumes
        return dataclasses.replace(wl.hydrogen_3d(n=128, nsteps=400), **PRODUCTION_3D)
    if name == "3d-small":          # the same problem on 32^3, for ncu captures of single kernels
        return dataclasses.replace(wl.hydrogen_3d(n=32, nsteps=400), **PRODUCTION_3D)
    if name == "3d-mid":            # on 64^3: one full wave of per-point kernels (1024 CTAs) for ncu
        return dataclasses.replace(wl.hydrogen_3d(n=64, nsteps=400), **PRODUCTION_3D)
    if name == "2d-square":         # the paper's square local form (Sec. II), single level, red-black
        return dataclasses.replace(wl.softcore_2d(n=256, levels=1, nsteps=200), local_form="square", nu1=1, nu2=1,
                                   trial=3)
    raise ValueError(name)


def action_trajectory(B, torch, w, dt, local_form, nsweeps):
    """N(c)/N(0) after each of nsweeps single sweeps of the first step from c = 0 (single level, one
    sweep per cycle), for the given local form and time step."""
    v = dataclasses.replace(w, dt=dt, levels=1, nu1=1, nu2=0, local_form=local_form, trial=0, coarse_nu=None)
    ctx = B.Context(B.config_from_workload(v))
    ctx.set_hamiltonian(torch.tensor(wl.potential(v).ravel(), dtype=torch.float64, device="cuda"), v.pulse)
    psi0 = torch.from_numpy(wl.initial_state(v).ravel()).cuda()
    c = torch.zeros(v.nunknowns, dtype=torch.complex128, device="cuda")
    out = []
    for s in range(1, nsweeps + 1):
        st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, 0.0, c, ncycles=s)
        out.append(rel)
    ctx.close()
    return out


def square_form_report(B, torch, w):
    """Action per sweep of the square form against the least-squares form at the workload's kappa and
    at kappa = 2.5 (dt = 0.2 on h = 0.2): Sec. II notes the square form need not decrease the action."""
    rep = {}
    for dt in (w.dt, 0.2):
        kappa = dt / (2 * w.h[0] ** 2)
        sq = action_trajectory(B, torch, w, dt, "square", 8)
        ls = action_trajectory(B, torch, w, dt, "lsq", 8)
        rep[f"kappa_{kappa:g}"] = {
            "square_rel_action_per_sweep": [float(f"{x:.3e}") for x in sq],
            "square_monotone": all(b <= a for a, b in zip([1.0] + sq, sq)),
            "least_squares_rel_action_per_sweep": [float(f"{x:.3e}") for x in ls],
            "least_squares_monotone": all(b <= a for a, b in zip([1.0] + ls, ls))}
    return rep


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(ms: float, sweeps: float, ws: int):
    """Whole-job figures of N replicas: the slowest rank's timed region and the sweeps of all ranks
    (each rank relaxes its own copy of the workload; the only exchange is this timing reduction)."""
    if ws <= 1:
        return ms, sweeps
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([ms, float(sweeps)], dtype=torch.float64, device=dev)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm_ = tt.clone()
    dist.all_reduce(sm_, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm_[1])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cycle_name(w) -> str:
    """V(nu1,nu2) of the finest level, with the Galerkin levels' shape when it differs."""
    s = f"V({w.nu1},{w.nu2})"
    if getattr(w, "coarse_nu", None) is not None:
        s += f", Galerkin levels ({w.coarse_nu[0]},{w.coarse_nu[1]})"
    return s


def hbm_peak():
    """Measured copy bandwidth (GB/s) from MEASURED_PEAKS.json beside this file, else the fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, TypeError, ValueError):
        return 6800.0, "of fallback (6.8 TB/s)"


def finest_factor_store(w, precision):
    """(subvolumes, bytes per subvolume factor) of the finest level, in the library's layout: packed
    lower-triangular 16 x 16 blocks of the padded size (least squares), or the dense padded LU
    (square local form); complex128 entries in FP64, complex64 in the mixed path."""
    nsub, pts = 1, 1
    for a in range(w.dim):
        nsub *= -(-w.n[a] // w.sub[a])
        pts *= w.sub[a]
    npad = next(s_ for s_ in (16, 32, 48, 64, 96, 128, 192, 256) if pts * w.nt <= s_)
    entry = 16 if precision == 0 else 8
    if getattr(w, "local_form", "lsq") == "square":
        return nsub, npad * npad * entry
    nb = npad // 16
    return nsub, nb * (nb + 1) // 2 * 256 * entry


def l2_note(w, precision):
    """How the timed steps stand to the L2: either the factor store that every sweep streams (rewritten
    each step) is larger than L2, or the whole working set fits and nothing is flushed."""
    nsub, per = finest_factor_store(w, precision)
    store, vec = nsub * per, w.nunknowns * 16
    if store > L2_BYTES:
        return (f"inputs ({vec / 1e6:.3g} MB per coefficient vector) {'larger' if vec > L2_BYTES else 'smaller'} "
                f"than L2; each step rewrites the {store / 1e6:.0f} MB finest-level factor store (> L2), "
                f"which every sweep streams")
    return (f"working set (coefficient vectors {vec / 1e6:.3g} MB, factors {store / 1e6:.3g} MB) fits in "
            f"L2; not flushed between steps")


def workload_config(w, precision, ws):
    """The "config" object of a bench line; the reference arm prints the same one."""
    return {"workload": w.name, "grid": list(w.shape), "K": w.nt, "subvolume": list(w.sub[:w.dim]),
            "levels": w.levels, "cycle": cycle_name(w), "coarse_sweeps": w.coarse_sweeps,
            "tol_rel_action": w.tol, "precision": precision, "trial": w.trial,
            "local_form": getattr(w, "local_form", "lsq"),
            "parallelism": "replicas" if ws > 1 else "single",
            "l2": l2_note(w, precision)}


def default_precision(name: str) -> int:
    """The arithmetic a workload is specified in: the 3D workload runs FP64 with complex64 local solves."""
    return 1 if name in ("3d", "3d-small", "3d-mid") else 0


def dominant_roofline(prof, w, precision, ms_total, traffic_ok, peaks=None):
    """Roofline of the dominant kernel class (the larger total device time of factor and sweep).
    peaks: (FP64, FP32) TFLOP/s measured in this run by la_fma_peaks, else the derived figures."""
    fac_ms = prof["ms_factor"] / max(prof["n_factor"], 1)
    swp_ms_full = prof["ms_sweep"] / max(prof["n_sweep"], 1)   # one event pair per full sweep
    nsub, fbytes = finest_factor_store(w, precision)
    wide = fbytes // (16 if precision == 0 else 8) > 136 * 128   # more than 128 unknowns: global-memory factor
    fac_name = "k_factor_wide" if wide else ("k_factor" if precision == 0 else "k_factor_blk")
    if prof["ms_factor"] >= prof["ms_sweep"]:
        dom, flops, dms, cls = f"{fac_name} (finest level)", prof["flops_factor"], fac_ms, "factor"
    else:
        dom, flops, dms, cls = "k_sweep_fine (one sweep, all colours)", prof["flops_sweep"], swp_ms_full, "sweep"
    bps = NCU_BYTES_PER_SUBVOLUME.get((cls + ("_wide" if wide else ""), precision)) if traffic_ok else None
    traffic = round(bps * nsub) if bps else None
    kms = {"factor_per_launch": round(fac_ms, 4), "sweep_full": round(swp_ms_full, 4),
           "factor_share": round(prof["ms_factor"] / max(ms_total, 1e-9), 3),
           "sweep_share": round(prof["ms_sweep"] / max(ms_total, 1e-9), 3)}
    tnote = ("DRAM read+write bytes of this kernel per launch: one ncu capture of the same kernel at 128^3 (a "
             "factorisation launch; a full sweep of eight colour launches), per subvolume times the subvolumes "
             "of a launch" if wide else
             "DRAM read+write bytes of this kernel per launch from one ncu capture of this workload")
    if precision == 1 and cls == "sweep":
        # the complex64 sweep streams the factor store: HBM roofline on its compulsory bytes, every
        # factor once plus c read and written, f read (8 B per complex64) and V0 read per point
        nunk = w.nunknowns
        algo = nsub * fbytes + nunk * 8 * 3 + w.npoints * 8
        gbs = algo / (dms * 1e-3) / 1e9
        peak, note = hbm_peak()
        return {"bound": "hbm", "kernel": dom, "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "traffic": traffic, "algorithmic_bytes": algo,
                "traffic_note": tnote, "peak_note": note, "kernel_ms": kms}
    achieved = flops / (dms * 1e-3) / 1e12
    if peaks is not None:
        peak = peaks[0] if precision == 0 else peaks[1]
        peak_note = (f"{'FP64' if precision == 0 else 'FP32'} FMA pipe of measured (la_fma_peaks in this run: "
                     f"{peaks[2]} SMs)")
    elif precision == 0:
        peak = FP64_PEAK_TFLOPS
        peak_note = "FP64 pipe: 152 SMs x 4 flop/clk x 2070 MHz (derived)"
    else:
        peak = FP32_PEAK_TFLOPS
        peak_note = "FP32 pipe (complex64 kernel): 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"
    return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4), "peak": round(peak, 4),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "algorithmic_flops": flops, "traffic_note": tnote, "peak_note": peak_note, "kernel_ms": kms}


def stencil_roofline(prof, precision, c64=False):
    """Finest-level action-residual stencil against HBM: algorithmic bytes / event time.  c64: the
    complex64 V-cycle residual of the mixed path (TMA-staged kernel on 2D/3D grids); else the FP64
    residual (S1, action norm and FP64 V-cycle)."""
    n, ms, by = (("n_resid32", "ms_resid32", "bytes_resid32") if c64 else ("n_resid", "ms_resid", "bytes_resid"))
    if not prof.get(n):
        return None
    peak, note = hbm_peak()
    gbs = prof[by] / (prof[ms] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": ("k_stencil_tma / k_mresid complex64 (V-cycle residual)" if c64 else
                                       "k_mresid FP64 (action residual, S1)"),
            "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "peak_note": note,
            "launches": prof[n], "us_per_launch": round(1e3 * prof[ms] / prof[n], 2),
            "note": ("bound by the FP64 pipe, not by HBM" if not c64 else
                     "algorithmic bytes: f, c, V0 in and z out per point")}


def transfer_roofline(prof):
    """The finest-level transfers (Sec. III: restriction of the normal residual to level 1, prolongation
    of level 1's correction added to the finest one) against HBM: algorithmic bytes / event time."""
    if not prof.get("n_restrict"):
        return None
    peak, note = hbm_peak()
    out = {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_note": note}
    for name, n, ms, by in (("restrict", "n_restrict", "ms_restrict", "bytes_restrict"),
                            ("prolong_add", "n_prolong", "ms_prolong", "bytes_prolong")):
        if prof.get(n):
            gbs = prof[by] / (prof[ms] * 1e-3) / 1e9
            out[name] = {"kernel": f"k_{name}", "achieved": round(gbs, 1), "frac": round(gbs / peak, 4),
                         "launches": prof[n], "us_per_launch": round(1e3 * prof[ms] / prof[n], 2)}
    return out


def make_context(B, torch, w, precision, **overrides):
    ctx = B.Context(B.config_from_workload(w, precision=precision, **overrides))
    ctx.set_hamiltonian(torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda"), w.pulse)
    return ctx


def timed_steps(torch, ctx, psi, w, t, steps, snapshots=()):
    """`steps` least-action steps from time t, timed with CUDA events on the current stream (one la_step
    call per step, so that per-step statistics and snapshots are available).  Returns
    (ms, per-step stats, t after, {step index: psi copy})."""
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats, snaps = [], {}
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(steps):
        st, s1 = ctx.step(psi, 1, t, stats=True)
        stats.append(s1[0])
        t += w.dt
        if k + 1 in snapshots:
            snaps[k + 1] = psi.clone()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), stats, t, snaps


def rel_l2(a, b) -> float:
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def subrecord_fp64_same_config(B, torch, w, psi_mixed, steps_mixed, ms_mixed):
    """The headline problem in plain FP64: time per step, and the mixed path's speed-up at the same
    tolerance, with the two propagations' states compared after the same steps from psi0."""
    ctx = make_context(B, torch, w, 0)
    psi = torch.from_numpy(wl.initial_state(w).ravel()).cuda()
    warm = 2
    t = 0.0
    for _ in range(warm):
        ctx.step(psi, 1, t)
        t += w.dt
    steps = 3
    clk = ClockSampler(0)
    clk.start()
    ms, stats, t, _ = timed_steps(torch, ctx, psi, w, t, steps)
    clocks = clk.stop()
    ctx.close()
    ms_step = ms / steps
    diff = rel_l2(psi_mixed, psi) if psi_mixed is not None and steps_mixed == warm + steps else None
    return {"what": f"{w.name} in FP64 throughout (complex128 factors and V-cycles)", "steps": steps,
            "warmup": warm, "ms_per_step": ms_step, "cycles_per_step": sum(s[0] for s in stats) / steps,
            "max_rel_action": max(s[3] for s in stats),
            "value": w.nunknowns * sum(s[1] for s in stats) / (ms * 1e-3), "unit": "unknowns/s",
            "mixed_speedup_at_same_tolerance": ms_step / ms_mixed,
            "psi_rel_l2_mixed_vs_fp64_after_5_steps": diff, "clocks": clocks}


def subrecord_2d_propagation(B, torch):
    """The 2D workload's whole 200-step propagation from t = 0 in FP64 and in mixed precision (each
    after 3 warm-up steps on the same context), with the mixed path's speed-up at the same tolerance
    and the two final states compared."""
    w = workload("2d")
    out, final = {}, {}
    for precision in (0, 1):
        ctx = make_context(B, torch, w, precision)
        psi0 = torch.from_numpy(wl.initial_state(w).ravel()).cuda()
        psi = psi0.clone()
        t = 0.0
        for _ in range(3):
            ctx.step(psi, 1, t)
            t += w.dt
        psi.copy_(psi0)   # t0 = 0 again: the trial history restarts with the propagation
        clk = ClockSampler(0)
        clk.start()
        ms, stats, _, _ = timed_steps(torch, ctx, psi, w, 0.0, w.nsteps)
        clocks = clk.stop()
        ctx.close()
        final[precision] = psi
        cyc = [s[0] for s in stats]
        out["fp64" if precision == 0 else "mixed"] = {
            "steps": w.nsteps, "ms_total": ms, "ms_per_step": ms / w.nsteps,
            "value": w.nunknowns * sum(s[1] for s in stats) / (ms * 1e-3), "unit": "unknowns/s",
            "cycles_per_step_mean": sum(cyc) / len(cyc), "cycles_per_step_max": max(cyc),
            "max_rel_action": max(s[3] for s in stats), "clocks": clocks}
    out["mixed_speedup_at_same_tolerance"] = out["fp64"]["ms_total"] / out["mixed"]["ms_total"]
    out["final_psi_rel_l2_mixed_vs_fp64"] = rel_l2(final[1], final[0])
    out["what"] = (f"{w.name}: {w.nsteps} steps from t = 0 (the field 0.05 sin(0.057 t) grows from 0 to "
                   f"{0.05 * abs(np.sin(0.057 * w.nsteps * w.dt)):.3f}), tolerance {w.tol} every step")
    return out


def batched_members(n, precision_trial=3):
    return [dataclasses.replace(wl.batched_2d(i), trial=precision_trial) for i in range(n)]


def batched_measure(B, torch, ws, precision, steps, warmup):
    """la_step_batch over all members against the same contexts stepped one after another."""
    ctxs = [make_context(B, torch, w, precision) for w in ws]
    psis = [torch.from_numpy(wl.initial_state(w).ravel()).cuda() for w in ws]
    t0s = [0.0] * len(ws)
    if warmup:
        B.step_batch(ctxs, psis, warmup, t0s)
    t0s = [warmup * w.dt for w in ws]
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    a = time.perf_counter()
    stats = B.step_batch(ctxs, psis, steps, t0s)
    torch.cuda.synchronize()
    el = time.perf_counter() - a
    clocks = clk.stop()
    work = sum(w.nunknowns * sum(s[1] for s in st) for w, st in zip(ws, stats))
    t1s = [t + steps * w.dt for t, w in zip(t0s, ws)]
    torch.cuda.synchronize()
    a = time.perf_counter()
    work_seq = 0
    for ctx, psi, w, t in zip(ctxs, psis, ws, t1s):
        st, sts = ctx.step(psi, steps, t, stats=True)
        work_seq += w.nunknowns * sum(x[1] for x in sts)
    torch.cuda.synchronize()
    el_seq = time.perf_counter() - a
    for c in ctxs:
        c.close()
    return {"value": work / el, "ms_per_step": 1e3 * el / steps, "unit": "unknowns/s",
            "sequential": {"value": work_seq / el_seq, "ms_per_step": 1e3 * el_seq / steps},
            "speedup_vs_sequential": (work / el) / (work_seq / el_seq),
            "max_rel_action": max(s[3] for st in stats for s in st),
            "cycles_per_step_mean": sum(s[0] for st in stats for s in st) / max(1, sum(len(st) for st in stats)),
            "clocks": clocks}


def subrecord_batched(B, torch, nbatch=512, steps=3, warmup=1):
    """The batched workload (512 seeded grids of 64^2 .. 256^2, K = 4) in FP64 and in mixed precision,
    schedule autotuned on a 128^2 member."""
    from paper_1111_4363_gb300 import autotune
    members = batched_members(nbatch)
    rep = dataclasses.replace(members[0], n=(128, 128, 1))
    out = {"members": nbatch, "unknowns_total": sum(w.nunknowns for w in members), "steps": steps,
           "warmup": warmup}
    for precision in (0, 1):
        best = autotune.tune(rep, precision=precision)
        ws = [dataclasses.replace(m, **best) for m in members]
        r = batched_measure(B, torch, ws, precision, steps, warmup)
        r["autotuned"] = {k: list(v) if isinstance(v, tuple) else v for k, v in best.items()}
        out["fp64" if precision == 0 else "mixed"] = r
    out["mixed_speedup_over_fp64_batched"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import binding as B

    precision = args.precision if args.precision >= 0 else default_precision(args.workload)
    w = workload(args.workload)
    if args.trial >= 0:
        w = dataclasses.replace(w, trial=args.trial)
    peaks = B.fma_peaks()
    ctx = make_context(B, torch, w, precision)
    psi0 = torch.from_numpy(wl.initial_state(w).ravel()).cuda()
    psi = psi0.clone()
    nunk = w.nunknowns
    # warm-up steps (untimed); the propagation continues from where warm-up ended
    t = 0.0
    snap_mixed = None
    for k in range(args.warmup):
        ctx.step(psi, 1, t)
        t += w.dt
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    want = (5 - args.warmup,) if 0 < 5 - args.warmup <= args.steps else ()
    ms, stats, t, snaps = timed_steps(torch, ctx, psi, w, t, args.steps, snapshots=want)
    if want:
        snap_mixed = snaps[want[0]]
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    sweeps = sum(s[1] for s in stats)
    cycles = [s[0] for s in stats]
    ms_max, sweeps_all = reduce_over_ranks(ms, sweeps, ws)
    value = nunk * sweeps_all / (ms_max * 1e-3)

    # end to end through the public call with host buffers: pinned psi copied in and out every step
    psi_host = torch.empty(w.npoints, dtype=torch.complex128, pin_memory=True)
    psi_host.copy_(psi.cpu())
    e2e_steps = max(1, min(args.steps, 5))
    e2e_sweeps = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st, s1 = ctx.step(psi_host, 1, t, stats=True)
        e2e_sweeps += s1[0][1]
        t += w.dt
    e2e_s = time.perf_counter() - t0
    e2e_value = nunk * e2e_sweeps / e2e_s * (ws if ws > 1 else 1)
    ctx.close()

    roofline = dominant_roofline(prof, w, precision, ms, traffic_ok=args.workload in ("2d", "3d"), peaks=peaks)
    if getattr(w, "local_form", "lsq") == "square":
        roofline["kernel"] = roofline["kernel"].replace("k_factor", "k_factor_square").replace("k_sweep_fine",
                                                                                               "k_sweep_square")
    prec_tag = "f64" if precision == 0 else "c64 local solves + f64 refinement"

    out = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": prec_tag, "data": "synthetic",
           "config": workload_config(w, precision, ws),
           "cycles_per_step": sum(cycles) / args.steps, "cycles_per_step_max": max(cycles),
           "fine_sweeps_per_step": sweeps / args.steps, "max_rel_action": max(s[3] for s in stats),
           "ms_per_time_step_to_tol": ms_max / args.steps,
           "e2e": {"value": e2e_value, "unit": "unknowns/s", "h2d_bytes_per_step": 16 * w.npoints,
                   "d2h_bytes_per_step": 16 * w.npoints, "steps": e2e_steps},
           "gpu_launches": int(prof["launches"]), "roofline": roofline,
           "stencil_roofline": stencil_roofline(prof, precision),
           "stencil_roofline_c64": stencil_roofline(prof, precision, c64=True),
           "transfer_roofline": transfer_roofline(prof), "clocks": clk,
           "peaks": {"fp64_tflops": round(peaks[0], 4), "fp32_tflops": round(peaks[1], 3), "sm_count": peaks[2],
                     "how": "la_fma_peaks: 8 independent FMA chains per thread, one full wave of 256-thread CTAs on every SM, "
                            "CUDA events, in this run"}}
    extras = rank == 0 and ws == 1 and not args.headline_only
    if extras and args.workload == "3d" and precision == 1:
        out["fp64_same_config"] = subrecord_fp64_same_config(B, torch, w, snap_mixed,
                                                             args.warmup + (want[0] if want else 0),
                                                             ms_max / args.steps)
    if extras and args.workload == "3d":
        out["config_2d_200_steps"] = subrecord_2d_propagation(B, torch)
        out["config_batched_512"] = subrecord_batched(B, torch)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and getattr(w, "local_form", "lsq") == "lsq":
        out["cpu_baseline"] = cpu_baseline(w)
    if rank == 0 and getattr(w, "local_form", "lsq") == "square":
        out["square_form"] = square_form_report(B, torch, w)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def oracle_cycle_rate(w: wl.Workload, budget_s: float):
    """Time the CPU oracle on the workload: one step's setup, then V-cycles until ``budget_s`` is used."""
    from oracle import multigrid, system
    from oracle.propagate import numpy_coarse_nu, numpy_coarse_sub, numpy_sub
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    t_a = time.perf_counter()
    M, f, W = system.assemble(prob, 0.0, psi0, w.weight)
    G0 = (M.conj().T @ W @ M).tocsr()
    g0 = M.conj().T @ (W @ f)
    hier = multigrid.Hierarchy(G0, prob.shape, prob.K, numpy_sub(w), w.levels, w.nu1, w.nu2, w.coarse_sweeps,
                                     numpy_coarse_sub(w), numpy_coarse_nu(w))
    setup_s = time.perf_counter() - t_a
    c = np.zeros(M.shape[1], dtype=np.complex128)
    ncyc = 0
    t_b = time.perf_counter()
    while True:
        hier.vcycle(0, c, g0)
        system.action_norm(system.residual(M, f, c), W)
        ncyc += 1
        if time.perf_counter() - t_b > budget_s:
            break
    cyc_s = (time.perf_counter() - t_b) / ncyc
    return setup_s, cyc_s, ncyc


# The oracle is plain NumPy/SciPy: sparse products and 96 x 96 dense Cholesky solves, which run on one
# thread (limiting BLAS to one thread does not change its time), so it uses one core of the host.
ORACLE_THREADS = 1


def oracle_sample(w: wl.Workload):
    """The workload itself when the oracle handles it in seconds, else the same problem on a 32^3 grid
    (3D): the oracle's time per unknown and sweep does not depend on the grid size (measured 2.9e5 and
    2.7e5 unknowns relaxed/s at 16^3 and 32^3), so the rate extrapolates to the full grid."""
    if w.dim == 3 and w.npoints > 32 ** 3:
        return dataclasses.replace(w, n=(32, 32, 32)), True
    return w, False


def cpu_baseline(w: wl.Workload):
    ws_, extrap = oracle_sample(w)
    setup_s, cyc_s, ncyc = oracle_cycle_rate(ws_, 8.0)
    sweeps = ws_.nu1 + ws_.nu2
    value = ws_.nunknowns * sweeps / cyc_s
    where = (f"the same problem on {'x'.join(map(str, ws_.shape))} points, per unknown extrapolated to "
             f"{'x'.join(map(str, w.shape))}") if extrap else f"{w.name}"
    return {"value": value, "unit": "unknowns/s", "cores": ORACLE_THREADS, "kind": "oracle",
            "host_cores": len(os.sched_getaffinity(0)), "extrapolated": extrap,
            "sample": f"one time step of {where}: setup (assembly, Galerkin levels, block Cholesky) "
                      f"{setup_s:.1f} s excluded, then {ncyc} V-cycles timed ({cyc_s:.2f} s each)",
            "setup_s": setup_s, "cycle_s": cyc_s}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    w_full = workload(args.workload)
    precision = args.precision if args.precision >= 0 else default_precision(args.workload)
    w, extrap = oracle_sample(w_full)
    cores = ORACLE_THREADS
    # each step = one oracle V-cycle on the workload (a 32^3 sample of the 3D one) after an untimed
    # setup; bounded to a few minutes
    from oracle import multigrid, system
    from oracle.propagate import numpy_coarse_nu, numpy_coarse_sub, numpy_sub
    prob = system.Problem.from_workload(w)
    psi0 = wl.initial_state(w).ravel()
    t_a = time.perf_counter()
    M, f, W = system.assemble(prob, 0.0, psi0, w.weight)
    G0 = (M.conj().T @ W @ M).tocsr()
    g0 = M.conj().T @ (W @ f)
    hier = multigrid.Hierarchy(G0, prob.shape, prob.K, numpy_sub(w), w.levels, w.nu1, w.nu2, w.coarse_sweeps,
                                     numpy_coarse_sub(w), numpy_coarse_nu(w))
    setup_s = time.perf_counter() - t_a
    c = np.zeros(M.shape[1], dtype=np.complex128)
    # the requested counts, capped so that the run stays within a few minutes (about 1-2 s per
    # V-cycle of the 256^2 workload or of the 32^3 sample on one host core)
    warm = max(0, min(args.warmup, 5))
    for _ in range(warm):
        hier.vcycle(0, c, g0)
    steps = max(1, min(args.steps, 60))
    t0 = time.perf_counter()
    for _ in range(steps):
        hier.vcycle(0, c, g0)
        system.action_norm(system.residual(M, f, c), W)
    el = time.perf_counter() - t0
    sweeps = w.nu1 + w.nu2
    value = w.nunknowns * sweeps * steps / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": ws,
           "steps": steps, "warmup": warm, "ms_per_step": el / steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(w_full, precision, ws),
           "reference_step": (f"one oracle V-cycle ({sweeps} finest-level sweeps, FP64) of "
                              + (f"the same problem on {'x'.join(map(str, w.shape))} points (rate per unknown "
                                 f"extrapolated to the full grid)" if extrap else "the workload")
                              + " on the host, from the same schedule; host memory, no L2 flush"),
           "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": cores, "kind": "oracle",
                            "extrapolated": extrap,
                            "sample": f"{steps} V-cycles of {w.name} on {'x'.join(map(str, w.shape))} points "
                                      f"after an untimed setup of {setup_s:.1f} s"},
           "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batched(args):
    """512 independent 2D propagations of uneven size (64^2 .. 256^2, K = 4): la_step_batch vs stepping
    the same contexts one after another, at the same tolerance.  The schedule is autotuned on a
    128 x 128 member."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import autotune
    from paper_1111_4363_gb300 import binding as B
    precision = args.precision if args.precision >= 0 else 0
    members = [dataclasses.replace(wl.batched_2d(i), trial=3 if args.trial < 0 else args.trial)
               for i in range(args.batch)]
    rep = dataclasses.replace(members[0], n=(128, 128, 1))
    best = autotune.tune(rep, precision=precision)
    ws = [dataclasses.replace(m, **best) for m in members]
    ctxs, psis = [], []
    for w in ws:
        ctx = B.Context(B.config_from_workload(w, precision=precision))
        ctx.set_hamiltonian(torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda"), w.pulse)
        ctxs.append(ctx)
        psis.append(torch.from_numpy(wl.initial_state(w).ravel()).cuda())
    t0s = [0.0] * len(ws)
    B.step_batch(ctxs, psis, args.warmup, t0s)
    t0s = [args.warmup * w.dt for w in ws]
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    a = time.perf_counter()
    stats = B.step_batch(ctxs, psis, args.steps, t0s)
    torch.cuda.synchronize()
    el = time.perf_counter() - a
    clk = clocks.stop()
    work = sum(w.nunknowns * sum(s[1] for s in st) for w, st in zip(ws, stats))
    value = work / el
    # the same contexts stepped one after another (plain per-context la_step), same number of steps
    t1s = [t + args.steps * w.dt for t, w in zip(t0s, ws)]
    torch.cuda.synchronize()
    a = time.perf_counter()
    work_seq = 0
    for ctx, psi, w, t in zip(ctxs, psis, ws, t1s):
        st, sts = ctx.step(psi, args.steps, t, stats=True)
        work_seq += w.nunknowns * sum(x[1] for x in sts)
    torch.cuda.synchronize()
    el_seq = time.perf_counter() - a
    value_seq = work_seq / el_seq
    out = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == 0 else "c64 local solves + f64 refinement",
           "data": "synthetic",
           "config": {"workload": f"2d_batched_{args.batch}_K4", "members": args.batch,
                      "grids": "seeded n in {64, 80, ..., 256}", "unknowns_total": sum(w.nunknowns for w in ws),
                      "autotuned": best, "tol_rel_action": ws[0].tol, "precision": precision},
           "sequential": {"value": value_seq, "ms_per_step": 1e3 * el_seq / args.steps},
           "speedup_vs_sequential": value / value_seq,
           "max_rel_action": max(s[3] for st in stats for s in st), "clocks": clk}
    print(json.dumps(out))


def run_3d_adjoint(args):
    """3D hydrogen in a 32-component pulse (128^3, K = 4, 4x4x4 subvolumes): forward propagation with
    checkpoints every 20 steps, then the gradient of the final dipole w.r.t. the 32 amplitudes."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import binding as B
    precision = args.precision if args.precision >= 0 else 1
    n = args.n3d
    w = dataclasses.replace(wl.hydrogen_3d(n=n, nsteps=args.steps), **PRODUCTION_3D)
    if args.trial >= 0:
        w = dataclasses.replace(w, trial=args.trial)
    # checkpoints every 20 steps; the backward pass keeps a recomputed segment's factors on the
    # device (20 steps x all levels: ~74 GB FP64, ~37 GB complex64) instead of factorising again
    cfg = B.config_from_workload(w, precision=precision, ckpt_every=20, cache_factors=1)
    ctx = B.Context(cfg)
    V0 = torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    a = time.perf_counter()
    ctx.set_hamiltonian(V0, w.pulse)    # builds the Galerkin stencils of every coarse level
    setup_s = time.perf_counter() - a
    psi = torch.from_numpy(wl.initial_state(w).ravel()).cuda()
    ctx.profile_enable(True)
    torch.cuda.synchronize()
    clk_f = ClockSampler(0)
    clk_f.start()
    a = time.perf_counter()
    st, stats = ctx.step(psi, args.steps, 0.0, stats=True)
    torch.cuda.synchronize()
    el_f = time.perf_counter() - a
    clocks_f = clk_f.stop()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    x = torch.from_numpy(wl.laser_coordinate(w).ravel()).cuda()
    hd = float(np.prod(w.h[:3]))
    dJ = (hd * x * psi).contiguous()
    clk_b = ClockSampler(0)
    clk_b.start()
    a = time.perf_counter()
    grad = ctx.backward(dJ, w.pulse.ncomp)
    torch.cuda.synchronize()
    el_b = time.perf_counter() - a
    clocks_b = clk_b.stop()
    sweeps = sum(s_[1] for s_ in stats)
    out = {"metric": METRIC, "value": w.nunknowns * sweeps / el_f, "unit": "unknowns/s", "n_gpus": 1,
           "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * el_f / args.steps, "higher_is_better": True,
           "dtype": "f64" if precision == 0 else "c64 local solves + f64 refinement", "data": "synthetic",
           "config": {"workload": w.name, "grid": list(w.shape), "K": w.nt, "subvolume": list(w.sub),
                      "levels": w.levels, "cycle": cycle_name(w), "trial": w.trial,
                      "pulse_components": w.pulse.ncomp, "ckpt_every": 20, "cache_factors": True,
                      "l2": l2_note(w, precision)},
           "cycles_per_step": sum(s_[0] for s_ in stats) / args.steps,
           "backward_ms_per_step": 1e3 * el_b / args.steps, "set_hamiltonian_s": setup_s,
           "roofline": dominant_roofline(prof, w, precision, 1e3 * el_f, traffic_ok=False),
           "stencil_roofline": stencil_roofline(prof, precision),
           "stencil_roofline_c64": stencil_roofline(prof, precision, c64=True),
           "dipole_T": float(hd * (x * psi.abs() ** 2).sum()), "grad_norm": float(np.linalg.norm(grad)),
           "grad_head": [float(g) for g in grad[:4]], "clocks": clocks_f, "clocks_backward": clocks_b}
    print(json.dumps(out))


LFA_SIZES = (3, 4, 6, 8)
LFA_KAPPA_NU = [(0.0, 0.0), (0.1, 0.0), (1.0, 0.0), (10.0, 0.0), (0.0, 1.0), (0.0, -1.0), (1.0, 1.0), (1.0, -1.0)]


def run_lfa(args):
    """The paper's plane-wave experiment (Sec. V) in its Legendre-element basis: log10 ratios of the
    residual norm and of |S| after one relaxation, for the 8 (kappa, nu) pairs of the paper's figures,
    Nx = Nt in LFA_SIZES, one element, two elements at once and two through the parent-element transfer,
    on a 256 x 256 (w, k) grid over [-8, 8]^2 (no point at k = w = 0, where N or S of the trial vanishes
    for nu = 0).  value: relaxation evaluations (case x grid point) per second of la_lfa_maps with the maps
    left on the device."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import binding as B
    ng = 256
    ks = np.linspace(-8.0, 8.0, ng)
    ws = np.linspace(-8.0, 8.0, ng)
    methods = ("one", "two", "transfer")
    cases = [(m, s_, s_, kappa, nu) for m in methods for s_ in LFA_SIZES for kappa, nu in LFA_KAPPA_NU]
    out = torch.empty((len(cases), 2, ng, ng), dtype=torch.float64, device="cuda")
    for _ in range(max(args.warmup, 1)):
        B.lfa_maps(cases, ks, ws, out=out)
    torch.cuda.synchronize()
    reps = max(1, min(args.steps, 5))
    clk = ClockSampler(0)
    clk.start()
    a = time.perf_counter()
    for _ in range(reps):
        B.lfa_maps(cases, ks, ws, out=out)
    torch.cuda.synchronize()
    el = (time.perf_counter() - a) / reps
    clocks = clk.stop()
    host = np.empty((len(cases), 2, ng, ng))
    a = time.perf_counter()
    B.lfa_maps(cases, ks, ws, out=host)
    el_e2e = time.perf_counter() - a
    maps = out.cpu().numpy()
    summary = {}
    for m in methods:
        for s_ in LFA_SIZES:
            idx = [c for c, cs in enumerate(cases) if cs[0] == m and cs[1] == s_]
            N = maps[idx, 0]
            summary[f"{m}_{s_}x{s_}"] = {
                "median_log10_N_ratio": round(float(np.median(N)), 3),
                "fraction_N_ratio_above_1": round(float(np.mean(N > 0)), 4),
                "median_log10_S_ratio": round(float(np.median(maps[idx, 1])), 3),
                "fraction_N_ratio_above_1_per_pair": [round(float(np.mean(maps[c, 0] > 0)), 4) for c in idx]}
    evals = len(cases) * ng * ng
    res = {"metric": "relaxation evaluations/s", "value": evals / el, "unit": "evaluations/s", "n_gpus": 1,
           "steps": reps, "warmup": max(args.warmup, 1), "ms_per_step": 1e3 * el, "higher_is_better": True,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "legendre_element_maps", "grid": [ng, ng], "k_range": [-8, 8],
                      "w_range": [-8, 8], "sizes": list(LFA_SIZES), "methods": list(methods),
                      "kappa_nu": LFA_KAPPA_NU, "cases": len(cases)},
           "e2e": {"value": evals / el_e2e, "unit": "evaluations/s", "h2d_bytes_per_step": 16 * ng,
                   "d2h_bytes_per_step": 8 * evals * 2},
           "summary": summary, "clocks": clocks}
    if not args.no_cpu_baseline:
        from oracle import lfa
        sub = np.linspace(-8.0, 8.0, 6)
        a = time.perf_counter()
        lfa.ratio_map("two", 6, 6, 1.0, 0.0, sub, sub)
        dt_o = time.perf_counter() - a
        res["cpu_baseline"] = {"value": sub.size ** 2 / dt_o, "unit": "evaluations/s", "cores": 1,
                               "kind": "oracle", "sample": "two elements, Nx = Nt = 6, kappa 1, nu 0, 6 x 6 points"}
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d",
                    choices=["3d", "3d-small", "3d-mid", "2d", "2d-small", "1d", "2d-square", "batched", "3d-adjoint", "lfa"])
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--n3d", type=int, default=128)
    ap.add_argument("--precision", type=int, default=-1, choices=[-1, 0, 1],
                    help="0 FP64, 1 complex64 local solves with FP64 refinement; -1: the workload's own "
                         "(1 for the 3D workload, 0 otherwise)")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline measurement (no sub-records), e.g. under ncu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trial", type=int, default=-1, choices=[-1, 0, 1, 2, 3],
                    help="trial iterate of each step (extrapolation order + 1); -1: the workload's setting")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "3d-adjoint":
        run_3d_adjoint(args)
    elif args.workload == "lfa":
        run_lfa(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
