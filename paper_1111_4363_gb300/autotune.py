"""Autotuner for the relaxation schedule and its launch shape: subvolume shape (2x2 up to 8x8 points,
at most 256 unknowns), levels, cycle shape V(nu1, nu2), the Galerkin levels' cycle shape, and the CTA
packing of the small-subvolume factorisations (several matrices per CTA or one).

Every candidate reaches the same tolerance on N/N(0) (the minimiser does not depend on the
schedule), so candidates are ranked by measured time per least-action step on the GPU (CUDA events,
the best of three repetitions).  The packing is tried on the three fastest schedules only.  The
colouring is not a free parameter: same-colour subvolumes must not interact through the radius-2
normal operator, which leaves the 2^d block-parity classes (a checkerboard is invalid).  Results
are cached in JSON next to the built library, keyed by grid, K, precision, weight and trial.
"""
from __future__ import annotations

import dataclasses
import json
import os
import time

from . import binding as B
from . import workloads as wl

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def candidates(w: wl.Workload):
    out = []
    subs = [(2, 2), (4, 2), (4, 4)]
    if w.nt * 32 <= 256:
        subs.append((8, 4))
    if w.nt * 64 <= 256:
        subs.append((8, 8))
    for sx, sy in subs:
        for levels in (1, 2, 3, 4):
            if any(w.n[a] % (1 << (levels - 1)) for a in range(w.dim)):
                continue
            # one level: nu1 + nu2 sweeps between action evaluations; with three or more levels the
            # Galerkin levels above the coarsest may take a lighter (1, 0) cycle
            shapes = ((1, 1, None), (1, 2, None)) if levels > 1 else ((1, 0, None), (1, 1, None), (2, 1, None))
            if levels > 2:
                shapes += ((1, 2, (1, 0)),)
            for nu1, nu2, cnu in shapes:
                out.append(dict(sub=(sx, sy, 1), coarse_sub=(2, 2, 1), levels=levels,
                                coarse_sweeps=1, nu1=nu1, nu2=nu2, coarse_nu=cnu))
    return out


def key(w: wl.Workload, precision: int) -> str:
    return f"{w.dim}:{'x'.join(map(str, w.n[:w.dim]))}:K{w.nt}:p{precision}:{w.weight}:t{w.trial}"


def measure(w: wl.Workload, precision: int, nsteps: int = 3, warmup: int = 3, reps: int = 3) -> dict:
    """Time per step (CUDA events on the current stream, best of `reps` runs of `nsteps` steps that
    continue the propagation after `warmup` steps)."""
    import torch
    cfg = B.config_from_workload(w, precision=precision)
    ctx = B.Context(cfg)
    ctx.set_hamiltonian(torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda"), w.pulse)
    psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
    t = 0.0
    for _ in range(warmup):
        ctx.step(psi, 1, t)
        t += w.dt
    best, cycles, rel = float("inf"), 0.0, 0.0
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st, stats = ctx.step(psi, nsteps, t, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t += nsteps * w.dt
        best = min(best, e0.elapsed_time(e1) / nsteps)
        cycles = max(cycles, sum(s[0] for s in stats) / nsteps)
        rel = max(rel, max(s[3] for s in stats))
    ctx.close()
    return {"ms_per_step": best, "cycles": cycles, "rel": rel}


def tune(w: wl.Workload, precision: int = 0, use_cache: bool = True, verbose: bool = False) -> dict:
    """Best schedule for workload ``w`` (a dict of Workload fields to replace)."""
    cache = {}
    if use_cache and os.path.exists(CACHE):
        with open(CACHE) as fh:
            cache = json.load(fh)
    k = key(w, precision)
    if use_cache and k in cache:
        # JSON holds the tuple-valued fields (subvolume shapes) as lists
        return {f: tuple(v) if isinstance(v, list) else v for f, v in cache[k]["best"].items()}
    results = []
    for cand in candidates(w):
        wc = dataclasses.replace(w, **cand)
        try:
            r = measure(wc, precision)
        except B.LeastActionError as e:
            if verbose:
                print("skip", cand, e)
            continue
        if r["rel"] <= w.tol:
            results.append((r["ms_per_step"], cand, r))
            if verbose:
                print(cand, r)
    if not results:
        raise RuntimeError(f"autotune: no candidate schedule reached N/N(0) <= {w.tol} for {k}")
    results.sort(key=lambda x: x[0])
    # CTA packing: one matrix per CTA instead of several, on the three fastest schedules
    for _, cand, _ in list(results[:3]):
        cg = dict(cand, factor_group=1)
        try:
            r = measure(dataclasses.replace(w, **cg), precision)
        except B.LeastActionError:
            continue
        if r["rel"] <= w.tol:
            results.append((r["ms_per_step"], cg, r))
    results.sort(key=lambda x: x[0])
    best = results[0][1]
    cache[k] = {"best": best, "table": [dict(c, **r) for _, c, r in results]}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as fh:
        json.dump(cache, fh, indent=1)
    return best
