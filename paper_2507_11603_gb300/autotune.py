"""Launch-shape autotuner for the persistent photon loops and the served rounds.

The photon loops are persistent kernels whose throughput depends on the block size,
the number of resident blocks per SM (register pressure versus latency hiding) and,
for served rounds, the number of events a lane runs per launch.  ``tune_run`` times a
short representative run for each candidate shape through the C ABI and keeps the
fastest; ``tune_server`` does the same for ``events_per_round`` on a small burst of
requests.  ``tune_modes`` times the execution modes that change no result -- for a grid,
the one-kernel loop against the event-based loop with a few slot counts; for a shell, the
lanes that run pipelined events and core bursts -- and keeps the fastest.  Results are
cached per device name and workload key in a JSON file next to the built library.
"""
from __future__ import annotations

import json
import os
import time

from . import _build

CACHE = os.path.join(_build.BUILD, "autotune.json")
BLOCKS = (64, 128, 256)
PER_SM = (0, 1, 2, 4)


def _load():
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def _device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def tune_run(ctx, geom, key, n_photons=20000, repeats=2, candidates=None, **run_kw):
    """Pick (block_size, blocks_per_sm) for thor_run on `geom`; returns the best and sets it."""
    cache = _load()
    dk = f"{_device_name()}|{key}|{n_photons}"
    if dk in cache:
        best = cache[dk]
        ctx.set_launch(best["block"], best["blocks_per_sm"])
        return best
    cands = candidates or [(b, s) for b in BLOCKS for s in PER_SM]
    results = []
    for b, s in cands:
        ctx.set_launch(b, s)
        ctx.run(geom, n_photons=n_photons, seed=99, **run_kw)  # warm-up
        ms = []
        for r in range(repeats):
            res = ctx.run(geom, n_photons=n_photons, seed=100 + r, **run_kw)
            ms.append(res.stats["elapsed_ms"])
        results.append({"block": b, "blocks_per_sm": s, "ms": min(ms)})
    best = min(results, key=lambda t: t["ms"])
    best = dict(best, table=results)
    cache[dk] = best
    _save(cache)
    ctx.set_launch(best["block"], best["blocks_per_sm"])
    return best


def tune_server(ctx, requests, key, candidates=(32, 64, 128, 256, 512, 1024), **submit_kw):
    """Pick events_per_round for the served stream from the burst completion time of `requests`."""
    cache = _load()
    dk = f"{_device_name()}|server|{key}"
    if dk in cache:
        return cache[dk]
    results = []
    for e in candidates:
        srv = ctx.server(max_requests=max(8, len(requests)), events_per_round=e)
        t0 = time.perf_counter()
        tickets = [srv.submit(**r, **submit_kw) for r in requests]
        for t in tickets:
            srv.wait(t)
        results.append({"events_per_round": e, "s": time.perf_counter() - t0})
        srv.close()
    best = min(results, key=lambda t: t["s"])
    best = dict(best, table=results)
    cache[dk] = best
    _save(cache)
    return best


GRID_MODES = ((0, 0), (1 << 16, 1 << 13), (1 << 18, 1 << 15))  # (slots, handoff); 0 = one kernel
SHELL_MODES = ((32, 1), (32, 2), (32, 4), (8, 1))              # (pipe_lanes, burst_lanes)


def tune_modes(ctx, geom, key, n_photons=20000, repeats=2, candidates=None, grid=False, **run_kw):
    """Pick the execution mode of thor_run on `geom` (grid: thor_ctx_set_grid_exec; shell:
    thor_ctx_set_bursts) from timed runs; returns the best and sets it."""
    cache = _load()
    dk = f"{_device_name()}|mode|{key}|{n_photons}"
    cands = list(candidates or (GRID_MODES if grid else SHELL_MODES))

    def apply(c):
        if grid:
            ctx.set_grid_exec(*c)
        else:
            ctx.set_bursts(*c)

    if dk in cache:
        apply(tuple(cache[dk]["mode"]))
        return cache[dk]
    results = []
    for c in cands:
        apply(c)
        ctx.run(geom, n_photons=n_photons, seed=99, **run_kw)  # warm-up
        ms = min(ctx.run(geom, n_photons=n_photons, seed=100 + r, **run_kw).stats["elapsed_ms"]
                 for r in range(repeats))
        results.append({"mode": list(c), "ms": ms})
    best = min(results, key=lambda t: t["ms"])
    best = dict(best, table=results)
    cache[dk] = best
    _save(cache)
    apply(tuple(best["mode"]))
    return best
