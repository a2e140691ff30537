"""Benchmark: Lyman-alpha resonant scatterings per second on one GB300.

Workload (default): the expanding thin shell -- R_in/R_out = 0.9, N_HI = 1e20 cm^-2,
homologous outflow 200 km/s at R_out, T = 1e4 K, dust absorption tau_d = 0.5, central
source with a Gaussian line sigma = 50 km/s, 1e5 photons, dipole phase function,
escaped spectrum in 400 bins over +-1500 km/s.  One step = one full run of the photon
loop over all 1e5 photons (thor_run).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload forest]

Timing: CUDA events on the context's stream around each step, L2 flushed (256 MiB
write) before every step outside the events; K timed steps between barriers and
device synchronisation; value = total scatterings / summed step time.  `e2e` repeats
the measurement through the public call with host buffers (wall clock, host<->device
copies inside).  Under torchrun each rank runs its own photon-id range (weak scaling,
no collective in the timed region).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lyα scatterings/sec on 1 GB300 vs oracle; p50/p99 latency of shell-model stream"
SHELL = dict(R_in=0.9, N_HI=1e20, T=1e4, v_max=200.0, tau_dust=0.5, phase="dipole")
RUN = dict(sigma=50.0, n_bins=400, X_min=-1500.0, X_max=1500.0)
N_PHOTONS = 100_000
WORKLOAD = "expanding shell R_in/R_out=0.9 N_HI=1e20 v_max=200km/s T=1e4K tau_d=0.5 sigma=50km/s 1e5 photons"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU baseline
def oracle_sample(seconds=15.0, first_id=0, cap=100_000):
    """The FP64 oracle on the same workload: photons first_id, first_id+1, ... in chunks
    on all host cores until `seconds` passed; trapped photons stop at `cap` scatterings."""
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    t0 = time.perf_counter()
    n_done, n_scat, pid = 0, 0, first_id
    chunk = 4 * ncores
    while time.perf_counter() - t0 < seconds:
        r = oracle.run_shell(tau0=SHELL["N_HI"] * oracle.line_params(SHELL["T"])["sigma0"], T=SHELL["T"],
                             R_in=SHELL["R_in"], v_max=SHELL["v_max"], tau_dust=SHELL["tau_dust"], phase="dipole",
                             line="gauss", sigma=RUN["sigma"], n_photons=chunk, first_id=pid, seed=1,
                             n_bins=RUN["n_bins"], X_min=RUN["X_min"], X_max=RUN["X_max"], max_scat=cap,
                             n_threads=ncores)
        n_done += chunk
        pid += chunk
        n_scat += r["sum_scat"]
    dt = time.perf_counter() - t0
    return {"value": n_scat / dt, "unit": "scatterings/s", "cores": ncores, "kind": "oracle",
            "sample": f"{n_done} photons (ids {first_id}..{pid - 1}) of the same workload, "
                      f"{n_scat} scatterings in {dt:.1f} s, photons stopped at {cap} scatterings"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(seconds=2.0)
    t0 = time.perf_counter()
    tot, vals = 0.0, []
    for i in range(args.steps):
        s = oracle_sample(seconds=args.ref_seconds, first_id=100_000 + 4096 * i)
        vals.append(s["value"])
    dt = time.perf_counter() - t0
    v = float(np.mean(vals))
    cb = oracle_sample(seconds=2.0)
    cb["value"] = v
    cb["sample"] = f"{args.steps} steps of ~{args.ref_seconds:.0f} s oracle work each on this workload; " + cb["sample"]
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "scatterings/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": "scatterings/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ GPU arm
def run_shell_bench(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2507_11603_gb300 import thor
    ctx = thor.Context(local)
    if args.block:
        ctx.set_launch(args.block, args.blocks_per_sm)
    if args.pipe_lanes >= 0 or args.burst_lanes >= 0:
        ctx.set_bursts(args.pipe_lanes if args.pipe_lanes >= 0 else 32, args.burst_lanes if args.burst_lanes >= 0 else 1)
    if args.no_tail_share:
        ctx.set_tail_share(False)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    geom = ctx.shell(**SHELL)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    from paper_2507_11603_gb300 import sharding

    def step(i, device_out=True, raw=False):
        # step i: the i-th block of world x 1e5 photon ids, rank r takes its own 1e5 (weak scaling)
        first, n = sharding.photon_range(rank, world, N_PHOTONS, base=i * world * N_PHOTONS)
        with torch.cuda.stream(stream):  # device outputs are allocated and cleared on the run's stream
            return ctx.run(geom, n_photons=n, seed=1, first_id=first, device_out=device_out, raw=raw, **RUN)

    for i in range(args.warmup):
        step(i)
    # measured issue peaks of this device (FP32 FMA: one warp instruction per scheduler per
    # clock; MUFU ex2), the denominators of the roofline below
    peak_fma = ctx.issue_peak("fma")
    peak_mufu = ctx.issue_peak("mufu")
    torch.cuda.synchronize()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms, n_scat, launches = 0.0, 0, 0
    step_scat, longest = [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            # per-photon records (9 B per photon, on the device) give each step's longest photon
            r = step(args.warmup + i, raw=True)
            ev[i][1].record(stream)
            kern_ms += r.stats["elapsed_ms"]
            n_scat += r.stats["n_scat"]
            step_scat.append(r.stats["n_scat"])
            launches += int(r.stats["n_launches"])
            longest.append(r.raw_nscat)
        torch.cuda.synchronize()
    barrier(world)
    longest = [(int(t.max().item()), int(torch.argmax(t).item())) for t in longest]
    per_step_ms = [a.elapsed_time(b) for a, b in ev]
    step_ms = sum(per_step_ms)
    t_max = max_over_ranks(step_ms, world)
    tot_scat = sum_over_ranks(float(n_scat), world)
    value = tot_scat / (t_max / 1000.0)
    kern_avg_ms = kern_ms / args.steps

    # e2e through the public call with host buffers (copies inside the timed region), on the
    # photon ids of the first e2e_steps timed steps: the same work, so e2e <= the device-timed
    # rate of those steps shows the cost of the copies and the host call
    n_e2e = min(args.e2e_steps, args.steps)
    e2e_ms, e2e_scat = 0.0, 0
    for i in range(n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = step(args.warmup + i, device_out=False)
        e2e_ms += (time.perf_counter() - t0) * 1000.0
        e2e_scat += r.stats["n_scat"]
        assert r.stats["n_scat"] == step_scat[i], "a photon run is deterministic"
    e2e_t = max_over_ranks(e2e_ms, world)
    e2e_value = sum_over_ranks(float(e2e_scat), world) / (e2e_t / 1000.0) if n_e2e > 0 else None
    same_ms = max_over_ranks(sum(per_step_ms[:n_e2e]), world)
    same_value = sum_over_ranks(float(sum(step_scat[:n_e2e])), world) / (same_ms / 1000.0) if n_e2e > 0 else None

    # latency of one event of a lone lane: the longest photon of the last timed step run
    # alone for a bounded number of events (its own history, stopped at the cap)
    ev_count, ev_pid = longest[-1]
    first_last, _ = sharding.photon_range(rank, world, N_PHOTONS, base=(args.warmup + args.steps - 1) * world * N_PHOTONS)
    cap = int(min(ev_count, args.lone_events))
    with torch.cuda.stream(stream):
        ctx.run(geom, n_photons=1, seed=1, first_id=first_last + ev_pid, max_scat=cap, device_out=True, **RUN)
        lone = ctx.run(geom, n_photons=1, seed=1, first_id=first_last + ev_pid, max_scat=cap, device_out=True, **RUN)
    lone_events = lone.stats["n_scat"] + lone.stats["n_dust_scat"]
    us_per_event = lone.stats["elapsed_ms"] * 1e3 / max(lone_events, 1)
    tail_frac = float(np.mean([c * us_per_event * 1e-3 / t for (c, _), t in zip(longest, per_step_ms)]))

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    # Issue roofline of the photon loop (no DRAM traffic to speak of, no dense contraction):
    # peak = the measured FP32-FMA issue rate of this device (thor_issue_peak: one warp
    # instruction per scheduler per clock; nominal 152 SMs x 4 x max SM clock); per-unit
    # figures = warp and thread instructions the kernel executes per resonant scattering on
    # this workload (ncu smsp__inst_executed.sum and smsp__thread_inst_executed.sum / n_scat)
    peak_issue = peak_fma
    inst_per_scat = args.inst_per_scat
    thread_inst_per_scat = args.thread_inst_per_scat
    simt = thread_inst_per_scat / (32.0 * inst_per_scat)
    # DRAM bytes of one bench launch of the shell kernel (ncu dram__bytes_read.sum +
    # dram__bytes_write.sum, one capture of the timed step; code, constants and tallies)
    launch_dram_bytes = args.launch_dram_bytes
    achieved = (n_scat / args.steps) * inst_per_scat / (kern_avg_ms / 1000.0)
    lane_achieved = (n_scat / args.steps) * thread_inst_per_scat / (kern_avg_ms / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": "scatterings/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "photons_per_step": N_PHOTONS, "l2": "flushed (256 MiB write) before each step",
                   "scatterings_per_step": n_scat / args.steps, "kernel_ms_per_step": kern_avg_ms,
                   "launch": {"block": args.block or 128, "blocks_per_sm": args.blocks_per_sm,
                              "pipelined_event_lanes": args.pipe_lanes if args.pipe_lanes >= 0 else 32,
                              "core_burst_lanes": args.burst_lanes if args.burst_lanes >= 0 else 1,
                              "tail_work_sharing": not args.no_tail_share}},
        "e2e": {"value": e2e_value, "unit": "scatterings/s", "h2d_bytes_per_step": 256 + 48,
                "d2h_bytes_per_step": (RUN["n_bins"] + 2) * 8 + 96, "steps": n_e2e,
                "photon_ids": f"those of the first {n_e2e} timed steps",
                "device_timed_value_same_steps": same_value},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_issue / 1e9,
                     "unit": "Gwarp-inst/s", "frac": achieved / peak_issue, "traffic": launch_dram_bytes,
                     "per_unit": f"{inst_per_scat:g} warp instructions per scattering (ncu)",
                     "peak_source": f"measured FP32-FMA issue rate (thor_issue_peak; nominal 152 SMs x 4 schedulers x "
                                    f"{sm_max:.0f} MHz = {152 * 4 * sm_max * 1e-3:.1f} Gwarp-inst/s)",
                     "mufu_peak": peak_mufu / 1e9,
                     "simt_efficiency": simt,
                     "lane_frac": lane_achieved / (32.0 * peak_issue),
                     "lane_per_unit": f"{thread_inst_per_scat:g} thread instructions per scattering (ncu)",
                     "lane_note": "the idle lanes of a cooperative burst form Philox blocks and evaluate throw-away "
                                  "events; their instructions count as executed, so the lane figures overstate "
                                  "useful lane work",
                     "tail": {"longest_photon_events": [c for c, _ in longest],
                              "lone_event_us": us_per_event, "lone_events_timed": lone_events,
                              "tail_frac": tail_frac,
                              "what": "longest photon's events x lone-lane event latency / step time"}},
        "clocks": clk.summary(),
    }
    if args.stream_in_line > 0:
        # p50/p99 latency of the served shell-model stream (the metric's second half), on a
        # stated subset of the 256-request stream
        line["stream"] = stream_bench(ctx, n_requests=args.stream_in_line, nhi_max=args.stream_nhi_max,
                                      core_skip=not args.no_core_skip)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(seconds=args.cpu_seconds)
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def stream_bench(ctx, n_requests=256, seed=2, load=0.75, events_per_round=256, nhi_max=1e21, core_skip=True,
                 priority=True, presort=False):
    """Served shell-model stream (Sec. 5.1 parameter grid): requests with Poisson arrivals at
    `load` x the measured batched capacity, continuous batching on the device.  Baseline,
    also live: the same requests at the same arrival times served one launch per model
    (thor_run), first come first served."""
    from paper_2507_11603_gb300 import synth
    reqs = synth.shell_stream(n_requests, seed=seed, nhi_max=nhi_max)
    common = dict(R_in=0.9, phase="dipole", sigma=50.0, n_bins=400, X_min=-1500.0, X_max=1500.0,
                  core_skip=core_skip)

    def submit(srv, r):
        return srv.submit(N_HI=r["N_HI"], T=r["T"], v_max=r["v_max"], tau_dust=r["tau_dust"],
                          n_photons=r["n_photons"], seed=r["seed"], **common)

    def one_launch(r):
        g = ctx.shell(R_in=0.9, N_HI=r["N_HI"], T=r["T"], v_max=r["v_max"], tau_dust=r["tau_dust"], phase="dipole",
                      core_skip=core_skip)
        res = ctx.run(g, n_photons=r["n_photons"], seed=r["seed"], sigma=50.0, n_bins=400, X_min=-1500.0,
                      X_max=1500.0)
        g.close()
        return res

    # 1) batched capacity: all requests at t = 0
    srv = ctx.server(max_requests=256, events_per_round=events_per_round, priority=priority, presort=presort)
    t0 = time.perf_counter()
    tickets = [submit(srv, r) for r in reqs]
    burst = [srv.wait(t, timeout_ms=600000) for t in tickets]
    burst_total = time.perf_counter() - t0
    burst_scat = sum(b.stats["n_scat"] for b in burst)
    capacity = n_requests / burst_total  # requests/s
    # 2) Poisson stream at `load` x capacity, continuous batching, live
    rate = load * capacity
    rng = np.random.default_rng(seed + 1000)
    arrivals = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0 / rate, n_requests - 1))])
    lat = np.zeros(n_requests)
    done_at = np.zeros(n_requests)
    t_start = time.perf_counter()
    tick = []
    for i, r in enumerate(reqs):
        now = time.perf_counter() - t_start
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        tick.append((i, submit(srv, r), time.perf_counter() - t_start))
    scat = 0
    for i, t, ts in tick:
        res = srv.wait(t, timeout_ms=600000)
        lat[i] = res.stats["elapsed_ms"]
        done_at[i] = ts + lat[i] / 1000.0
        scat += res.stats["n_scat"]
    span = done_at.max()
    stats = srv.stats()
    srv.close()
    # 3) the same arrivals served one launch per model, first come first served, live: a
    # request waits for the runs of the requests before it
    fifo_lat, solo_ms, fifo_scat = np.zeros(n_requests), np.zeros(n_requests), 0
    t_start = time.perf_counter()
    for i, r in enumerate(reqs):
        now = time.perf_counter() - t_start
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        res = one_launch(r)
        fifo_lat[i] = (time.perf_counter() - t_start - arrivals[i]) * 1000.0
        solo_ms[i] = res.stats["elapsed_ms"]
        fifo_scat += res.stats["n_scat"]
    fifo_span = time.perf_counter() - t_start
    j = int(np.argmax(lat))  # the request that sets the batched tail
    slowest = {"request": j, "N_HI": reqs[j]["N_HI"], "T": reqs[j]["T"], "v_max": reqs[j]["v_max"],
               "photons": reqs[j]["n_photons"], "batched_ms": float(lat[j]), "one_launch_run_ms": float(solo_ms[j]),
               "one_launch_fifo_ms": float(fifo_lat[j])}
    return {"requests": n_requests, "slowest": slowest, "photons": int(sum(r["n_photons"] for r in reqs)),
            "core_skip": core_skip, "N_HI_max": nhi_max, "load": load, "rate_per_s": rate, "age_priority": priority,
            "presort": presort,
            "batched": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                        "scatterings_per_s": scat / span, "burst_scatterings_per_s": burst_scat / burst_total,
                        "rounds": stats["rounds"], "mean_resident": stats["mean_resident"],
                        "max_over_own_solo_run": float(np.max(lat / np.maximum(solo_ms, 1e-3)))},
            "one_launch_per_model": {"kind": "live, same arrival times, first come first served",
                                     "p50_ms": float(np.percentile(fifo_lat, 50)),
                                     "p99_ms": float(np.percentile(fifo_lat, 99)),
                                     "scatterings_per_s": fifo_scat / fifo_span,
                                     "slowest_solo_run_ms": float(solo_ms.max())}}


def run_stream_bench(args):
    import torch
    from paper_2507_11603_gb300 import thor
    ctx = thor.Context(0)
    with ClockSampler(0) as clk:
        s = stream_bench(ctx, n_requests=args.stream_requests, nhi_max=args.stream_nhi_max,
                         core_skip=not args.no_core_skip, priority=not args.no_priority,
                         presort=args.presort)
    print(json.dumps({"metric": METRIC, "value": s["batched"]["scatterings_per_s"], "unit": "scatterings/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "served shell-model stream"}, "stream": s, "clocks": clk.summary()}))
    del torch


def run_probe(args):
    """Small launch for profiling, run twice (the second launch is the one to capture).
    --probe-model sphere: a static sphere (tau0 = --probe-tau0, T = 1e4 K, dipole);
    --probe-model shell: the bench's expanding shell.  Photons --probe-first-id ..
    + --probe-photons - 1, each stopped after --probe-max-scat scatterings (0 = never).
    With one photon this times the per-event latency of a lone lane, which bounds the
    tail of the shell run."""
    from paper_2507_11603_gb300 import thor
    ctx = thor.Context(0)
    if args.no_tail_share:
        ctx.set_tail_share(False)
    n = args.probe_photons
    first = args.probe_first_id
    if first < 0 and args.probe_model == "shell":
        # the longest photon of the first 1e5 of the bench workload (one run with records)
        g0 = ctx.shell(**SHELL)
        r0 = ctx.run(g0, n_photons=N_PHOTONS, seed=1, raw=True, **RUN)
        first = int(np.argmax(np.asarray(r0.raw_nscat)))
        g0.close()
    kw = dict(n_photons=n, first_id=max(first, 0), max_scat=args.probe_max_scat)
    if args.probe_model == "shell":
        g = ctx.shell(**SHELL)
        for i in range(2):
            r = ctx.run(g, seed=1, **RUN, **kw)
        desc = {"probe": "expanding shell (bench workload)"}
    else:
        g = ctx.shell(tau0=args.probe_tau0, T=1e4, phase="dipole")
        for i in range(2):
            r = ctx.run(g, seed=i, n_bins=50, X_min=-500, X_max=500, **kw)
        desc = {"probe": "static sphere", "tau0": args.probe_tau0}
    events = r.stats["n_scat"] + r.stats["n_dust_scat"]
    print(json.dumps({**desc, "photons": n, "first_id": max(first, 0), **r.stats,
                      "us_per_event_chain": r.stats["elapsed_ms"] * 1e3 / max(events / n, 1e-30)}))


def run_grid_bench(args):
    """Config 4: 256^3 grid, 100 pc cells, lognormal n_HI (mean 1e-3, sigma_ln 1.5), lognormal T
    (median 1e4 K, sigma_ln 0.5), GRF velocities (k^-11/3, 50 km/s per axis), dust 0.01 n_HI,
    emitters ~ n_HI^2, peeling-off to three axis observers (128x128 x 256 bins).  The photon
    count is a stated subset of the 1e7 of the full configuration."""
    import torch
    from paper_2507_11603_gb300 import synth, thor
    ctx = thor.Context(0)
    f = synth.grid_fields(n=256, seed=3)
    t0 = time.perf_counter()
    g = ctx.grid(f["n_HI"], f["T"], f["v"], f["kd"], 100 * synth.PC_CM)
    t_build = time.perf_counter() - t0
    kw = dict(n_bins=256, X_min=-1000.0, X_max=1000.0, peel=True, img_n=128, peel_bins=256, peel_X_min=-1000.0,
              peel_X_max=1000.0, device_out=True, max_scat=args.grid_max_scat)
    if args.grid_slots:
        ctx.set_grid_exec(args.grid_slots, args.grid_handoff if args.grid_handoff >= 0 else args.grid_slots // 8)
    ctx.run(g, n_photons=max(256, args.grid_photons // 16), seed=4, first_id=10 ** 9, **kw)
    ms, scat, steps, rays, cells = [], 0, 0, 0, 0
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            r = ctx.run(g, n_photons=args.grid_photons, seed=4, first_id=i * args.grid_photons, **kw)
            ms.append(r.stats["elapsed_ms"])
            scat += r.stats["n_scat"]
            steps += r.stats["n_steps"]
            rays += r.stats["n_peel_rays"]
            cells += r.stats["n_peel_cells"]
    t = sum(ms) / 1000.0
    gathers = steps + cells
    print(json.dumps({"metric": "Lyα scatterings/s (grid + peeling-off)", "value": scat / t, "unit": "scatterings/s",
                      "n_gpus": 1, "steps": args.steps, "ms_per_step": 1000 * t / args.steps,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"256^3 grid, {args.grid_photons} photons per step (subset of 1e7)",
                                 "max_scat": args.grid_max_scat, "grid_build_s": t_build,
                                 "execution": (f"event-based, {args.grid_slots} slots" if args.grid_slots
                                               else "one kernel")},
                      "cell_steps_per_s": steps / t, "peel_rays_per_s": rays / t, "peel_cells_per_s": cells / t,
                      # 32 B per cell step and per peel cell, whether the record comes from memory or,
                      # for the photon's current cell, from registers
                      "algorithmic_gather_bytes_per_s": 32.0 * gathers / t, "clocks": clk.summary()}))
    del torch


def run_sweep_bench(args):
    """Shell-model sweep (Sec. 5.1): one radiative-transfer run of the paper's mock model
    (log N_HI = 18.4, v_avg = 120 km/s, log T = 4, alpha_v = 1, alpha_rho = -0.5, ratio of
    the radii 10, dipole phase function, intrinsic line sigma = 800 km/s and EW = 3 A on a
    continuum over +-2500 km/s, 2e5 photons, no dust in the transport), then the
    post-processing that reweights its escaped photons to --sweep-targets (sigma, EW, tau_d)
    combinations (400 bins over +-2500 km/s)."""
    import torch
    from paper_2507_11603_gb300 import thor
    ctx = thor.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    g = ctx.shell(profile="power_law", R_in=0.1, R_out=1.0, N_HI=10 ** 18.4, T=1e4, v_max=120.0, alpha_rho=-0.5,
                  alpha_v=1.0, phase="dipole")
    ew3 = 3.0 / 1215.67 * 299792.458
    kw = dict(n_photons=200_000, sigma=800.0, ew=ew3, C_cont=2500.0, n_bins=400, X_min=-2500.0, X_max=2500.0,
              raw=True, raw_sweep=True, device_out=True)
    ctx.run(g, seed=9, first_id=10 ** 9, **kw)
    rng = np.random.default_rng(12)
    K = args.sweep_targets
    targets = np.stack([rng.uniform(100.0, 800.0, K), rng.uniform(10.0, 200.0, K) / 1215.67 * 299792.458,
                        np.full(K, 2500.0), rng.uniform(0.0, 2.0, K)], axis=1)
    ms_rt, ms_rw, scat = [], [], 0
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            r = ctx.run(g, seed=9, first_id=i * 200_000, **kw)
            ms_rt.append(r.stats["elapsed_ms"])
            scat += r.stats["n_scat"]
            ctx.reweight(r.raw_X0, r.raw_X, r.raw_col, r.raw_status, sample=(800.0, ew3, 2500.0), targets=targets,
                         n_bins=400, X_min=-2500.0, X_max=2500.0)
            ms_rw.append(ctx.last_elapsed_ms())
    t_rt, t_rw = sum(ms_rt) / 1000.0, sum(ms_rw) / 1000.0
    print(json.dumps({"metric": "Lya scatterings/s (power-law shell sweep model, Sec. 5.1)", "value": scat / t_rt,
                      "unit": "scatterings/s", "n_gpus": 1, "steps": args.steps, "ms_per_step": 1000 * t_rt / args.steps,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "power-law shell, log N_HI 18.4, v_avg 120, log T 4, alpha_v 1, "
                                             "alpha_rho -0.5, radius ratio 10, 2e5 photons", "targets": K},
                      "reweight": {"ms_per_call": 1000 * t_rw / args.steps,
                                   "photon_targets_per_s": 200_000 * K * args.steps / t_rw},
                      "clocks": clk.summary()}))


def run_mgii_bench(args):
    """Mg II doublet (Sec. 2.4) in the paper's test geometry: uniform sphere, homologous outflow
    (--mgii-v km/s distance-averaged), N_MgII = 10^14.5 cm^-2, T = 1e4 K, dipole K / isotropic
    H, lit by a flat continuum over -1800..+1000 km/s (K scale); 1e5 photons per step."""
    import torch
    from paper_2507_11603_gb300 import thor
    ctx = thor.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    g = ctx.shell(profile="power_law", species="MgII", R_in=1e-3, R_out=1.0, N_HI=10 ** 14.5, T=1e4,
                  v_max=args.mgii_v, alpha_rho=0.0, alpha_v=1.0, phase="dipole")
    kw = dict(n_photons=100_000, X0=-400.0, sigma=100.0, ew=0.0, C_cont=1400.0, n_bins=300, X_min=-2000.0,
              X_max=1000.0, device_out=True)
    for i in range(args.warmup):
        ctx.run(g, seed=19, first_id=10 ** 9 + i * 100_000, **kw)
    ms, scat = [], 0
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            r = ctx.run(g, seed=19, first_id=i * 100_000, **kw)
            ms.append(r.stats["elapsed_ms"])
            scat += r.stats["n_scat"]
    t = sum(ms) / 1000.0
    print(json.dumps({"metric": "Mg II scatterings/s (doublet, uniform outflowing sphere)", "value": scat / t,
                      "unit": "scatterings/s", "n_gpus": 1, "steps": args.steps, "ms_per_step": 1000 * t / args.steps,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"Mg II sphere N=10^14.5 T=1e4 v_avg={args.mgii_v} km/s, 1e5 photons"},
                      "clocks": clk.summary()}))


def run_peaks_bench(args):
    """Measured issue peaks of the device: FP32 FMA and MUFU ex2 warp instructions/s."""
    from paper_2507_11603_gb300 import thor
    ctx = thor.Context(0)
    with ClockSampler(0) as clk:
        fma = [ctx.issue_peak("fma") for _ in range(3)]
        mufu = [ctx.issue_peak("mufu") for _ in range(3)]
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    print(json.dumps({"metric": "issue peaks", "fma_warp_inst_per_s": max(fma), "mufu_warp_inst_per_s": max(mufu),
                      "fma_lane_flop_per_s": 2 * 32 * max(fma),
                      "nominal_fma_warp_inst_per_s": 152 * 4 * sm_max * 1e6,
                      "nominal_mufu_warp_inst_per_s": 152 * 0.5 * sm_max * 1e6, "clocks": clk.summary()}))


def run_forest_bench(args):
    import torch
    from paper_2507_11603_gb300 import synth, thor
    ctx = thor.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    n = args.forest_n
    xy = args.forest_xy or n  # sightlines per side (a box of n cells along each sightline)
    nHI, T, v = synth.forest_fields_torch(n, seed=5, shape=(n, xy, xy))
    torch.cuda.synchronize()
    ds = synth.forest_scale(2.0, 2.0)
    out = torch.empty((xy * xy, 2 * n), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.forest(nHI, T, v, ds_cm=ds, dv_cell=2.0, n_bins=2 * n, dv_bin=1.0, out=out)
    ms = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            ctx.forest(nHI, T, v, ds_cm=ds, dv_cell=2.0, n_bins=2 * n, dv_bin=1.0, out=out)
            ms.append(ctx.last_elapsed_ms())
    evals = float(xy) * xy * n * 2 * n
    t = float(np.mean(ms)) / 1000.0
    # e2e: the same box from pinned host memory (staged through the library's reused
    # buffers, copies overlapped with the kernel) and the optical depths back to pinned
    # host memory; pinning happens before the timed region
    hn, hT, hv = (x.cpu().pin_memory().numpy() for x in (nHI, T, v))
    hout = torch.empty((xy * xy, 2 * n), dtype=torch.float32, pin_memory=True).numpy()
    del out
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    ctx.forest(hn, hT, hv, ds_cm=ds, dv_cell=2.0, n_bins=2 * n, dv_bin=1.0, out=hout)
    e2e_s = time.perf_counter() - t0
    print(json.dumps({"metric": "Voigt evaluations/s (Lya forest, Eq. 11)", "value": evals / t,
                      "unit": "evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1000 * t, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"forest {xy}x{xy}x{n} box, {xy * xy} sightlines of {n} cells x "
                                             f"{2 * n} bins"},
                      "e2e": {"value": evals / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": 3 * 4 * xy * xy * n,
                              "d2h_bytes_per_step": 4 * xy * xy * 2 * n, "host_memory": "pinned"},
                      "clocks": clk.summary()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="shell",
                    choices=["shell", "forest", "stream", "grid", "probe", "sweep", "mgii", "peaks"])
    ap.add_argument("--mgii-v", type=float, default=100.0)
    ap.add_argument("--sweep-targets", type=int, default=256)
    ap.add_argument("--probe-tau0", type=float, default=1e5)
    ap.add_argument("--probe-photons", type=int, default=64)
    ap.add_argument("--probe-model", choices=("sphere", "shell"), default="sphere")
    ap.add_argument("--probe-first-id", type=int, default=0,
                    help="first photon id of the probe (-1: the longest photon of the first 1e5, shell model)")
    ap.add_argument("--probe-max-scat", type=int, default=0)
    ap.add_argument("--grid-photons", type=int, default=20000)
    ap.add_argument("--grid-slots", type=int, default=0,
                    help="grid workload: event-based loop with this many packets in flight (0 = one kernel)")
    ap.add_argument("--grid-handoff", type=int, default=-1,
                    help="grid workload: packets left when the event-based loop hands over (default slots/8)")
    ap.add_argument("--grid-max-scat", type=int, default=0,
                    help="stop grid photons after this many scatterings (0 = never; for short profiling runs)")
    ap.add_argument("--stream-requests", type=int, default=256)
    ap.add_argument("--stream-in-line", type=int, default=256,
                    help="requests of the served stream measured after the main bench (0 = skip)")
    ap.add_argument("--stream-nhi-max", type=float, default=1e21)
    ap.add_argument("--no-core-skip", action="store_true")
    ap.add_argument("--no-priority", action="store_true", help="served stream without age priority")
    ap.add_argument("--presort", action="store_true", help="served stream with frequency pre-sorting between rounds")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--lone-events", type=int, default=200000,
                    help="events of the longest photon run alone to time the lone-lane event latency")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--pipe-lanes", type=int, default=-1,
                    help="pipelined events in warps with at most this many live packets (-1 = library default)")
    ap.add_argument("--no-tail-share", action="store_true",
                    help="shell workload: no work sharing in the tail of the one-launch run")
    ap.add_argument("--burst-lanes", type=int, default=-1,
                    help="core bursts in warps with at most this many live packets (-1 = library default)")
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--inst-per-scat", type=float, default=365.0,
                    help="warp instructions per scattering of the shell photon loop (ncu, photons 0..19999 of the "
                         "bench workload)")
    ap.add_argument("--thread-inst-per-scat", type=float, default=9276.0,
                    help="thread instructions per scattering of the shell photon loop (ncu, same capture)")
    ap.add_argument("--launch-dram-bytes", type=float, default=798976.0,
                    help="DRAM bytes read + written by one launch of the shell kernel (ncu, same capture; fixed per "
                         "launch: code, constants, tables)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forest-n", type=int, default=1024)
    ap.add_argument("--forest-xy", type=int, default=0,
                    help="sightlines per side of the forest box (0 = forest-n, a cube)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "forest":
        run_forest_bench(args)
    elif args.workload == "stream":
        run_stream_bench(args)
    elif args.workload == "grid":
        run_grid_bench(args)
    elif args.workload == "probe":
        run_probe(args)
    elif args.workload == "sweep":
        run_sweep_bench(args)
    elif args.workload == "mgii":
        run_mgii_bench(args)
    elif args.workload == "peaks":
        run_peaks_bench(args)
    else:
        run_shell_bench(args)


if __name__ == "__main__":
    main()
