#!/usr/bin/env python
"""Throughput of the TRANSIMS cellular-automaton step on one GB300.

One benchmark step is one whole simulation job on the scale-up network
(seeded planar network of 200,000 directed links and 85,000 nodes, the size
of the TIGER network of Sec. 8; 2,000,000 trips with shortest-path routes)
simulated for 10,800 one-second time steps from the empty network, i.e. 3
simulated hours of lane change, velocity update, move and node transfer for
every vehicle in every step.  Inputs are resident in device memory when the
timed region starts; each timed job begins with a device-side reset.

Printed metric: vehicle-updates/s (vehicles that went through the velocity
update, summed over steps, per second), with the multiple of real time
(simulated seconds per wall-clock second, the paper's real-time ratio of
Sec. 8), the share of vehicles that move, and the link kernel's in-graph
duration against the HBM roofline.  The oracle legs (the CPU baseline and
--impl reference) time bounded windows from a seeded peak-hour state, and
the GPU is timed on the same window.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload config2|config1|config0|config3|config4|empty|relax|plan1|yield1|signal1]

With N > 1 (torchrun) every rank runs an independent replica of the job;
there is no exchange between GPUs.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vehicle-updates/s"
L2_FLUSH_BYTES = 512 << 20
STEP_MODES = {"auto": 0, "fused": 1, "split": 2}
PEAK_STEP = 5400  # the departure peak (trips depart ~ Normal(5,400 s, 2,400 s))
KERNEL_SRC = os.path.join(ROOT, "paper_cs_0105004_gb300", "csrc", "kernels.cu")
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _launches(steps, mode, every=0, start=0):
    """Kernel launches of one ts_step call of `steps` steps: the target-setting
    kernel, then per chunk (at most 32 steps, never across a load-balancing
    boundary) a link and a node kernel per step (split steps) or one link
    kernel per step and one node kernel (fused steps), and the chunk close."""
    n, done = 1, 0
    while done < steps:
        seg = steps - done
        if every:
            seg = min(seg, ((start + done) // every + 1) * every - (start + done))
        chunks = (seg + 31) // 32
        n += (seg + 2 * chunks) if mode == "fused" else (2 * seg + chunks)
        done += seg
    return n


def _workload(name):
    from paper_cs_0105004_gb300.inputs import networks as N
    sc = {"config1": N.config1, "config2": N.config2, "config0": N.config0, "plan1": N.config1,
          "yield1": N.config1, "signal1": N.config1}[name]()
    if name == "signal1":
        sc = dataclasses.replace(sc, name="config1-signals",
                                 net=dataclasses.replace(sc.net, link_signal=N.signals_by_rank(sc.net, 60, 30)))
    if name in ("plan1", "yield1"):
        sc = dataclasses.replace(sc, name="config1-turn-lanes",
                                 net=dataclasses.replace(sc.net, turn_lanes=N.turn_lanes_by_rank(sc.net)))
    if name == "yield1":
        sc = dataclasses.replace(sc, name="config1-turn-lanes-yield",
                                 net=dataclasses.replace(sc.net, link_yield=N.yield_by_lanes(sc.net, 8)))
    desc = {
        "config0": "5x5 grid, 80 links of 2 lanes x 60 cells, 2,000 trips",
        "config1": "Portland-shaped planar network, 20,024 links, 8,500 nodes, 300,000 trips",
        "config2": "scale-up planar network, 200,000 links, 85,000 nodes, 2,000,000 trips",
        "plan1": "config 1 (20,024 links, 300,000 trips) with turn lanes: plan-following lane changes",
        "yield1": "config 1 (20,024 links, 300,000 trips) with turn lanes and gap acceptance (narrower "
                  "approaches yield, 8-cell gap)",
        "signal1": "config 1 (20,024 links, 300,000 trips) with a 30 s / 30 s light at every approach of "
                   "every node with two or more approaches",
    }[name]
    return sc, desc


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _loaded(sc, step=None):
    """The seeded peak-hour state that the oracle legs and the GPU window
    start from (inputs.networks.loaded_state: departed trips placed on their
    routes, a share of the links queued up to their end)."""
    import dataclasses
    from paper_cs_0105004_gb300.inputs import networks as N
    t = PEAK_STEP if step is None else step
    return dataclasses.replace(sc, init=N.loaded_state(sc, t, seed=7))


def _sample_steps(args, name, default_big, default_small):
    v = getattr(args, name)
    if v is not None:
        return v
    return default_big if args.workload == "config2" else default_small


def _cpu_baseline(sc, sample_steps):
    """The oracle as it stands, single thread, on `sample_steps` steps from the
    seeded peak-hour state."""
    import oracle
    scl = _loaded(sc)
    orc = oracle.Oracle(scl)
    t0 = time.perf_counter()
    st = orc.step(sample_steps)
    dt = time.perf_counter() - t0
    upd = int(st["vehicle_updates"].sum())
    orc.close()
    return {"value": upd / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{sc.name}: steps {PEAK_STEP}..{PEAK_STEP + sample_steps - 1} from the seeded peak-hour "
                      f"state at step {PEAK_STEP}, one thread, {upd} vehicle updates in {dt:.1f} s",
            "x_real_time": sample_steps / dt}


def run_reference(args, rank, world):
    """Reference arm: the plain CPU oracle timed on bounded samples of the
    workload, consecutive windows from the seeded peak-hour state."""
    if rank != 0:
        return
    import oracle
    sc, desc = _workload(args.workload)
    per = _sample_steps(args, "ref_sample_steps", 10, 100)
    orc = oracle.Oracle(_loaded(sc))
    for _ in range(args.warmup):
        orc.step(per)
    upd, dt = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = orc.step(per)
        dt += time.perf_counter() - t0
        upd += int(st["vehicle_updates"].sum())
    orc.close()
    value = upd / dt
    first = PEAK_STEP + args.warmup * per
    sample = (f"{sc.name}: {args.steps} samples of {per} consecutive steps (steps {first}.."
              f"{first + args.steps * per - 1}) after {args.warmup * per} warm-up steps, from the seeded "
              f"peak-hour state at step {PEAK_STEP}; one thread")
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "x_real_time": per * args.steps / dt,
            "config": {"workload": desc, "steps_per_sample": per, "from_state": f"peak-hour state at step {PEAK_STEP}"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_window(args):
    """For profilers started with --profile-from-start off: steps the workload
    (one scenario, or the config-3 batch) unprofiled to step S, then runs N
    steps between cudaProfilerStart and cudaProfilerStop."""
    import torch
    from paper_cs_0105004_gb300 import transsim as T
    from paper_cs_0105004_gb300.inputs import networks as N
    S, n = (int(x) for x in args.profile_window.split(":"))
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.workload == "config3":
        scs = [N.config3_scenario(i) for i in range(args.scenarios)]
        sims = [T.Simulation(sc, tile_words=args.tile_words) for sc in scs]
        runner = T.Batch(len(sims))
        runner.set_step_mode(STEP_MODES[args.step_mode])
        runner.add_many(sims, S + n)
        advance = lambda k: runner.step(k, stream)
    else:
        sc, _ = _workload(args.workload)
        sim = T.Simulation(sc, tile_words=args.tile_words)
        if args.load_balance:
            sim.set_load_balance(args.load_balance, args.tile_vehicles or 1024)
        sim.set_step_mode(STEP_MODES[args.step_mode])
        sims = [sim]
        advance = lambda k: sim.step(k, stream)
    advance(S)
    stream.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    advance(n)
    stream.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    upd = sum(s.totals()["vehicle_updates"] for s in sims)
    print(json.dumps({"profile_window": {"workload": args.workload, "first_step": S, "steps": n,
                                         "vehicle_updates_to_end": upd}}), flush=True)


def aggregate_over_ranks(t_region, work, dist, device):
    """Replicas (one independent job stream per GPU, no data exchange): the
    job's time is the slowest rank's timed region, its work the sum of the
    ranks' work."""
    import torch
    tt = torch.tensor([t_region], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ww = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(ww, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ww.item())


def kernel_sha():
    """Short hash of the step kernels' source: a stored ncu traffic figure is
    valid only for the kernel build it was captured from."""
    import hashlib
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _profile_traffic(kernel, workload, tag="bench-traffic"):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summaries (a line '<tag>: kernel=K workload=W kernel_sha=S
    dram_bytes_per_launch=B' in profiles/*.md; tag bench-traffic: caches
    flushed before the launch, bench-traffic-warm: caches left warm), or None
    when no summary was taken from the current kernel source."""
    import glob
    import re
    sha = kernel_sha()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for ln in open(path):
            m = re.match(re.escape(tag) + r": kernel=(\S+) workload=(\S+) kernel_sha=(\S+) "
                         r"dram_bytes_per_launch=([0-9.eE+]+)", ln.strip())
            if m and m.group(1) == kernel and m.group(2) == workload and m.group(3) == sha:
                return float(m.group(4)), os.path.relpath(path, ROOT)
    return None, None


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_cs_0105004_gb300 import transsim as T

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    sc, desc = _workload(args.workload)
    steps_per_job = sc.steps if args.job_steps is None else args.job_steps
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    sim = T.Simulation(sc, tile_words=args.tile_words)
    # the re-tiling budget (load per warp tile, a moving vehicle counting 8,
    # a standing one 1): given, or tuned on the
    # first warm-up jobs, one candidate each, the fastest kept
    tune = [] if (args.tile_vehicles or not args.load_balance) else [256, 512, 1024]
    if len(tune) + 2 > args.warmup:
        tune = []  # the first warm-up job captures the graphs, the last runs the choice
    budget = args.tile_vehicles or 1024
    if args.load_balance:
        sim.set_load_balance(args.load_balance, budget)
    sim.set_step_mode(STEP_MODES[args.step_mode])
    net = sc.net
    C = net.n_lane_cells

    def job(s):
        sim.reset(s)
        sim.step(steps_per_job, s)

    # warm-up jobs (also capture the CUDA graphs)
    ref_tot = None
    tuned = {}
    for w in range(args.warmup):
        if 1 <= w <= len(tune):
            sim.set_load_balance(args.load_balance, tune[w - 1])
        elif w == len(tune) + 1 and tune:
            budget = min(tuned, key=tuned.get)
            sim.set_load_balance(args.load_balance, budget)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            job(stream)
            b.record(stream)
        stream.synchronize()
        if 1 <= w <= len(tune):
            tuned[tune[w - 1]] = a.elapsed_time(b)
        tot = sim.totals()
        if ref_tot is not None and tot != ref_tot:
            raise RuntimeError("two runs of the same job differ")
        ref_tot = tot

    sampler = ClockSampler(local_rank)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler.start()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # evict the L2 before every job
            starts[k].record(stream)
            job(stream)
            ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    times_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot = sim.totals()
    if ref_tot is not None and tot != ref_tot:
        raise RuntimeError("timed run differs from the warm-up run")
    job_ms = float(np.mean(times_ms))
    updates = tot["vehicle_updates"]
    # max over ranks of the timed region, sum of the work
    t_region = sum(times_ms) / 1000.0
    work = float(updates) * args.steps
    if dist:
        t_region, work = aggregate_over_ranks(t_region, work, dist, dev)
    value = work / t_region

    # the kernels' own durations inside the same graphs: one more job with
    # kernel spans on (first block past the wait for the previous kernel to
    # the last block's exit), bracketed by CUDA events on the same stream
    sim.set_kernel_timing(True)
    sim.kernel_times(reset=True)
    with torch.cuda.stream(stream):
        flush.fill_(7)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        job(stream)
        b.record(stream)
    torch.cuda.synchronize()
    timed_job_ms = a.elapsed_time(b)
    kt = sim.kernel_times()
    sim.set_kernel_timing(False)
    if sim.totals() != tot:
        raise RuntimeError("the job with kernel spans differs from the timed jobs")
    link_us = 1e6 * kt["link_s"] / max(1, kt["link_launches"])
    node_us = 1e6 * kt["node_s"] / max(1, kt["node_launches"])
    # algorithmic bytes of one link-kernel launch: read + write of v (1 B) and
    # id (4 B) of every vehicle it updates, and of one occupancy bit per
    # lane-cell; in fused steps it also completes the previous step's node
    # transfers (~20 B each) and insertions (~10 B each)
    link_bytes = 10.0 * updates + 0.25 * C * steps_per_job
    if args.step_mode == "fused":
        link_bytes += 20.0 * tot["transfers"] + 10.0 * tot["inserted"]
    link_bytes /= steps_per_job
    peak, peak_kind = _peaks()
    achieved = link_bytes / (link_us * 1e-6) / 1e9
    turns = getattr(net, "turn_lanes", None) is not None or getattr(net, "link_yield", None) is not None
    kernel = "turn_link_kernel" if turns else "link_kernel"
    traffic, traffic_src = _profile_traffic(kernel, args.workload)
    traffic_warm, _ = _profile_traffic(kernel, args.workload, "bench-traffic-warm")
    if args.traffic is not None:
        traffic, traffic_src = args.traffic, "command line"
    step_bytes = (10.0 * updates + 0.25 * C * steps_per_job + 20.0 * tot["transfers"]
                  + 10.0 * tot["inserted"]) / steps_per_job
    roofline = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                "traffic_source": traffic_src, "traffic_note": "ncu, caches flushed before the launch",
                "traffic_warm_l2": traffic_warm, "avg_launch_us": link_us,
                "algorithmic_bytes_per_launch": link_bytes,
                "timing": "in-graph kernel spans (%globaltimer) of one extra job, same graphs and launch shapes",
                "span_job_ms": timed_job_ms, "spans_ms_per_job": 1e3 * (kt["link_s"] + kt["node_s"]),
                "share_of_step_time": kt["link_s"] / max(1e-30, kt["link_s"] + kt["node_s"]),
                "node_kernel": {"launches": kt["node_launches"], "avg_launch_us": node_us},
                "whole_step": {"algorithmic_bytes": step_bytes,
                               "achieved": step_bytes / (job_ms * 1e-3 / steps_per_job) / 1e9,
                               "frac": step_bytes / (job_ms * 1e-3 / steps_per_job) / 1e9 / peak}}

    # the same seeded peak-hour window the oracle legs time, on the GPU
    window = None
    if args.window_steps > 0 and rank == 0:
        scl = _loaded(sc)
        wsecs, wupd = [], None
        for _ in range(3):
            sim.write_state(scl.init)
            with torch.cuda.stream(stream):
                flush.fill_(3)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.step(args.window_steps, stream)
                b.record(stream)
            torch.cuda.synchronize()
            wsecs.append(a.elapsed_time(b) / 1000.0)
            u = sim.totals()["vehicle_updates"]
            if wupd is not None and u != wupd:
                raise RuntimeError("window runs differ")
            wupd = u
        window = {"value": wupd / float(np.median(wsecs)), "unit": METRIC, "from_step": PEAK_STEP,
                  "steps": args.window_steps, "vehicle_updates": wupd,
                  "us_per_step": 1e6 * float(np.median(wsecs)) / args.window_steps,
                  "state": "seeded peak-hour state (inputs.networks.loaded_state, seed 7)"}

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_jobs > 0 and rank == 0:
        dem = sc.demand
        h2d = (net.link_from.nbytes + net.link_to.nbytes + net.link_cells.nbytes + net.link_lanes.nbytes
               + net.link_ring.nbytes + dem.depart_step.nbytes + dem.route_offsets.nbytes + dem.route_links.nbytes
               + sum(a.nbytes for a in (getattr(net, "turn_lanes", None), getattr(net, "link_yield", None),
                                        getattr(net, "link_signal", None)) if a is not None))
        d2h = 9 * 8
        times = []
        for k in range(args.e2e_jobs + 1):
            t0 = time.perf_counter()
            s2 = T.Simulation(sc, tile_words=args.tile_words)
            if args.load_balance:
                s2.set_load_balance(args.load_balance, budget)
            s2.set_step_mode(STEP_MODES[args.step_mode])
            s2.step(steps_per_job)
            t2 = s2.totals()
            s2.close()
            dt = time.perf_counter() - t0
            if t2 != tot:
                raise RuntimeError("end-to-end run differs")
            if k > 0:
                times.append(dt)
        e2e = {"value": updates / float(np.mean(times)), "unit": METRIC, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": d2h, "seconds_per_job": float(np.mean(times))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(sc, _sample_steps(args, "cpu_sample_steps", 40, 300))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": job_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "x_real_time": steps_per_job / (job_ms / 1000.0),
                "config": {"workload": desc, "steps_per_job": steps_per_job, "links": net.n_links,
                           "nodes": net.n_nodes, "trips": sc.demand.n, "lane_cells": C,
                           "vehicle_updates_per_job": updates,
                           "mean_vehicles_updated_per_step": updates / steps_per_job,
                           "moving_share": tot["moving"] / max(1, tot["active"]),
                           "arrived_per_job": tot["arrived"],
                           "l2": "flushed (512 MB write) before every job; the simulation state stays resident "
                                 "across the steps of a job",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "tile_words": sim.tile_words, "step_mode": args.step_mode,
                           "load_balance": {"every_steps": args.load_balance, "vehicles_per_tile": budget,
                                            "tuned_on_warmup_ms": {str(k): round(v, 2) for k, v in tuned.items()}},
                           "bit_exact_hash": str(tot["last_state_hash"])},
                "roofline": roofline, "window": window, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * _launches(steps_per_job, args.step_mode, args.load_balance),
                "clocks": clocks, "wall_s_timed_region": wall}
        print(json.dumps(line), flush=True)
    sim.close()


def _oracle_grid_sample(i, steps):
    """Worker of the all-cores CPU baseline: the oracle, one thread, on the
    first `steps` steps of batch member i."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_cs_0105004_gb300.inputs import networks as N
    sc = N.config3_scenario(i)
    orc = oracle.Oracle(sc)
    t0 = time.perf_counter()
    st = orc.step(steps)
    dt = time.perf_counter() - t0
    orc.close()
    return int(st["vehicle_updates"].sum()), dt


def _cpu_baseline_grids(n_members, steps):
    """The oracle as it stands on the host's cores: one process per core, each
    on one batch member (independent scenarios), processes started by spawn."""
    import multiprocessing as mp
    cores = max(1, min(os.cpu_count() or 1, n_members))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_grid_sample, [(i, steps) for i in range(cores)])
    upd = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": upd / wall, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"config-3 members 0..{cores - 1}, steps 0..{steps - 1} each, one oracle process per core "
                      f"(spawned), {upd} vehicle updates, slowest process {wall:.1f} s"}


def run_config3(args):
    """Batching: 256 independent grid scenarios in one launch set per phase,
    against the same scenarios run one after another."""
    import torch
    from paper_cs_0105004_gb300 import batching as Bt
    from paper_cs_0105004_gb300 import transsim as T
    from paper_cs_0105004_gb300.inputs import networks as N
    torch.cuda.set_device(0)
    steps = args.job_steps or 3600
    scs = [N.config3_scenario(i) for i in range(args.scenarios)]
    stream = torch.cuda.Stream()
    mode_names = {v: k for k, v in STEP_MODES.items()}
    if args.tune_sample > 0:
        best, timings = Bt.autotune(scs[:args.tune_sample], stream, window=256)
    else:
        best, timings = (args.tile_words or 128, 0, STEP_MODES[args.step_mode]), {}
    sims = Bt.make_members(scs, tile_words=best[0])
    batch = T.Batch(len(sims))
    batch.add_many(sims, steps)
    Bt.apply_shape(batch, best)
    chosen_mode = "fused" if best[2] == STEP_MODES["fused"] else "split"
    for _ in range(args.warmup):
        Bt.run_batched(sims, steps, stream, batch)
    sampler = ClockSampler(0)
    sampler.start()
    runs = [Bt.run_batched(sims, steps, stream, batch) for _ in range(args.steps)]
    clocks = sampler.stop()
    if len({r.vehicle_updates for r in runs}) != 1:
        raise RuntimeError("batched runs differ")
    batch.close()
    seq = None
    if args.seq_sample > 0:
        seq = Bt.run_sequential(sims[:args.seq_sample], steps, stream)
        if seq.per_member_updates != runs[0].per_member_updates[:args.seq_sample]:
            raise RuntimeError("sequential and batched results differ")
    sec = sum(r.seconds for r in runs)
    value = sum(r.vehicle_updates for r in runs) / sec
    lane_cells = sum(sc.net.n_lane_cells for sc in scs)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "x_real_time": steps / (sec / args.steps),
            "config": {"workload": f"{args.scenarios} grid scenarios (side 10-60, 1-3 lanes, 30-120 cells, "
                                   f"0.1-0.4 trips per lane-cell), {steps} steps each, one batch",
                       "lane_cells": lane_cells, "trips": int(sum(sc.demand.n for sc in scs)),
                       "vehicle_updates_per_run": runs[0].vehicle_updates,
                       "launch_shape": {"tile_words": best[0], "link_blocks_per_sm": best[1] or "all resident",
                                        "step_mode": chosen_mode},
                       "autotune_seconds": {f"tile_words={k[0]} blocks_per_sm={k[1]} {mode_names[k[2]]}": v
                                            for k, v in sorted(timings.items(), key=lambda kv: kv[1])},
                       "l2": "inputs larger than L2"},
            "sequential": None if seq is None else {"value": seq.updates_per_s, "unit": METRIC,
                                                    "scenarios": args.seq_sample, "seconds": seq.seconds},
            "batched_over_sequential": None if seq is None else value / seq.updates_per_s,
            "cpu_baseline": None if args.no_cpu_baseline else _cpu_baseline_grids(args.scenarios, 600),
            "gpu_launches": args.steps * (_launches(steps, chosen_mode) - 1 + args.scenarios),
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    for s_ in sims:
        s_.close()


def run_empty(args):
    """The config 1 network with no vehicles: the cost of sweeping every
    lane-cell's occupancy each step, which the step pays at any load (Sec. 9
    notes the same floor for an empty network)."""
    import numpy as np
    import torch
    from paper_cs_0105004_gb300 import transsim as T
    from paper_cs_0105004_gb300.inputs import networks as N
    torch.cuda.set_device(0)
    full = N.config1()
    steps = args.job_steps or full.steps
    none = N.Demand(np.zeros(0, np.uint32), np.zeros(1, np.uint32), np.zeros(0, np.uint32))
    sc = N.Scenario("config1-empty", full.net, none, steps, full.seed)
    sim = T.Simulation(sc)
    sim.set_step_mode(STEP_MODES[args.step_mode])
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def job():
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.reset(stream)
        sim.step(steps, stream)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1000.0

    for _ in range(args.warmup):
        job()
    sampler = ClockSampler(0)
    sampler.start()
    secs = [job() for _ in range(args.steps)]
    clocks = sampler.stop()
    # the kernels' durations inside the same graphs (kernel spans of one more job)
    sim.set_kernel_timing(True)
    sim.kernel_times(reset=True)
    job()
    kt = sim.kernel_times()
    sim.set_kernel_timing(False)
    sec = sum(secs)
    C = sc.net.n_lane_cells
    peak, src = _peaks()
    link_us = 1e6 * kt["link_s"] / max(1, kt["link_launches"])
    node_us = 1e6 * kt["node_s"] / max(1, kt["node_launches"])
    line = {"metric": "lane-cell updates/s", "value": C * steps * args.steps / sec, "unit": "lane-cell updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "x_real_time": steps / (sec / args.steps),
            "config": {"workload": "config 1 network (20,024 links, 8,500 nodes) with no trips",
                       "steps_per_job": steps, "lane_cells": C,
                       "l2": "flushed (512 MB write) before every job"},
            "us_per_sim_step": 1e6 * sec / (args.steps * steps),
            "roofline": {"bound": "hbm", "kernel": "link_kernel", "achieved": 0.25 * C / (link_us * 1e-6) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": 0.25 * C / (link_us * 1e-6) / 1e9 / peak,
                         "peak_source": src, "traffic": None, "avg_launch_us": link_us,
                         "timing": "in-graph kernel spans of one extra job",
                         "node_kernel_avg_launch_us": node_us},
            "gpu_launches": args.steps * _launches(steps, args.step_mode),
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    sim.close()


def run_relax(args):
    """Relaxation iterations (Sec. 1) on config 1: each iteration is one full
    GPU run of 10,800 steps, then 10 % of the travellers are re-planned on
    the run's link travel times (host Dijkstra)."""
    import torch
    from paper_cs_0105004_gb300 import relaxation as R
    from paper_cs_0105004_gb300.inputs import networks as N
    torch.cuda.set_device(0)
    sc = N.config1()
    if args.job_steps:
        sc = dataclasses.replace(sc, steps=args.job_steps)
    stream = torch.cuda.Stream()
    run = lambda s: R.gpu_run(s, stream)
    R.relax(sc, 1, run=run)  # warm-up: library load, graph capture
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    last, its = R.relax(sc, args.relax_iters, fraction=0.1, seed=0, run=run)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    sim_s = sum(it.run.seconds for it in its)
    upd = sum(it.run.vehicle_updates for it in its)
    line = {"metric": METRIC, "value": upd / sim_s, "unit": METRIC, "n_gpus": 1, "steps": args.relax_iters,
            "warmup": 1, "ms_per_step": 1000.0 * sim_s / args.relax_iters, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "relaxation iterations on config 1 (20,024 links, 300,000 trips), "
                                   "10 % re-planned per iteration on measured link travel times",
                       "steps_per_run": sc.steps, "iterations": args.relax_iters},
            "wall_seconds_per_iteration": wall / args.relax_iters,
            "iterations": [{"gpu_s": round(it.run.seconds, 4), "plan_s": round(it.plan_seconds, 3),
                            "vehicle_updates": it.run.vehicle_updates, "arrived": it.run.arrived,
                            "mean_link_time": round(it.run.mean_link_time, 3), "replanned": it.replanned}
                           for it in its],
            "gpu_launches": args.relax_iters * _launches(sc.steps, "auto"),
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_config4(args):
    """Serving: a Poisson stream of simulation jobs admitted by device-memory
    budget into a continuously running batch."""
    import torch
    from paper_cs_0105004_gb300 import serving as Sv
    from paper_cs_0105004_gb300.inputs import networks as N
    torch.cuda.set_device(0)
    steps = args.job_steps or 3600
    c0 = N.config0()
    c1 = N.config1() if args.serve_mix[1] > 0 else None
    grids = [N.config3_scenario(i) for i in range(args.grid_pool)]
    arrivals = Sv.poisson_arrivals(args.rate, args.duration, seed=7)
    rng = np.random.default_rng(7)
    mix = np.array(args.serve_mix, dtype=float)
    kinds = rng.choice(3, size=arrivals.size, p=mix / mix.sum())
    jobs = []
    for jid, (t, kd) in enumerate(zip(arrivals, kinds)):
        base = [c0, c1, grids[jid % len(grids)]][kd]
        def make(base=base, jid=jid):
            return N.Scenario(f"{base.name}/job{jid}", base.net, base.demand, steps, seed=100000 + jid,
                              vmax=base.vmax, p_threshold=base.p_threshold)
        jobs.append(Sv.Job(jid, ["config0", "config1", "grid"][kd], float(t), make, steps))
    import copy
    seq_jobs = copy.deepcopy(jobs) if args.serve_compare else None
    srv = Sv.Server(budget_bytes=int(args.budget_gb * 2**30), chunk_steps=args.chunk)
    sampler = ClockSampler(0)
    sampler.start()
    rep = srv.run(jobs, time_scale=args.time_scale)
    clocks = sampler.stop()
    srv.close()
    summ = rep.summary()
    one = None
    if seq_jobs is not None:
        # the same stream served one job at a time (each job alone on the GPU)
        srv1 = Sv.Server(budget_bytes=int(args.budget_gb * 2**30), capacity=1, chunk_steps=args.chunk)
        rep1 = srv1.run(seq_jobs, time_scale=args.time_scale)
        srv1.close()
        one = rep1.summary()
        by = {j.jid: j for j in rep.jobs}
        if any(by[j.jid].last_state_hash != j.last_state_hash for j in rep1.jobs):
            raise RuntimeError("a job differs between the batched and the one-at-a-time server")
    line = {"metric": METRIC, "value": summ["vehicle_updates_per_s"], "unit": METRIC, "n_gpus": 1,
            "steps": len(rep.jobs), "warmup": 0, "ms_per_step": 1000.0 * rep.wall_s / max(1, len(rep.jobs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"Poisson {args.rate}/s jobs for {args.duration} s, mix config0:config1:grid = "
                                   f"{args.serve_mix}, {steps} steps per job, arrival clock x{args.time_scale}",
                       "budget_gb": args.budget_gb, "chunk_steps": args.chunk},
            "serving": summ, "one_job_at_a_time": one,
            "served_over_one_at_a_time": (None if one is None else
                                          summ["vehicle_updates_per_s"] / one["vehicle_updates_per_s"]),
            "gpu_launches": summ["chunks"] * (2 * args.chunk + (args.chunk + 31) // 32), "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config2", choices=["config0", "config1", "config2", "config3", "config4", "empty", "relax", "plan1",
                                                  "yield1", "signal1"])
    ap.add_argument("--scenarios", type=int, default=256, help="config3: batch members")
    ap.add_argument("--tune-sample", type=int, default=32, help="config3: members used by the autotuner")
    ap.add_argument("--seq-sample", type=int, default=256, help="config3: members run one by one for comparison")
    ap.add_argument("--rate", type=float, default=20.0, help="config4: job arrivals per second")
    ap.add_argument("--duration", type=float, default=600.0, help="config4: seconds of arrivals")
    ap.add_argument("--time-scale", type=float, default=1.0, help="config4: arrival clock factor")
    ap.add_argument("--serve-mix", type=float, nargs=3, default=[60, 10, 30], help="config4: config0 config1 grid")
    ap.add_argument("--grid-pool", type=int, default=256,
                    help="config4: distinct grid networks (the config-3 members), each job with its own seed")
    ap.add_argument("--budget-gb", type=float, default=160.0, help="config4: device memory for jobs")
    ap.add_argument("--chunk", type=int, default=128, help="config4: steps per batch step")
    ap.add_argument("--serve-compare", type=int, default=1, help="config4: also serve the stream one job at a time")
    ap.add_argument("--job-steps", type=int, default=None, help="steps per job (default: the config's)")
    ap.add_argument("--relax-iters", type=int, default=4, help="relax: iterations")
    ap.add_argument("--e2e-jobs", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=None,
                    help="oracle steps of the CPU baseline from the peak-hour state (default 40 on config2, else 300)")
    ap.add_argument("--ref-sample-steps", type=int, default=None,
                    help="reference arm: oracle steps per sample (default 10 on config2, else 100)")
    ap.add_argument("--window-steps", type=int, default=300,
                    help="GPU steps timed from the peak-hour state the oracle legs start from")
    ap.add_argument("--tile-words", type=int, default=None, help="occupancy words per link tile (8..256)")
    ap.add_argument("--profile-window", default=None, metavar="S:N",
                    help="step unprofiled to S, then run N steps inside cudaProfilerStart/Stop, and exit")
    ap.add_argument("--step-mode", default="auto", choices=list(STEP_MODES),
                    help="fused: one launch per step; split: link and node kernel per step")
    ap.add_argument("--load-balance", type=int, default=512, help="re-tile from the occupancy every N steps (0 = off)")
    ap.add_argument("--tile-vehicles", type=int, default=None,
                    help="re-tiling budget per warp tile, a moving vehicle counting 8 and a standing one 1 "
                         "(default: tuned on the warm-up jobs among 256, 512 and 1024 when there are at least five, "
                         "else 1024)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per link_kernel launch from an ncu capture of this kernel")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_window:
        if rank == 0:
            run_profile_window(args)
        return
    if args.workload == "config3":
        if rank == 0:
            run_config3(args)
        return
    if args.workload == "config4":
        if rank == 0:
            run_config4(args)
        return
    if args.workload == "empty":
        if rank == 0:
            run_empty(args)
        return
    if args.workload == "relax":
        if rank == 0:
            run_relax(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
