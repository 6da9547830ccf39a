"""Throughput of batched fire-spread simulations on GB300.

One step = one GA generation of the 512 x 512 calibration workload: 256
parameter vectors drawn from the Gauss(0, 5) initial distribution (Table 1)
x 16 replicate seeds = 4096 independent simulations from the fixed centre
ignition, each run to extinction and scored against the reference burnt map
(Eq. 2 counts fused in the simulation kernel, fitness ratios by a second
kernel).  Inputs are resident on the device before timing; every step uses
fresh seeds; L2 is flushed (256 MB write) between timed steps.

Prints one JSON line (see the keys below).  ``--impl reference`` times the
CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1701_03549_gb300 import parallel, synth, workloads  # noqa: E402

METRIC = "CA sims/s"
UNIT = "sims/s"
POP, REPS = 256, 16
SIMS = POP * REPS
# Algorithmic operations of one trial: one Philox4x32-10 output word (10
# rounds of 8 integer operations per 4-word block: 20) plus Eq. 1 for one
# direction and its comparison with the draw (the five-term sum as 4 FMAs,
# exponential 2, 1 + e 1, reciprocal 1, draw to float 2, compare 1: 11).
OPS_PER_TRIAL = 31
ALU_LANES_PER_SM = 128
WORKLOAD = ("ga_generation_512: 512x512 map, 256 Gauss(0,5) parameter "
            "vectors x 16 replicates = 4096 simulations/step, centre "
            "ignition, constant 45 deg wind, target from the reference "
            "parameters")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("fire_kernels.cu", "fire_device.cuh", "fire_internal.h"):
        with open(os.path.join(ROOT, "paper_1701_03549_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _committed_profile(name="k_simulate_traffic.json"):
    """The committed ncu record of the simulation kernel (DRAM and L2 bytes
    per launch), or None when the kernel changed since it was captured."""
    p = os.path.join(ROOT, "profiles", name)
    try:
        with open(p) as f:
            d = json.load(f)
    except OSError:
        return None
    if d.get("source_sha256") != _kernel_hash():
        return None
    return d


def _committed_traffic():
    d = _committed_profile()
    return None if d is None else d.get("dram_bytes_per_launch")


def _memory_roofs(kernel_s, peaks, peaks_kind, name="k_simulate_traffic.json"):
    """DRAM and L2 bandwidth of the simulation kernel: bytes per launch from
    the committed ncu capture over the event-timed launch duration, against
    the measured HBM copy bandwidth and ncu's L2 sector peak."""
    d = _committed_profile(name)
    if d is None:
        return None
    dram = d["dram_bytes_per_launch"] / kernel_s / 1e9
    l2 = d["l2_bytes_per_launch"] / kernel_s / 1e9
    l2_peak = (d["l2_bytes_per_launch"] / (d["ncu_duration_ms"] / 1e3) / 1e9 /
               (d["l2_pct_of_peak_sectors"] / 100.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    return {"dram_gbs": dram, "dram_frac": dram / hbm,
            "dram_peak_gbs": hbm, "dram_peak_source": f"hbm_gbs ({peaks_kind})",
            "l2_gbs": l2, "l2_frac": l2 / l2_peak, "l2_peak_gbs": l2_peak,
            "l2_peak_source": "ncu lts__t_sectors peak"}


def _dense_sweep_roof(cell_updates_per_s, peaks, peaks_kind):
    """Cell-updates/s (dense-equivalent: steps x H x W per second) against
    what a dense sweep of the whole grid every step could reach at the
    measured HBM bandwidth, streaming only the 2-bit state (2 bits read and 2
    written per cell-update, 0.5 B) and nothing else.  A reference point for
    the rate, not this kernel's bound: the worklists skip quiet tiles, so
    the kernel moves far fewer bytes than such a sweep."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    dense = hbm * 1e9 / 0.5
    return {"model": "dense 2-bit-state sweep, 0.5 B per cell-update",
            "dense_rate": dense, "unit": "cell-updates/s",
            "ratio": cell_updates_per_s / dense,
            "dense_rate_source": f"hbm_gbs ({peaks_kind})"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarise(lines)

    @staticmethod
    def summarise(lines):
        """Median and maximum SM clock and the throttle reasons seen, from
        the sampler's CSV rows (malformed rows are skipped)."""
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() in ("active", "1", "yes")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


_WORKER = {}


def _oracle_init(land_args, target):
    """Spawned worker: build the oracle's covariates and target once."""
    import oracle

    _WORKER["F"] = oracle.Features(synth.landscape(*land_args))
    _WORKER["target"] = target


def _oracle_job(args):
    """One oracle simulation in a worker process; returns its step count."""
    beta, ign, seed = args
    res, _ = _WORKER["F"].simulate(beta, ign, int(seed),
                                   target=_WORKER["target"], want_steps=False)
    return res["steps"]


def oracle_throughput(wl, target, nsims: int, cores: int):
    """Oracle simulations/s on the first nsims simulations of the workload,
    one simulation per task, `cores` single-threaded worker processes."""
    import multiprocessing as mp

    p = synth.PRESETS["ga_generation_512"]
    land_args = (p["H"], p["W"], p["map_seed"], p["wind_seed"])
    jobs = [(wl.params[i], wl.ignition, int(wl.seeds[i]))
            for i in range(nsims)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_init,
                  initargs=(land_args, target)) as pool:
        pool.map(_oracle_job, [(np.full(5, -1000.0), wl.ignition, 1)] * cores,
                 chunksize=1)  # wait until every worker is initialised
        t0 = time.perf_counter()
        steps = pool.map(_oracle_job, jobs, chunksize=1)
        dt = time.perf_counter() - t0
    return nsims / dt, dt, sum(steps)


def oracle_target(wl):
    import oracle

    F = oracle.Features(wl.land)
    return workloads.pick_target(
        lambda s: F.simulate(synth.TRUTH_BETA, wl.ignition, s)[1] >= 0,
        int(F.burnable.sum()))


def run_reference(args):
    rank, world, _ = parallel.env_rank()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    wl = workloads.ga_generation_512(POP, REPS)
    _, target = oracle_target(wl)
    per_step = min(SIMS, 4 * cores)
    times = []
    for k in range(args.warmup + args.steps):
        sub = workloads.ga_generation_512(POP, REPS,
                                          first_seed=1 + k * SIMS)
        v, dt, _ = oracle_throughput(sub, target, per_step, cores)
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "H": 512,
                                        "W": 512, "sims_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": f"first {per_step} simulations of each "
                                   "4096-simulation generation"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_native(args):
    import torch

    rank, world, local = parallel.env_rank()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__

    __graft_entry__.build()
    from paper_1701_03549_gb300 import fire

    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = fire.Context(local, stream)
    first = parallel.rank_seed_offset(rank, SIMS * (args.warmup + args.steps + 2))
    wl = workloads.ga_generation_512(POP, REPS, first_seed=first)
    m = ctx.landscape_upload(wl.land)
    H, W = wl.shape
    # target: reference parameters, first seed from TARGET_SEED with a
    # non-trivial fire (simulated on this GPU)
    burnable = int((wl.land.veg != 0).sum())

    def sim_target(seed):
        _, bs = m.simulate_batch(np.asarray([synth.TRUTH_BETA]),
                                 np.asarray([wl.ignition], np.int32),
                                 np.asarray([seed], np.uint64),
                                 want_steps=True)
        return bs[0] >= 0

    tseed, target = workloads.pick_target(sim_target, burnable)
    m.target_upload(target)
    # launch shape: the autotuner times its candidate shapes on this batch in
    # the step's longest-first order (outside the timed region) and the
    # library uses the fastest
    tuned = fire.fire_autotune(ctx, [m], None, wl.params, wl.ignitions,
                               wl.seeds, longest_first=True)

    nsteps = args.warmup + args.steps
    p_dev = torch.tensor(wl.params, dtype=torch.float64, device=dev)
    g_dev = torch.tensor(wl.ignitions, dtype=torch.int32, device=dev)
    seeds_all = [wl.seeds + np.uint64(k * SIMS) for k in range(nsteps)]
    s_dev = [torch.tensor(s.view(np.int64), device=dev) for s in seeds_all]
    outs = [torch.zeros((SIMS, 6), dtype=torch.int32, device=dev)
            for _ in range(nsteps)]
    fit = [torch.zeros(SIMS, dtype=torch.float64, device=dev)
           for _ in range(nsteps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step(k):
        m.simulate_batch(p_dev, g_dev, s_dev[k], device=True, out=outs[k],
                         longest_first=True)
        fire.fire_fitness(ctx, outs[k], fire.FITNESS_JACCARD, device=True,
                          out=fit[k])

    for k in range(args.warmup):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    for j in range(args.steps):
        k = args.warmup + j
        flush.zero_()
        e0, e1, e2 = ev[j]
        e0.record(stream)
        m.simulate_batch(p_dev, g_dev, s_dev[k], device=True, out=outs[k],
                         longest_first=True)
        e1.record(stream)
        fire.fire_fitness(ctx, outs[k], fire.FITNESS_JACCARD, device=True,
                          out=fit[k])
        e2.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    sim_ms = [ev[j][0].elapsed_time(ev[j][1]) for j in range(args.steps)]
    step_ms = [ev[j][0].elapsed_time(ev[j][2]) for j in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    total_s = parallel.max_over_ranks(total_s, world, dev)

    # statistics of the timed steps
    res = [fire.results_view(outs[args.warmup + j]) for j in range(args.steps)]
    steps_sum = sum(int(r["steps"].astype(np.int64).sum()) for r in res)
    trials_sum = sum(int(r["trials"].astype(np.int64).sum()) for r in res)
    # all ranks' counts (each rank simulates its own seeds)
    steps_all = parallel.sum_over_ranks(steps_sum, world, dev)
    trials_all = parallel.sum_over_ranks(trials_sum, world, dev)
    assert all(int((r["status"] & (fire.STATUS_BAD_IGNITION
                                    | fire.STATUS_TIMEOUT)).max()) == 0
               for r in res)
    sims_total = SIMS * args.steps * world
    value = sims_total / total_s

    # roofline of the simulation kernel (ALU bound): algorithmic operations
    # per launch over its mean event-timed duration
    peaks, peaks_kind = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    peak_ops = props.multi_processor_count * ALU_LANES_PER_SM * sm_max * 1e6
    mean_sim_s = sum(sim_ms) / len(sim_ms) / 1e3
    ops_per_launch = trials_sum / args.steps * OPS_PER_TRIAL
    achieved = ops_per_launch / mean_sim_s
    traffic = _committed_traffic()

    # end to end through the C ABI with host buffers (pinned)
    pin_p = torch.from_numpy(wl.params.copy()).pin_memory().numpy()
    pin_g = torch.from_numpy(wl.ignitions.copy()).pin_memory().numpy()
    e2e_steps = max(3, min(args.steps, 10))
    e2e_seeds = [torch.from_numpy((wl.seeds + np.uint64((nsteps + j) * SIMS))
                                  .view(np.int64)).pin_memory().numpy()
                 .view(np.uint64) for j in range(e2e_steps)]
    m.simulate_batch(pin_p, pin_g, e2e_seeds[0],    # warm the staging buffers
                     longest_first=True)
    t0 = time.perf_counter()
    for j in range(e2e_steps):
        r, _ = m.simulate_batch(pin_p, pin_g, e2e_seeds[j], longest_first=True)
        f = fire.fire_fitness(ctx, r, fire.FITNESS_JACCARD)
    e2e_s = time.perf_counter() - t0
    e2e_s = parallel.max_over_ranks(e2e_s, world, dev)
    e2e_value = SIMS * e2e_steps * world / e2e_s
    h2d = SIMS * (40 + 8 + 8) + SIMS * 24
    d2h = SIMS * 24 + SIMS * 8

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        tw = workloads.ga_generation_512(POP, REPS, first_seed=first)
        nsample = min(SIMS, 32 * cores)
        v, dt, _ = oracle_throughput(tw, target, nsample, cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {nsample} simulations of one 4096-simulation "
                         f"generation ({dt:.1f} s wall)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W,
                       "sims_per_step": SIMS, "target_seed": tseed,
                       "target_cells": int(target.sum()),
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}",
                       "order": "longest-first by predicted spread "
                                "(FIRE_LONGEST_FIRST)",
                       "launch": {k: tuned[k] for k in (
                           "warps_per_block", "blocks_per_sm",
                           "queue_entries", "state_mode")}},
            "cell_updates_per_s": steps_all * H * W / total_s,
            "cell_updates_vs_dense_sweep": _dense_sweep_roof(
                steps_all * H * W / total_s, peaks, peaks_kind),
            "trials_per_s": trials_all / total_s,
            "mean_steps_per_sim": steps_all / (SIMS * args.steps * world),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tops/s",
                         "frac": achieved / peak_ops, "traffic": traffic,
                         "kernel": "k_simulate",
                         "peak_source": f"{props.multi_processor_count} SMs x "
                                        f"{ALU_LANES_PER_SM} lanes x "
                                        f"{sm_max:.0f} MHz ({peaks_kind} max "
                                        "SM clock)",
                         "ops_per_trial": OPS_PER_TRIAL,
                         "kernel_ms": 1e3 * mean_sim_s,
                         "memory": _memory_roofs(mean_sim_s, peaks, peaks_kind)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            # per step: k_spread_key and k_rank_desc (longest-first order),
            # k_simulate, k_fitness
            "gpu_launches": 4 * args.steps,
            "clocks": ck,
        }
        print(json.dumps(line))
    m.free()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


UNEVEN = ("uneven_fires: nine fires on 200x300 ... 2000x1500 grids (10.9 M "
          "cells), 100,000 simulations in one persistent launch (11,112 on "
          "the first fire, 11,111 on each other), Uniform[-30,30] parameters, "
          "centre ignitions, targets from the reference parameters")


def run_uneven(args):
    """Nine-fire uneven batch: one fire_simulate_multi call per step (CUDA
    graph replay) plus the fitness kernel."""
    import torch

    rank, world, local = parallel.env_rank()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_1701_03549_gb300 import fire

    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = fire.Context(local, stream)
    nsteps = args.warmup + args.steps
    wl = workloads.uneven_fires(first_seed=1 + rank * 100_000 * (nsteps + 1))
    n = wl.n
    maps = [ctx.landscape_upload(L) for L in wl.lands]
    for j, (m, L) in enumerate(zip(maps, wl.lands)):
        ign = np.asarray([wl.ignitions[np.argmax(wl.map_of_sim == j)]],
                         np.int32)
        burnable = int((L.veg != 0).sum())

        def sim_target(seed, m=m, ign=ign):
            _, bs = m.simulate_batch(np.asarray([synth.TRUTH_BETA]), ign,
                                     np.asarray([seed], np.uint64),
                                     want_steps=True)
            return bs[0] >= 0

        _, tg = workloads.pick_target(sim_target, burnable)
        m.target_upload(tg)
    # autotune on a stratified tenth of the batch
    sub = np.arange(0, n, 10)
    tuned = fire.fire_autotune(ctx, maps, wl.map_of_sim[sub], wl.params[sub],
                               wl.ignitions[sub], wl.seeds[sub])
    t_mi = torch.tensor(wl.map_of_sim, device=dev)
    t_p = torch.tensor(wl.params, dtype=torch.float64, device=dev)
    t_g = torch.tensor(wl.ignitions, device=dev)
    t_s = torch.tensor(wl.seeds.view(np.int64), device=dev)
    seeds_all = [torch.tensor((wl.seeds + np.uint64(k * n)).view(np.int64),
                              device=dev) for k in range(nsteps)]
    out = torch.zeros((n, 6), dtype=torch.int32, device=dev)
    fit = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step(k):
        t_s.copy_(seeds_all[k])
        fire.fire_simulate_multi(ctx, maps, t_mi, t_p, t_g, t_s, device=True,
                                 out=out, graph=True)
        fire.fire_fitness(ctx, out, fire.FITNESS_JACCARD, device=True, out=fit)

    for k in range(args.warmup):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    total_ms = 0.0
    steps_sum = trials_sum = cells = 0
    sizes = np.array([L.veg.size for L in wl.lands], np.int64)[wl.map_of_sim]
    for j in range(args.steps):
        k = args.warmup + j
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t_s.copy_(seeds_all[k])
        e0.record(stream)
        fire.fire_simulate_multi(ctx, maps, t_mi, t_p, t_g, t_s, device=True,
                                 out=out, graph=True)
        fire.fire_fitness(ctx, out, fire.FITNESS_JACCARD, device=True, out=fit)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        r = fire.results_view(out)
        steps_sum += int(r["steps"].astype(np.int64).sum())
        cells += int((r["steps"].astype(np.int64) * sizes).sum())
        trials_sum += int(r["trials"].astype(np.int64).sum())
    ck = clocks.stop()
    total_s = parallel.max_over_ranks(total_ms / 1e3, world, dev)
    value = n * args.steps * world / total_s
    cells_all = parallel.sum_over_ranks(cells, world, dev)
    trials_all = parallel.sum_over_ranks(trials_sum, world, dev)
    if rank == 0:
        peaks, peaks_kind = _peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        props = torch.cuda.get_device_properties(dev)
        peak_ops = props.multi_processor_count * ALU_LANES_PER_SM * sm_max * 1e6
        achieved = trials_sum * OPS_PER_TRIAL / (total_ms / 1e3)
        uprof = _committed_profile("k_simulate_uneven_traffic.json")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": UNEVEN, "sims_per_step": n,
                       "cells_total": int(sum(L.veg.size for L in wl.lands)),
                       "graph": True, "l2": "flushed between timed steps "
                       "(256 MB write)",
                       "launch": {k: tuned[k] for k in (
                           "warps_per_block", "blocks_per_sm",
                           "queue_entries", "state_mode")}},
            "cell_updates_per_s": cells_all / total_s,
            "cell_updates_vs_dense_sweep": _dense_sweep_roof(
                cells_all / total_s, peaks, peaks_kind),
            "trials_per_s": trials_all / total_s,
            "mean_steps_per_sim": steps_sum / (n * args.steps),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tops/s",
                         "frac": achieved / peak_ops,
                         "traffic": (None if uprof is None
                                     else uprof["dram_bytes_per_launch"]),
                         "kernel": "k_simulate",
                         "peak_source": f"{props.multi_processor_count} SMs x "
                                        f"{ALU_LANES_PER_SM} lanes x "
                                        f"{sm_max:.0f} MHz ({peaks_kind})",
                         "ops_per_trial": OPS_PER_TRIAL,
                         "kernel_ms": total_ms / args.steps,
                         "memory": _memory_roofs(
                             total_ms / args.steps / 1e3, peaks, peaks_kind,
                             "k_simulate_uneven_traffic.json")},
            "cpu_baseline": None, "e2e": None,
            "gpu_launches": 5 * args.steps,
            "clocks": ck,
        }
        print(json.dumps(line))
    for m in maps:
        m.free()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


SURROGATE = ("surrogate_screened_ga_1024: 1024x1024 map (spatially varying "
             "wind), target from the reference parameters at the centre "
             "ignition; BF16 surrogate (S=256, ~1.05M params) trained on "
             "200k automaton runs (6250 Gauss(0,5) draws x 16 replicates on "
             "each of the 512x512 and 1024x1024 maps); plain GA population "
             "1024 x 16 replicates against the screened GA (1024 candidates "
             "per generation, 256 simulated x 16 replicates: the 192 best "
             "predicted and 64 drawn from the rest)")
TRAIN_FLOP_PER_PIXEL = 2.0 * 128 * ((144 + 7 * 1152) * 2 + 7 * 1152)
FWD_FLOP_PER_PIXEL = 2.0 * 128 * (144 + 7 * 1152)


def _recovery(ctx, m, ign, hist, truth, f_star, torch, reps=64, frac=0.1,
              tol=0.05, seed=1 << 33):
    """Per generation: the ensemble (best `frac` of the evaluated population)
    mean, its fitness re-scored with `reps` fresh replicates, and the
    relative error of each parameter.  Recovered = the first generation whose
    ensemble fits the target within `tol` of the reference parameters' own
    fitness f_star; returns (fits, errors, generation, seconds) with the
    seconds of the GA up to and including that generation."""
    from paper_1701_03549_gb300 import calibrate, fire

    ens = []
    for P, F in zip(hist.params, hist.fitness):
        order = np.argsort(F, kind="stable")
        ens.append(P[order[:max(1, int(len(F) * frac))]].mean(axis=0))
    ens = np.asarray(ens)
    G = len(ens)
    fits = calibrate.evaluate(
        ctx, m, torch.tensor(ens, device="cuda"), ign,
        np.arange(seed, seed + G * reps, dtype=np.uint64), reps,
        fire.FITNESS_JACCARD, torch).cpu().numpy()
    errs = np.abs(ens - truth) / np.abs(truth)
    t = np.cumsum(hist.seconds)
    hit = np.nonzero(fits <= (1.0 + tol) * f_star)[0]
    g = int(hit[0]) if hit.size else None
    return fits, errs, g, (float(t[g]) if g is not None else None)


def run_surrogate(args):
    """Config 4: surrogate-screened GA against the plain GA (one GPU)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1701_03549_gb300 import calibrate, fire, surrogate

    rank, world, local = parallel.env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = fire.Context(local, stream)
    truth = np.asarray(synth.TRUTH_BETA, np.float64)
    land = synth.preset_landscape("ignition_search_1024")
    land2 = synth.preset_landscape("ga_generation_512")
    m = ctx.landscape_upload(land)
    m2 = ctx.landscape_upload(land2)
    ign = synth.centre_ignition(land.veg)

    def sim_target(seed):
        _, bs = m.simulate_batch(truth[None], np.asarray([ign], np.int32),
                                 np.asarray([seed], np.uint64), want_steps=True)
        return bs[0] >= 0

    _, tgt = workloads.pick_target(sim_target, int((land.veg != 0).sum()))
    m.target_upload(tgt)
    sur = surrogate.Surrogate(ctx, S=256, max_batch=8, seed=1)

    # training data from the automaton
    t0 = time.perf_counter()
    groups = args.train_groups
    data = [surrogate.make_dataset(ctx, m2, land2, sur, groups, 16, 21),
            surrogate.make_dataset(ctx, m, land, sur, groups, 16, 22)]
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    # training
    t0 = time.perf_counter()
    losses = sur.train(data, steps=args.train_steps, lr=2e-3, lr_final=1e-4,
                       seed=3)
    t_train = time.perf_counter() - t0
    pix_per_step = 8 * 256 * 256
    train_tflops = (args.train_steps * pix_per_step * TRAIN_FLOP_PER_PIXEL /
                    t_train / 1e12)
    # forward pass alone (roofline of the convolution path)
    x = torch.empty((8, 256, 256, 16), dtype=torch.bfloat16, device=dev)
    sur.inputs(data[1].planes, 1024, 1024, data[1].params[:8].contiguous(),
               data[1].ign[:8].contiguous(), out=x)
    prob = torch.empty((8, 256, 256), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(3):
        sur.net.forward(x, prob)
    ms = []
    for _ in range(10):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sur.net.forward(x, prob)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    fwd_ms = statistics.median(ms)
    fwd_tflops = pix_per_step * FWD_FLOP_PER_PIXEL / (fwd_ms / 1e3) / 1e12

    # the two GAs
    gens = args.generations
    clocks = Clocks(local)
    t0 = time.perf_counter()
    plain = calibrate.run_ga(ctx, m, ign, pop=1024, reps=16, generations=gens,
                             ga_seed=5, sim_seed=1 << 30)
    t_plain = time.perf_counter() - t0
    plain256 = calibrate.run_ga(ctx, m, ign, pop=256, reps=16,
                                generations=gens, ga_seed=5,
                                sim_seed=1 << 32)
    t0 = time.perf_counter()
    scr = surrogate.run_screened_ga(ctx, m, land, sur, ign, pop=256, pool=1024,
                                    reps=16, generations=gens, ga_seed=5,
                                    sim_seed=1 << 31)
    t_scr = time.perf_counter() - t0
    ck = clocks.stop()
    f_star = float(calibrate.evaluate(
        ctx, m, torch.tensor(truth[None], device=dev), ign,
        np.arange(1 << 34, (1 << 34) + 64, dtype=np.uint64), 64,
        fire.FITNESS_JACCARD, torch).cpu().numpy()[0])
    f_plain, e_plain, g_plain, s_plain = _recovery(ctx, m, ign, plain, truth,
                                                   f_star, torch)
    f_scr, e_scr, g_scr, s_scr = _recovery(ctx, m, ign, scr, truth, f_star,
                                           torch)
    f_p256, e_p256, g_p256, s_p256 = _recovery(ctx, m, ign, plain256, truth,
                                               f_star, torch)
    peaks, kind = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    line = {
        "metric": "time-to-recover 5 params, surrogate-GA vs plain GA",
        "value": s_scr, "unit": "s", "n_gpus": world, "steps": gens,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_scr / gens,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (surrogate) / u32 (automaton)", "data": "synthetic",
        "config": {"workload": SURROGATE, "S": 256, "train_groups": 2 * groups,
                   "train_runs": 2 * groups * 16,
                   "train_steps": args.train_steps, "batch": 8,
                   "recovered_when": "the mean of the best 10% of a generation, "
                                     "re-scored with 64 fresh replicates, fits "
                                     "the target within 5% of the reference "
                                     "parameters' own fitness (64 replicates)"},
        "reference_fitness": f_star,
        "plain_ga": {"generations": gens, "seconds": t_plain,
                     "recovered_generation": g_plain, "recovered_s": s_plain,
                     "sims_per_generation": 1024 * 16,
                     "ensemble_fitness_by_gen": [round(float(x), 4)
                                                 for x in f_plain],
                     "final_rel_error": [round(float(x), 3)
                                         for x in e_plain[-1]]},
        "plain_ga_256": {"generations": gens,
                         "seconds": float(sum(plain256.seconds)),
                         "recovered_generation": g_p256,
                         "recovered_s": s_p256,
                         "sims_per_generation": 256 * 16,
                         "ensemble_fitness_by_gen": [round(float(x), 4)
                                                     for x in f_p256],
                         "final_rel_error": [round(float(x), 3)
                                             for x in e_p256[-1]]},
        "screened_ga": {"generations": gens, "seconds": t_scr,
                        "recovered_generation": g_scr, "recovered_s": s_scr,
                        "sims_per_generation": 256 * 16,
                        "ensemble_fitness_by_gen": [round(float(x), 4)
                                                    for x in f_scr],
                        "final_rel_error": [round(float(x), 3)
                                            for x in e_scr[-1]]},
        "training": {"data_s": t_data, "train_s": t_train,
                     "tflops": train_tflops,
                     "loss_first": float(np.mean(losses[:10])),
                     "loss_last": float(np.mean(losses[-50:]))},
        "roofline": {"bound": "tensor", "achieved": fwd_tflops, "peak": peak,
                     "unit": "TFLOP/s", "frac": fwd_tflops / peak,
                     "traffic": None, "kernel": "surrogate forward "
                     "(k_conv_tma_p x7 + layer-1 k_conv1_tma + head), batch 8 x 256^2",
                     "peak_source": f"bf16_tflops ({kind})"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None,
        "clocks": ck,
    }
    if rank == 0:
        print(json.dumps(line))
    sur.net.free()
    m.free()
    m2.free()
    ctx.close()
    return 0


def run_surrogate_step(args):
    """Surrogate network alone: forward passes and training steps (forward,
    backward, Adam) on a batch of 8 inputs of 256 x 256 (random weights and
    inputs; no automaton), with the tensor-core roofline."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1701_03549_gb300 import fire, surrogate

    rank, world, local = parallel.env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = fire.Context(local, stream)
    B, S = 8, 256
    net = fire.Net(ctx, S, B)
    net.set_params(surrogate.init_params(1))
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.rand((B, S, S, 16), device=dev, generator=g).to(torch.bfloat16)
    t = torch.rand((B, S, S), device=dev, generator=g)
    prob = torch.empty((B, S, S), device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    pix = B * S * S

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    clocks = Clocks(local)
    fwd_ms = timed(lambda: net.forward(x, prob))
    train_ms = timed(lambda: (net.backward(x, t, loss), net.adam(1e-4)))
    ck = clocks.stop()
    fwd = pix * FWD_FLOP_PER_PIXEL / (fwd_ms / 1e3) / 1e12
    trn = pix * TRAIN_FLOP_PER_PIXEL / (train_ms / 1e3) / 1e12
    peaks, kind = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    if rank == 0:
        print(json.dumps({
            "metric": "surrogate training throughput", "value": trn,
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": train_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "surrogate_step: 1.05M-parameter dilated "
                       "conv net, batch 8 x 256 x 256 x 16, random weights "
                       "and inputs", "l2": "flushed between timed steps "
                       "(256 MB write)"},
            "forward_ms": fwd_ms, "forward_tflops": fwd,
            "roofline": {"bound": "tensor", "achieved": trn, "peak": peak,
                         "unit": "TFLOP/s", "frac": trn / peak,
                         "traffic": None, "kernel": "training step (k_conv_tma_p "
                         "forward and input gradient, k_wgrad_tma, layer-1 "
                         "tile, head, Adam)",
                         "peak_source": f"bf16_tflops ({kind})"},
            "cpu_baseline": None, "e2e": None,
            # per training step: the forward pass (first layer + seven
            # 128 -> 128 convolutions), head and head gradient, per layer a
            # weight gradient and a bias gradient (8 each) and, above the
            # first, an input gradient (7), and Adam
            "gpu_launches": 34 * args.steps,
            "clocks": ck}))
    net.free()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"),
                    default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload",
                    choices=("ga512", "uneven", "surrogate", "surrogate_step"),
                    default="ga512",
                    help="ga512: 512x512 GA generation (default line); "
                         "uneven: nine fires 200x300..2000x1500, 100k "
                         "simulations in one launch; surrogate: the "
                         "surrogate-screened GA against the plain GA")
    ap.add_argument("--generations", type=int, default=50)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--train-groups", type=int, default=6250)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "surrogate_step":
        return run_surrogate_step(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
