"""Parameter calibration on top of the CUDA library: the paper's genetic
algorithm (Sec. 2.2, Appendix B), its brute-force Monte Carlo alternative
(Appendix C) and the ensemble estimate (Sec. 2.1 rules: rank the simulations
by fitness and keep those below a cutoff; the estimate is the ensemble's mean
and standard deviation, the best set the one of least fitness).

All simulation, fitness, replicate averaging and GA arithmetic runs in the
library's kernels on device-resident torch tensors; this module only sequences
the calls and keeps the per-generation history.  The context may issue work
on a stream other than torch's, so tensors are synchronised at each hand-off
between torch and the library.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import fire, synth


@dataclass
class History:
    params: list = field(default_factory=list)     # per generation (P, 5)
    fitness: list = field(default_factory=list)    # per generation (P,)
    seconds: list = field(default_factory=list)    # wall time per generation

    def all(self):
        return np.concatenate(self.params), np.concatenate(self.fitness)


def _meta(kind_of_run, **kw):
    return json.dumps(dict(run=kind_of_run, **{k: (float(v) if isinstance(
        v, float) else v) for k, v in kw.items()}), sort_keys=True)


def save_checkpoint(path: str, generation: int, genes: np.ndarray,
                    hist: History, meta: str) -> None:
    """State of a GA run after `generation` generations: the population of
    the next generation, every finished generation's population, fitness and
    wall time, and the run's settings (the keyed draws of the GA step and of
    the simulations depend only on them and the generation index, so a
    resumed run continues bit for bit).  Written to a temporary file and
    renamed, so an interrupted write leaves the previous checkpoint."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, generation=np.int64(generation), genes=np.asarray(genes),
             params=np.asarray(hist.params), fitness=np.asarray(hist.fitness),
             seconds=np.asarray(hist.seconds, np.float64), meta=np.str_(meta))
    os.replace(tmp, path)


def load_checkpoint(path: str, meta: str):
    """(generation, genes, History) of a checkpoint written by a run with the
    same settings; ValueError for one of another run."""
    with np.load(path) as z:
        if str(z["meta"]) != meta:
            raise ValueError(f"checkpoint {path} belongs to another run")
        hist = History(list(z["params"]), list(z["fitness"]),
                       [float(x) for x in z["seconds"]])
        return int(z["generation"]), np.array(z["genes"]), hist


def sim_seeds(base: int, generation: int, pop: int, reps: int) -> np.ndarray:
    """Seeds of generation g: base + (g P + i) R + r for individual i,
    replicate r."""
    first = base + (generation * pop) * reps
    return np.arange(first, first + pop * reps, dtype=np.uint64)


def evaluate(ctx, m, params_dev, ignition, seeds, reps, kind, torch):
    """Mean fitness over `reps` replicates of each parameter vector (device
    tensors in, device tensor out)."""
    dev = params_dev.device
    P = params_dev.shape[0]
    n = P * reps
    p_sims = params_dev.repeat_interleave(reps, dim=0).contiguous()
    ign = torch.tensor(np.tile(np.asarray(ignition, np.int32), (n, 1)),
                       device=dev)
    s = torch.tensor(np.asarray(seeds, np.uint64).view(np.int64), device=dev)
    out = torch.zeros((n, 6), dtype=torch.int32, device=dev)
    fit = torch.zeros(n, dtype=torch.float64, device=dev)
    mean = torch.zeros(P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    m.simulate_batch(p_sims, ign, s, device=True, out=out, longest_first=True)
    fire.fire_fitness(ctx, out, kind, device=True, out=fit)
    fire.fire_group_mean(ctx, fit, reps, device=True, out=mean)
    ctx.sync()
    return mean


def evaluate_sharded(ctx, m, params_dev, ignition, seeds, reps, kind, torch,
                     rank: int, world: int):
    """evaluate() with the generation's P x reps simulations split over
    `world` ranks (one GPU each): each rank simulates its contiguous block,
    the fire_result records are all-gathered (24 bytes per simulation, the
    only collective), and every rank computes the same fitness and replicate
    means on its device."""
    from . import parallel

    dev = params_dev.device
    P = params_dev.shape[0]
    n = P * reps
    p_all = params_dev.repeat_interleave(reps, dim=0).contiguous()
    s_all = np.asarray(seeds, np.uint64)

    def shard(lo, hi):
        k = hi - lo
        if k == 0:
            return np.zeros(0, fire.RESULT_DTYPE)
        ign = torch.tensor(np.tile(np.asarray(ignition, np.int32), (k, 1)),
                           device=dev)
        s = torch.tensor(s_all[lo:hi].view(np.int64), device=dev)
        out = torch.zeros((k, 6), dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        m.simulate_batch(p_all[lo:hi].contiguous(), ign, s, device=True,
                         out=out, longest_first=True)
        ctx.sync()
        return fire.results_view(out)

    res = parallel.sharded_results(n, shard, rank, world)
    raw = np.ascontiguousarray(res).view(np.int32).reshape(n, 6)
    out = torch.tensor(raw, device=dev)
    fit = torch.zeros(n, dtype=torch.float64, device=dev)
    mean = torch.zeros(P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    fire.fire_fitness(ctx, out, kind, device=True, out=fit)
    fire.fire_group_mean(ctx, fit, reps, device=True, out=mean)
    ctx.sync()
    return mean


def run_ga(ctx, m, ignition, pop=256, reps=16, generations=50,
           prior="gauss", lo=-30.0, hi=30.0, ga_seed=1, sim_seed=1,
           kind=fire.FITNESS_JACCARD, init=None, rank=0, world=1,
           checkpoint=None, stop_after=None):
    """The Appendix B genetic algorithm on map `m` (which holds the target).
    Returns the History of every generation's population and fitness.  With
    world > 1 (one process per GPU, default process group initialised) each
    generation's simulations are split over the ranks (evaluate_sharded);
    the GA step is replicated, so every rank holds the same population.
    checkpoint: a path; the run saves its state there after every
    generation and, when the file exists, resumes from it (bit-identical to
    an uninterrupted run).  stop_after: return after that many generations
    of this call (the history so far)."""
    import torch

    dev = torch.device("cuda", ctx.device)
    G = 5
    meta = _meta("ga5", pop=pop, reps=reps, generations=generations,
                 prior=prior, lo=lo, hi=hi, ga_seed=ga_seed,
                 sim_seed=sim_seed, kind=int(kind), ignition=list(map(
                     int, ignition)), custom_init=init is not None)
    if init is None:
        init = (synth.gauss_population(pop, ga_seed) if prior == "gauss"
                else synth.uniform_population(pop, ga_seed, lo=lo, hi=hi))
    init = np.clip(np.asarray(init, np.float64), lo, hi)
    start, hist = 0, History()
    if checkpoint and os.path.exists(checkpoint):
        start, init, hist = load_checkpoint(checkpoint, meta)
    genes = torch.tensor(init, dtype=torch.float64, device=dev)
    nxt = torch.empty_like(genes)
    tlo = torch.full((G,), float(lo), dtype=torch.float64, device=dev)
    thi = torch.full((G,), float(hi), dtype=torch.float64, device=dev)
    for g in range(start, generations):
        t0 = time.perf_counter()
        seeds = sim_seeds(sim_seed, g, pop, reps)
        if world > 1:
            f = evaluate_sharded(ctx, m, genes, ignition, seeds, reps, kind,
                                 torch, rank, world)
        else:
            f = evaluate(ctx, m, genes, ignition, seeds, reps, kind, torch)
        hist.params.append(genes.cpu().numpy())
        hist.fitness.append(f.cpu().numpy())
        if g + 1 < generations:
            torch.cuda.synchronize(dev)
            fire.ga_step(ctx, genes, f, g, generations, ga_seed, tlo, thi,
                         device=True, out=nxt)
            ctx.sync()
            genes, nxt = nxt, genes
        hist.seconds.append(time.perf_counter() - t0)
        if checkpoint and rank == 0:
            save_checkpoint(checkpoint, g + 1, genes.cpu().numpy(), hist, meta)
        if stop_after is not None and g + 1 - start >= stop_after:
            break
    return hist


def scar_layout(pop: int, scars: int, reps: int) -> np.ndarray:
    """Scar index of every simulation of a multi-scar generation: individual
    i, scar k, replicate r is simulation (i K + k) R + r."""
    return np.tile(np.repeat(np.arange(scars, dtype=np.int32), reps), pop)


def evaluate_multi(ctx, maps, params_dev, ignitions, seeds, reps, kind, torch):
    """Mean fitness of each parameter vector over several reference scars:
    every individual is simulated `reps` times on each scar k (maps[k] holds
    that scar's landscape and target burnt map, ignitions[k] its ignition),
    in one uneven-batch launch; each simulation is scored against its own
    scar's target and an individual's fitness is the mean over its K x reps
    simulations (scar-major, then replicate order)."""
    dev = params_dev.device
    P = params_dev.shape[0]
    K = len(maps)
    n = P * K * reps
    mos = scar_layout(P, K, reps)
    p_sims = params_dev.repeat_interleave(K * reps, dim=0).contiguous()
    t_mos = torch.tensor(mos, device=dev)
    t_ign = torch.tensor(np.asarray(ignitions, np.int32).reshape(K, 2)[mos],
                         device=dev)
    s = torch.tensor(np.asarray(seeds, np.uint64).view(np.int64), device=dev)
    out = torch.zeros((n, 6), dtype=torch.int32, device=dev)
    fit = torch.zeros(n, dtype=torch.float64, device=dev)
    mean = torch.zeros(P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    fire.fire_simulate_multi(ctx, maps, t_mos, p_sims, t_ign, s, device=True,
                             out=out)
    fire.fire_fitness(ctx, out, kind, device=True, out=fit)
    fire.fire_group_mean(ctx, fit, K * reps, device=True, out=mean)
    ctx.sync()
    return mean


def run_ga_multi(ctx, maps, ignitions, pop=256, reps=8, generations=50,
                 prior="gauss", lo=-30.0, hi=30.0, ga_seed=1, sim_seed=1,
                 kind=fire.FITNESS_JACCARD, init=None, checkpoint=None,
                 stop_after=None):
    """The Appendix B genetic algorithm fitted to several reference scars at
    once (the paper's suggestion for parameters one scar leaves weakly
    determined, Sec. 4): the fitness of an individual is its mean over the
    scars of the replicate-mean fitness against each scar (evaluate_multi);
    selection, crossover and mutation are those of run_ga.  maps[k] holds
    scar k's landscape and target, ignitions[k] its ignition (row, col).
    Seeds of generation g: sim_seeds(sim_seed, g, pop, K reps).
    checkpoint and stop_after as in run_ga."""
    import torch

    dev = torch.device("cuda", ctx.device)
    G = 5
    K = len(maps)
    meta = _meta("ga5multi", pop=pop, reps=reps, generations=generations,
                 prior=prior, lo=lo, hi=hi, ga_seed=ga_seed,
                 sim_seed=sim_seed, kind=int(kind), scars=K,
                 ignitions=[list(map(int, g)) for g in ignitions],
                 custom_init=init is not None)
    if init is None:
        init = (synth.gauss_population(pop, ga_seed) if prior == "gauss"
                else synth.uniform_population(pop, ga_seed, lo=lo, hi=hi))
    init = np.clip(np.asarray(init, np.float64), lo, hi)
    start, hist = 0, History()
    if checkpoint and os.path.exists(checkpoint):
        start, init, hist = load_checkpoint(checkpoint, meta)
    genes = torch.tensor(init, dtype=torch.float64, device=dev)
    nxt = torch.empty_like(genes)
    tlo = torch.full((G,), float(lo), dtype=torch.float64, device=dev)
    thi = torch.full((G,), float(hi), dtype=torch.float64, device=dev)
    for g in range(start, generations):
        t0 = time.perf_counter()
        f = evaluate_multi(ctx, maps, genes, ignitions,
                           sim_seeds(sim_seed, g, pop, K * reps), reps, kind,
                           torch)
        hist.params.append(genes.cpu().numpy())
        hist.fitness.append(f.cpu().numpy())
        if g + 1 < generations:
            torch.cuda.synchronize(dev)
            fire.ga_step(ctx, genes, f, g, generations, ga_seed, tlo, thi,
                         device=True, out=nxt)
            ctx.sync()
            genes, nxt = nxt, genes
        hist.seconds.append(time.perf_counter() - t0)
        if checkpoint:
            save_checkpoint(checkpoint, g + 1, genes.cpu().numpy(), hist, meta)
        if stop_after is not None and g + 1 - start >= stop_after:
            break
    return hist


def evaluate_at(ctx, m, params_dev, ign_dev, seeds, reps, kind, torch):
    """Mean fitness over `reps` replicates of each parameter vector, each
    replicate starting from its own ignition (ign_dev: (P reps, 2) int32
    device tensor, replicates of an individual consecutive)."""
    dev = params_dev.device
    P = params_dev.shape[0]
    n = P * reps
    p_sims = params_dev.repeat_interleave(reps, dim=0).contiguous()
    s = torch.tensor(np.asarray(seeds, np.uint64).view(np.int64), device=dev)
    out = torch.zeros((n, 6), dtype=torch.int32, device=dev)
    fit = torch.zeros(n, dtype=torch.float64, device=dev)
    mean = torch.zeros(P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    m.simulate_batch(p_sims, ign_dev, s, device=True, out=out,
                     longest_first=True)
    fire.fire_fitness(ctx, out, kind, device=True, out=fit)
    fire.fire_group_mean(ctx, fit, reps, device=True, out=mean)
    ctx.sync()
    return mean


def initial_population_7(target, burnable, pop, seed, prior="gauss",
                         lo=-30.0, hi=30.0):
    """Seven-gene individuals (beta_0..beta_4, x, y): the parameters from the
    Table 1 prior, the ignition point from the reference fire's burnt area
    (Sec. 3: fires start from random points of the reference scar)."""
    beta = (synth.gauss_population(pop, seed) if prior == "gauss"
            else synth.uniform_population(pop, seed, lo=lo, hi=hi))
    xy = synth.burnt_area_points(np.asarray(target) & np.asarray(burnable),
                                 pop, seed)
    return np.concatenate([np.clip(beta, lo, hi), xy], axis=1)


def run_ga_ignition(ctx, m, target, burnable, pop=256, reps=16,
                    generations=50, prior="gauss", lo=-30.0, hi=30.0,
                    ga_seed=1, sim_seed=1, kind=fire.FITNESS_JACCARD,
                    init=None, checkpoint=None, stop_after=None):
    """The Appendix B genetic algorithm with the ignition point unknown
    (Sec. 3, Table 3): seven genes, the five parameters of Eq. 1 and the
    ignition's x (column) and y (row), bounded by the grid.  Each
    generation maps every individual's (x, y) to the nearest burnable cell
    of the target scar (fire_snap_ignitions), simulates it `reps` times
    from there, scores the replicate-mean fitness and breeds the next
    generation (ga_step, G = 7).  History.params holds (P, 7) arrays.
    checkpoint and stop_after as in run_ga."""
    import torch

    dev = torch.device("cuda", ctx.device)
    H, W = m.H, m.W
    meta = _meta("ga7", pop=pop, reps=reps, generations=generations,
                 prior=prior, lo=lo, hi=hi, ga_seed=ga_seed,
                 sim_seed=sim_seed, kind=int(kind), shape=[H, W],
                 custom_init=init is not None)
    if init is None:
        init = initial_population_7(target, burnable, pop, ga_seed, prior,
                                    lo, hi)
    start, hist = 0, History()
    if checkpoint and os.path.exists(checkpoint):
        start, init, hist = load_checkpoint(checkpoint, meta)
    genes = torch.tensor(np.asarray(init, np.float64), device=dev)
    nxt = torch.empty_like(genes)
    tlo = torch.tensor([lo] * 5 + [0.0, 0.0], dtype=torch.float64, device=dev)
    thi = torch.tensor([hi] * 5 + [W - 1.0, H - 1.0], dtype=torch.float64,
                       device=dev)
    ign = torch.empty((pop * reps, 2), dtype=torch.int32, device=dev)
    for g in range(start, generations):
        t0 = time.perf_counter()
        torch.cuda.synchronize(dev)
        fire.fire_snap_ignitions(ctx, m, genes, 5, 6, reps, device=True,
                                 out=ign)
        f = evaluate_at(ctx, m, genes[:, :5].contiguous(), ign,
                        sim_seeds(sim_seed, g, pop, reps), reps, kind, torch)
        hist.params.append(genes.cpu().numpy())
        hist.fitness.append(f.cpu().numpy())
        if g + 1 < generations:
            torch.cuda.synchronize(dev)
            fire.ga_step(ctx, genes, f, g, generations, ga_seed, tlo, thi,
                         device=True, out=nxt)
            ctx.sync()
            genes, nxt = nxt, genes
        hist.seconds.append(time.perf_counter() - t0)
        if checkpoint:
            save_checkpoint(checkpoint, g + 1, genes.cpu().numpy(), hist, meta)
        if stop_after is not None and g + 1 - start >= stop_after:
            break
    return hist


def run_mc(ctx, m, ignition, n=4096, reps=1, lo=-30.0, hi=30.0, seed=1,
           sim_seed=1, kind=fire.FITNESS_JACCARD):
    """Appendix C brute-force Monte Carlo: parameters uniform in [lo, hi]^5,
    each simulated `reps` times; returns (params, mean fitness)."""
    import torch

    dev = torch.device("cuda", ctx.device)
    params = synth.uniform_population(n, seed, lo=lo, hi=hi)
    f = evaluate(ctx, m, torch.tensor(params, dtype=torch.float64, device=dev),
                 ignition, sim_seeds(sim_seed, 0, n, reps), reps, kind, torch)
    return params, f.cpu().numpy()


def ensemble(params, fitness, cutoff=None, keep=None):
    """Ensemble estimate: the simulations with fitness <= cutoff (or the
    `keep` best); returns dict(mean, sd, best, size)."""
    params = np.asarray(params, np.float64)
    fitness = np.asarray(fitness, np.float64)
    order = np.argsort(fitness, kind="stable")
    if cutoff is not None:
        sel = order[fitness[order] <= cutoff]
    else:
        sel = order[: (keep or max(1, len(order) // 10))]
    if sel.size == 0:
        sel = order[:1]
    ens = params[sel]
    sd = ens.std(axis=0, ddof=1) if len(sel) > 1 else np.zeros(params.shape[1])
    return {"mean": ens.mean(axis=0), "sd": sd, "best": params[order[0]],
            "best_fitness": float(fitness[order[0]]), "size": int(sel.size)}
