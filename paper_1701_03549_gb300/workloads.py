"""Workload presets: seeded inputs of the measured configurations.

Inputs only (maps, ignitions, parameter populations, seeds); no arithmetic of
the method.  The target burnt map of a workload is produced by simulating the
reference parameters (Table 2) with the target seed; the caller supplies the
simulator, so the same preset serves the CUDA path and the CPU oracle.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth

# Smallest share of the burnable cells a target fire must burn; seeds are
# tried upward from synth.TARGET_SEED until a fire reaches it.
TARGET_MIN_FRACTION = 0.01


@dataclass
class Workload:
    name: str
    land: synth.Landscape
    ignition: tuple
    params: np.ndarray      # (n, 5)
    ignitions: np.ndarray   # (n, 2) int32
    seeds: np.ndarray       # (n,) uint64

    @property
    def n(self):
        return self.params.shape[0]

    @property
    def shape(self):
        return self.land.veg.shape


def pick_target(simulate_fn, burnable_count: int, max_tries: int = 64):
    """First seed >= TARGET_SEED whose reference fire burns at least
    TARGET_MIN_FRACTION of the burnable cells.  simulate_fn(seed) returns a
    boolean burnt map."""
    need = max(1, int(np.ceil(TARGET_MIN_FRACTION * burnable_count)))
    for k in range(max_tries):
        seed = synth.TARGET_SEED + k
        burnt = simulate_fn(seed)
        if int(burnt.sum()) >= need:
            return seed, burnt
    raise RuntimeError("no target seed reached the minimum fire size")


def single_fire_128(replicates: int = 64) -> Workload:
    """128 x 128, constant 45 degree wind, the reference parameters, centre
    ignition, replicate seeds 1..replicates."""
    land = synth.preset_landscape("single_fire_128")
    ign = synth.centre_ignition(land.veg)
    n = replicates
    params = np.tile(np.asarray(synth.TRUTH_BETA, np.float64), (n, 1))
    return Workload("single_fire_128", land, ign, params,
                    np.tile(np.asarray(ign, np.int32), (n, 1)),
                    synth.replicate_seeds(n))


def ga_generation_512(population: int = 256, replicates: int = 16,
                      generation_seed: int = 0, first_seed: int = 1) -> Workload:
    """512 x 512 GA generation: `population` parameter vectors drawn from the
    Gauss(0, 5) initial distribution of Table 1, each simulated with
    `replicates` seeds, all from the fixed centre ignition."""
    land = synth.preset_landscape("ga_generation_512")
    ign = synth.centre_ignition(land.veg)
    pop = synth.gauss_population(population, 1000 + generation_seed)
    params = np.repeat(pop, replicates, axis=0)
    n = params.shape[0]
    return Workload("ga_generation_512", land, ign, params,
                    np.tile(np.asarray(ign, np.int32), (n, 1)),
                    synth.replicate_seeds(n, first_seed))


@dataclass
class MultiWorkload:
    name: str
    lands: list
    map_of_sim: np.ndarray   # (n,) int32
    params: np.ndarray       # (n, 5)
    ignitions: np.ndarray    # (n, 2) int32
    seeds: np.ndarray        # (n,) uint64

    @property
    def n(self):
        return self.params.shape[0]


def uneven_lands():
    """Maps of the nine-fire uneven batch: fire i on a (200 + 225 i) x
    (300 + 150 i) grid from map seed 100 + i, constant 45 degree wind."""
    return [synth.landscape(H, W, seed=100 + i)
            for i, (H, W) in enumerate(synth.uneven_fire_shapes())]


def uneven_fires(n_total: int = 100_000, param_seed: int = 0,
                 first_seed: int = 1) -> MultiWorkload:
    """Nine fires on grids 200x300 ... 2000x1500 (fire i: 200 + 225 i rows,
    300 + 150 i columns, map seed 100 + i, constant 45 degree wind), each with
    its centre ignition; n_total simulations spread as evenly as possible
    over the fires (the first fires take the remainder), parameters drawn
    from the Uniform[-30, 30] initial distribution of Table 1."""
    lands = uneven_lands()
    k = len(lands)
    counts = [n_total // k + (1 if i < n_total % k else 0) for i in range(k)]
    map_of_sim = np.repeat(np.arange(k, dtype=np.int32), counts)
    ign = np.array([synth.centre_ignition(L.veg) for L in lands], np.int32)
    params = synth.uniform_population(n_total, 2000 + param_seed)
    return MultiWorkload("uneven_fires", lands, map_of_sim, params,
                         ign[map_of_sim], synth.replicate_seeds(n_total,
                                                               first_seed))


def stratified_sample(groups: np.ndarray, per_group: int) -> np.ndarray:
    """Indices of a stratified sample of a batch: for every group label g
    (0, 1, ...), `per_group` members evenly spaced over the batch positions
    of that group (all of them when the group is smaller), in the order
    round 0 of every group, round 1 of every group, ... so that a prefix of
    the sample covers every group."""
    groups = np.asarray(groups)
    rounds = []
    for g in range(int(groups.max()) + 1):
        pos = np.flatnonzero(groups == g)
        k = min(per_group, pos.size)
        rounds.append(pos[(np.arange(k) * pos.size) // max(k, 1)])
    width = max(r.size for r in rounds)
    out = [r[j] for j in range(width) for r in rounds if j < r.size]
    return np.asarray(out, np.int64)
