"""Parity at full sizes and at the largest grid the library accepts, on sampled
outputs the oracle computes one by one (the benchmark's own launches are
checked in test_gpu_bench_launch.py):

* the 1024 x 1024 ignition search (32 x 32 candidates x 64 replicates =
  65,536 simulations): candidate cells against the nearest-cell definition,
  the fitness map against the replicate means of the batch's own results,
  and sampled simulations of that batch against the oracle;
* a 4096 x 4096 map (the maximum tile count): burn-step maps and counts of
  fires from its corners and centre.

The oracle runs in a spawn process pool (started before any GPU call).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_W = {}


def _init_ign(H, W, map_seed, wind_seed):
    import oracle

    from paper_1701_03549_gb300 import synth

    land = synth.landscape(H, W, seed=map_seed, wind_seed=wind_seed)
    _W["F"] = oracle.Features(land)


def _run_ign(args):
    beta, ign, seed, target = args
    r, _ = _W["F"].simulate(beta, ign, int(seed), target=target,
                            want_steps=False)
    return r


MAX_HW = 4096          # 128 x 128 tiles of 32 x 32 = FIRE_MAX_TILES
MAX_SIMS = [           # (beta, ignition, seed, step cap)
    ([2.0, 0, 0, 0, 0], (0, 0), 11, 60),
    ([2.0, 0, 0, 0, 0], (4095, 4095), 12, 60),
    ([0.5, 0.5, 0.5, 1.0, -1.0], (0, 4095), 13, 60),
    ([0.0, 1.0, 0.5, 1.0, -1.0], (4095, 0), 14, 60),
    ([1000.0, 0, 0, 0, 0], (2047, 2048), 15, 40),
    ([-1.2, 0, 0, 0, 0], (1000, 3000), 17, 60),   # dies out at step 44
]


def _max_land(seed):
    from paper_1701_03549_gb300 import synth

    land = synth.noise_landscape(MAX_HW, MAX_HW, seed)
    for _, (r, c), _, _ in MAX_SIMS:
        land.veg[r, c] = 1
    target = np.random.default_rng(seed + 1).random(land.veg.shape) < 0.3
    return land, target


def _init_max(seed):
    import oracle

    land, target = _max_land(seed)
    _W["F"] = oracle.Features(land)
    _W["target"] = target


def _run_max(k):
    beta, ign, seed, cap = MAX_SIMS[k]
    r, bs = _W["F"].simulate(beta, ign, seed, target=_W["target"],
                             want_steps=True, max_steps=cap)
    idx = np.flatnonzero(bs.ravel() >= 0)
    return r, idx, bs.ravel()[idx]


def _pool(init, initargs=(), procs=16):
    return mp.get_context("spawn").Pool(min(procs, os.cpu_count() or 1),
                                        initializer=init, initargs=initargs)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    oracle.build()
    return torch


def test_ignition_search_full_size_sample(env):
    torch = env
    import oracle

    from paper_1701_03549_gb300 import fire, synth

    p = synth.PRESETS["ignition_search_1024"]
    H, W = p["H"], p["W"]
    pool = _pool(_init_ign, (H, W, p["map_seed"], p["wind_seed"]))
    try:
        land = synth.preset_landscape("ignition_search_1024")
        ign0 = synth.centre_ignition(land.veg)
        beta = np.asarray(synth.TRUTH_BETA, np.float64)
        F = oracle.Features(land)
        _, tb = F.simulate(beta, ign0, synth.TARGET_SEED)
        target = tb >= 0
        ctx = fire.Context(0)
        m = ctx.landscape_upload(land)
        m.target_upload(target)
        LH = LW = p["lattice"]
        reps, seed = p["replicates"], 7
        fm, cells, xy = fire.ignition_search(ctx, m, beta, LH, LW, reps, seed,
                                             kind=fire.FITNESS_JACCARD,
                                             cutoff=0.3)
        # the same 65,536 simulations as one batch
        cl = cells.reshape(-1, 2)
        n = LH * LW * reps
        params = np.tile(beta, (n, 1))
        ign = np.repeat(cl, reps, axis=0).astype(np.int32)
        seeds = np.arange(seed, seed + n, dtype=np.uint64)
        res, _ = m.simulate_batch(params, ign, seeds)
        m.free()
        ctx.close()
        rng = np.random.default_rng(3)
        picks = sorted(set(rng.integers(0, n, 10).tolist()) | {0, n - 1})
        checked = pool.map(_run_ign, [(beta, tuple(ign[i]), int(seeds[i]),
                                       target) for i in picks], chunksize=1)
    finally:
        pool.close()
        pool.join()
    for i, o in zip(picks, checked):
        for k in ("burnt", "inter", "target", "steps", "status", "trials"):
            assert int(res[k][i]) == o[k], (i, k)
    # candidate cells: the burnable burnt cell nearest each lattice point
    # (squared distance, ties to the lower row-major index)
    rows, cols = np.nonzero(target & (land.veg != 0))
    r0, r1 = np.nonzero(target)[0].min(), np.nonzero(target)[0].max()
    c0, c1 = np.nonzero(target)[1].min(), np.nonzero(target)[1].max()
    for a in range(LH):
        for b in range(LW):
            R = r0 + ((2 * a + 1) * (r1 - r0 + 1)) // (2 * LH)
            C = c0 + ((2 * b + 1) * (c1 - c0 + 1)) // (2 * LW)
            d = (rows - R) ** 2 + (cols - C) ** 2
            best = np.flatnonzero(d == d.min())
            k = best[np.argmin(rows[best] * W + cols[best])]
            assert cells[a, b].tolist() == [rows[k], cols[k]], (a, b)
    # fitness map: replicate means (index order) of the batch's fitness
    f = np.array([oracle.fitness(int(r["burnt"]), int(r["inter"]),
                                 int(r["target"]), fire.FITNESS_JACCARD)
                  for r in res])
    want = np.zeros(LH * LW)
    for c in range(LH * LW):
        s = 0.0
        for v in f[c * reps:(c + 1) * reps]:
            s = s + v
        want[c] = s / reps
    assert np.array_equal(fm.reshape(-1), want)


def test_maximum_grid(env):
    """A 4096 x 4096 map, exactly FIRE_MAX_TILES tiles: fires from the four
    corners (the first and last tiles), a certain fire across the centre
    tile boundary and one that dies out on its own, each against the
    oracle's burn-step map and counts (the target covers every tile, so the
    final sweep's counts check all of them).  One tile row more is refused.
    The oracle sweeps the whole grid every step (about 0.2 s per step),
    hence the step caps."""
    from paper_1701_03549_gb300 import fire

    seed = 4242
    pool = _pool(_init_max, (seed,), len(MAX_SIMS))   # before any GPU call
    try:
        land, target = _max_land(seed)
        ctx = fire.Context(0)
        with pytest.raises(fire.FireError):
            z = np.zeros((MAX_HW + 32, MAX_HW), np.float32)
            ctx.maps_upload(np.ones(z.shape, np.uint8), z, z, z, z)
        m = ctx.landscape_upload(land)
        m.target_upload(target)
        params = np.array([s[0] for s in MAX_SIMS], np.float64)
        ign = np.array([s[1] for s in MAX_SIMS], np.int32)
        seeds = np.array([s[2] for s in MAX_SIMS], np.uint64)
        got = []
        for k, (_, _, _, cap) in enumerate(MAX_SIMS):
            r, bs = m.simulate_batch(params[k:k + 1], ign[k:k + 1],
                                     seeds[k:k + 1], want_steps=True,
                                     max_steps=cap)
            flat = bs[0].ravel()
            idx = np.flatnonzero(flat >= 0)
            unburnt = flat[flat < 0]
            veg0 = land.veg.ravel()[flat < 0] == 0
            assert np.array_equal(unburnt, np.where(veg0, -2, -1)), k
            got.append((r[0], idx, flat[idx]))
        m.free()
        ctx.close()
        want = pool.map(_run_max, range(len(MAX_SIMS)), chunksize=1)
    finally:
        pool.close()
        pool.join()
    for k, ((r, idx, val), (o, oidx, oval)) in enumerate(zip(got, want)):
        for f in ("burnt", "inter", "target", "steps", "status", "trials"):
            assert int(r[f]) == o[f], (k, f, int(r[f]), o[f])
        assert np.array_equal(idx, oidx) and np.array_equal(val, oval), k
    assert all(g[0]["target"] == int(target.sum()) for g in got)
