"""GPU parity of the genetic-algorithm layer (Appendix B): ga_step and the
replicate mean against the oracle, bit for bit, and a whole GA run driven by
the library against the same run driven by the oracle."""
import numpy as np
import pytest

from paper_1701_03549_gb300 import synth, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    oracle.build()
    from paper_1701_03549_gb300 import fire

    ctx = fire.Context(0)
    yield torch, fire, oracle, ctx
    ctx.close()


@pytest.mark.parametrize("P,G", [(256, 5), (257, 5), (2, 5), (3, 7), (1, 5),
                                 (64, 1), (100, 2)])
def test_ga_step_matches_oracle(env, P, G):
    torch, fire, oracle, ctx = env
    rng = np.random.default_rng(P * 31 + G)
    genes = rng.normal(0, 8, (P, G))
    f = rng.random(P)
    f[rng.random(P) < 0.1] = np.nan
    f[rng.random(P) < 0.2] = 0.5
    lo, hi = np.full(G, -30.0), np.full(G, 30.0)
    for g, NG, seed in ((0, 50, 1), (17, 50, 2 ** 40 + 3), (49, 50, 7)):
        got = fire.ga_step(ctx, genes, f, g, NG, seed, lo, hi)
        want = oracle.ga_step(genes, f, g, NG, seed, lo, hi)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_ga_step_rejects_overlapping_genes(env):
    """Children are written while parents are read: an output buffer that
    overlaps the input is an error, not a race."""
    torch, fire, oracle, ctx = env
    dev = torch.device("cuda")
    genes = torch.zeros((8, 5), dtype=torch.float64, device=dev)
    f = torch.zeros(8, dtype=torch.float64, device=dev)
    lo = torch.full((5,), -30.0, dtype=torch.float64, device=dev)
    hi = torch.full((5,), 30.0, dtype=torch.float64, device=dev)
    with pytest.raises(fire.FireError):
        fire.ga_step(ctx, genes, f, 0, 10, 1, lo, hi, device=True, out=genes)
    with pytest.raises(fire.FireError):
        fire.ga_step(ctx, genes[:6], f[:6], 0, 10, 1, lo, hi, device=True,
                     out=genes[2:])
    out = torch.empty_like(genes)
    fire.ga_step(ctx, genes, f, 0, 10, 1, lo, hi, device=True, out=out)
    ctx.sync()


def test_group_mean_matches_oracle(env):
    torch, fire, oracle, ctx = env
    v = np.random.default_rng(1).normal(0, 10, 256 * 16)
    assert np.array_equal(fire.fire_group_mean(ctx, v, 16),
                          oracle.group_mean(v, 16))


def test_group_mean_rejects_overlapping_device_buffers(env):
    torch, fire, oracle, ctx = env
    v = torch.arange(64, dtype=torch.float64, device="cuda")
    with pytest.raises(fire.FireError):
        fire.fire_group_mean(ctx, v, 4, device=True, out=v)
    with pytest.raises(fire.FireError):
        fire.fire_group_mean(ctx, v[:32], 4, device=True, out=v[30:38])
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    fire.fire_group_mean(ctx, v, 4, device=True, out=out)
    ctx.sync()
    want = v.view(16, 4).cpu().numpy().sum(axis=1) / 4
    assert np.array_equal(out.cpu().numpy(), want)


def test_ga_run_matches_oracle_driven_run(env):
    """Four generations of population 8 x 2 replicates on a small map: every
    generation's population and fitness must equal those of the same GA run
    with the oracle's simulation, fitness, averaging and GA step."""
    torch, fire, oracle, ctx = env
    from paper_1701_03549_gb300 import calibrate

    land = synth.landscape(48, 56, seed=31, wind_seed=31)
    ign = synth.centre_ignition(land.veg)
    F = oracle.Features(land)
    _, target = workloads.pick_target(
        lambda s: F.simulate(synth.TRUTH_BETA, ign, s)[1] >= 0,
        int(F.burnable.sum()))
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    P, R, NG = 8, 2, 4
    hist = calibrate.run_ga(ctx, m, ign, pop=P, reps=R, generations=NG,
                            ga_seed=11, sim_seed=5)
    genes = np.clip(synth.gauss_population(P, 11), -30, 30)
    lo, hi = np.full(5, -30.0), np.full(5, 30.0)
    for g in range(NG):
        seeds = calibrate.sim_seeds(5, g, P, R)
        fit = []
        for i in range(P * R):
            o, _ = F.simulate(genes[i // R], ign, int(seeds[i]), target=target,
                              want_steps=False)
            fit.append(oracle.fitness(o["burnt"], o["inter"], o["target"], 1))
        f = oracle.group_mean(np.asarray(fit), R)
        assert np.array_equal(hist.params[g], genes), g
        assert np.array_equal(hist.fitness[g], f), g
        genes = oracle.ga_step(genes, f, g, NG, 11, lo, hi)
    m.free()


def test_multi_scar_ga_run_matches_oracle_driven_run(env):
    """Three generations of population 6 fitted to three scars at once (two
    ignitions on one map, one on a map of another size) x 2 replicates:
    every generation's population and fitness equal those of the same run
    with the oracle's simulation (each simulation against its own scar's
    target), fitness, averaging over scars and replicates, and GA step."""
    torch, fire, oracle, ctx = env
    from paper_1701_03549_gb300 import calibrate

    lands = [synth.landscape(48, 56, seed=31, wind_seed=31),
             synth.landscape(48, 56, seed=31, wind_seed=31),
             synth.landscape(40, 70, seed=32, wind_seed=32)]
    ignitions = [synth.centre_ignition(lands[0].veg),
                 tuple(int(v) for v in np.argwhere(lands[1].veg != 0)[300]),
                 synth.centre_ignition(lands[2].veg)]
    Fs, targets, maps = [], [], []
    for land, ign in zip(lands, ignitions):
        F = oracle.Features(land)
        _, target = workloads.pick_target(
            lambda s, F=F, ign=ign: F.simulate(synth.TRUTH_BETA, ign, s)[1] >= 0,
            int(F.burnable.sum()))
        m = ctx.landscape_upload(land)
        m.target_upload(target)
        Fs.append(F)
        targets.append(target)
        maps.append(m)
    P, R, NG, K = 6, 2, 3, len(maps)
    hist = calibrate.run_ga_multi(ctx, maps, ignitions, pop=P, reps=R,
                                  generations=NG, ga_seed=13, sim_seed=7)
    genes = np.clip(synth.gauss_population(P, 13), -30, 30)
    lo, hi = np.full(5, -30.0), np.full(5, 30.0)
    scar = calibrate.scar_layout(P, K, R)
    for g in range(NG):
        seeds = calibrate.sim_seeds(7, g, P, K * R)
        fit = []
        for j in range(P * K * R):
            k = int(scar[j])
            o, _ = Fs[k].simulate(genes[j // (K * R)], ignitions[k],
                                  int(seeds[j]), target=targets[k],
                                  want_steps=False)
            fit.append(oracle.fitness(o["burnt"], o["inter"], o["target"], 1))
        f = oracle.group_mean(np.asarray(fit), K * R)
        assert np.array_equal(hist.params[g], genes), g
        assert np.array_equal(hist.fitness[g], f), g
        genes = oracle.ga_step(genes, f, g, NG, 13, lo, hi)
    for m in maps:
        m.free()


def test_ga_improves_fitness_on_a_synthetic_scar(env):
    torch, fire, oracle, ctx = env
    from paper_1701_03549_gb300 import calibrate

    land = synth.landscape(128, 128, seed=1)
    ign = synth.centre_ignition(land.veg)
    m = ctx.landscape_upload(land)
    _, bs = m.simulate_batch([synth.TRUTH_BETA], [ign], [synth.TARGET_SEED + 1],
                             want_steps=True)
    m.target_upload(bs[0] >= 0)
    hist = calibrate.run_ga(ctx, m, ign, pop=128, reps=4, generations=15,
                            ga_seed=3, sim_seed=9)
    first, last = hist.fitness[0], hist.fitness[-1]
    assert np.nanmean(last) < np.nanmean(first)
    assert np.nanmin(last) <= np.nanmin(first) + 0.05
    est = calibrate.ensemble(*hist.all(), keep=64)
    assert est["size"] == 64 and np.all(np.isfinite(est["mean"]))
    m.free()


def test_sharded_evaluation_on_one_rank_equals_evaluate(env):
    """The sharded path (split simulations, gathered results, fitness on the
    device) gives the same replicate means as the single-call path."""
    torch, fire, oracle, ctx = env
    from paper_1701_03549_gb300 import calibrate

    land = synth.landscape(96, 96, seed=6)
    m = ctx.landscape_upload(land)
    ign = synth.centre_ignition(land.veg)
    _, bs = m.simulate_batch(np.asarray([synth.TRUTH_BETA]),
                             np.asarray([ign], np.int32),
                             np.asarray([9], np.uint64), want_steps=True)
    m.target_upload(bs[0] >= 0)
    genes = torch.tensor(synth.gauss_population(12, 3), device="cuda")
    seeds = calibrate.sim_seeds(5, 0, 12, 4)
    a = calibrate.evaluate(ctx, m, genes, ign, seeds, 4,
                           fire.FITNESS_JACCARD, torch)
    b = calibrate.evaluate_sharded(ctx, m, genes, ign, seeds, 4,
                                   fire.FITNESS_JACCARD, torch, 0, 1)
    assert torch.equal(a, b)
    m.free()


def test_snap_ignitions_match_the_oracle(env):
    """Ignition cells of coordinate genes against the oracle's nearest-cell
    rule on a map with non-burnable cells inside the scar: points inside,
    outside (clamped), exactly half-way between cells, NaN, and both
    host and device buffers; reps copies per individual."""
    torch, fire, oracle, ctx = env
    land = synth.landscape(70, 90, seed=12, wind_seed=12)
    F = oracle.Features(land)
    ign = synth.centre_ignition(land.veg)
    _, tb = F.simulate(synth.TRUTH_BETA, ign, synth.TARGET_SEED)
    target = tb >= 0
    target[5:9, 5:9] = True               # a second patch, partly blocked
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    rng = np.random.default_rng(4)
    n, G, reps = 300, 7, 3
    genes = rng.normal(0, 5, (n, G))
    genes[:, 5] = rng.uniform(-20, 110, n)
    genes[:, 6] = rng.uniform(-20, 90, n)
    genes[:40, 5] = np.floor(genes[:40, 5]) + 0.5
    genes[40:60, 6] = np.floor(genes[40:60, 6]) + 0.5
    genes[60, 5:] = np.nan
    got = fire.fire_snap_ignitions(ctx, m, genes, 5, 6, reps)
    want = np.array([F.snap_ignition(target, genes[i, 5], genes[i, 6])
                     for i in range(n)], np.int32)
    assert np.array_equal(got, np.repeat(want, reps, axis=0))
    gd = torch.tensor(genes, device="cuda")
    out = torch.full((n * reps, 2), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    fire.fire_snap_ignitions(ctx, m, gd, 5, 6, reps, device=True, out=out)
    assert np.array_equal(out.cpu().numpy(), got)
    m.free()


def test_seven_gene_ga_run_matches_oracle_driven_run(env):
    """The variable-ignition GA (Sec. 3, Table 3: x and y as genes 6 and 7):
    four generations of population 16 x 2 replicates, every generation's
    population and fitness equal to the same run with the oracle's snapping,
    simulation, fitness, averaging and seven-gene GA step."""
    torch, fire, oracle, ctx = env
    from paper_1701_03549_gb300 import calibrate

    land = synth.landscape(48, 56, seed=33, wind_seed=33)
    ign = synth.centre_ignition(land.veg)
    F = oracle.Features(land)
    _, target = workloads.pick_target(
        lambda s: F.simulate(synth.TRUTH_BETA, ign, s)[1] >= 0,
        int(F.burnable.sum()))
    burnable = land.veg != 0
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    P, R, NG = 16, 2, 4
    hist = calibrate.run_ga_ignition(ctx, m, target, burnable, pop=P, reps=R,
                                     generations=NG, ga_seed=13, sim_seed=7)
    genes = calibrate.initial_population_7(target, burnable, P, 13)
    H, W = land.veg.shape
    lo = np.array([-30.0] * 5 + [0.0, 0.0])
    hi = np.array([30.0] * 5 + [W - 1.0, H - 1.0])
    for g in range(NG):
        seeds = calibrate.sim_seeds(7, g, P, R)
        fit = []
        for i in range(P * R):
            cell = F.snap_ignition(target, genes[i // R, 5], genes[i // R, 6])
            o, _ = F.simulate(genes[i // R, :5], cell, int(seeds[i]),
                              target=target, want_steps=False)
            fit.append(oracle.fitness(o["burnt"], o["inter"], o["target"], 1))
        f = oracle.group_mean(np.asarray(fit), R)
        assert np.array_equal(hist.params[g], genes), g
        assert np.array_equal(hist.fitness[g], f), g
        genes = oracle.ga_step(genes, f, g, NG, 13, lo, hi)
    # the ignition genes stay on the grid
    last = hist.params[-1]
    assert np.all((last[:, 5] >= 0) & (last[:, 5] <= W - 1))
    assert np.all((last[:, 6] >= 0) & (last[:, 6] <= H - 1))
    m.free()


@pytest.mark.parametrize("genes7", [False, True, "scars"])
def test_checkpoint_resume_is_bit_identical(env, tmp_path, genes7):
    """A GA run stopped after two of five generations and resumed from its
    checkpoint ends with exactly the populations and fitness of the run that
    was never interrupted (five and seven genes, and five genes fitted to two
    scars)."""
    torch, fire, oracle, ctx = env
    from paper_1701_03549_gb300 import calibrate

    land = synth.landscape(64, 64, seed=41, wind_seed=41)
    ign = synth.centre_ignition(land.veg)
    m = ctx.landscape_upload(land)
    _, bs = m.simulate_batch(np.asarray([synth.TRUTH_BETA]),
                             np.asarray([ign], np.int32),
                             np.asarray([synth.TARGET_SEED], np.uint64),
                             want_steps=True)
    target = bs[0] >= 0
    m.target_upload(target)
    burnable = land.veg != 0
    path = str(tmp_path / "ga.npz")

    m2 = None
    if genes7 == "scars":
        ign2 = tuple(int(v) for v in np.argwhere(burnable)[500])
        m2 = ctx.landscape_upload(land)
        _, bs2 = m2.simulate_batch(np.asarray([synth.TRUTH_BETA]),
                                   np.asarray([ign2], np.int32),
                                   np.asarray([synth.TARGET_SEED], np.uint64),
                                   want_steps=True)
        m2.target_upload(bs2[0] >= 0)

    def run(**kw):
        if genes7 == "scars":
            return calibrate.run_ga_multi(ctx, [m, m2], [ign, ign2], pop=12,
                                          reps=2, generations=5, ga_seed=2,
                                          sim_seed=3, **kw)
        if genes7:
            return calibrate.run_ga_ignition(ctx, m, target, burnable, pop=12,
                                             reps=2, generations=5, ga_seed=2,
                                             sim_seed=3, **kw)
        return calibrate.run_ga(ctx, m, ign, pop=12, reps=2, generations=5,
                                ga_seed=2, sim_seed=3, **kw)

    full = run()
    part = run(checkpoint=path, stop_after=2)
    assert len(part.params) == 2
    resumed = run(checkpoint=path)
    assert len(resumed.params) == 5
    for g in range(5):
        assert np.array_equal(resumed.params[g], full.params[g]), g
        assert np.array_equal(resumed.fitness[g], full.fitness[g]), g
    m.free()
    if m2 is not None:
        m2.free()
