"""GPU parity of uneven multi-map batches (one persistent launch over maps of
different sizes), of their CUDA-graph replay and of the autotuned launch
shape: every simulation must match the CPU oracle, and results must not
depend on batch composition, order, replay or launch shape."""
import numpy as np
import pytest

from paper_1701_03549_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("burnt", "inter", "target", "steps", "status", "trials")


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


def _batch(lands, n, seed):
    rng = np.random.default_rng(seed)
    mi = rng.integers(0, len(lands), n).astype(np.int32)
    params = rng.normal(0.0, 3.0, (n, 5))
    params[::7] = synth.TRUTH_BETA
    ign = np.zeros((n, 2), np.int32)
    for i in range(n):
        cells = np.argwhere(lands[mi[i]].veg != 0)
        ign[i] = cells[rng.integers(0, len(cells))]
    seeds = rng.integers(1, 2 ** 63, n, dtype=np.uint64)
    return mi, params, ign, seeds


@pytest.fixture(scope="module")
def uneven(env):
    torch, fire, oracle, ctx = env
    shapes = [(37, 61), (64, 64), (100, 33), (150, 90), (33, 200)]
    lands = [synth.landscape(H, W, seed=20 + j, wind_seed=20 + j)
             for j, (H, W) in enumerate(shapes)]
    maps = [ctx.landscape_upload(L) for L in lands]
    rng = np.random.default_rng(9)
    targets = [rng.random(L.veg.shape) < 0.2 for L in lands]
    for m, tg in zip(maps, targets):
        m.target_upload(tg)
    yield lands, maps, targets
    for m in maps:
        m.free()


def test_multi_matches_oracle_and_single_map_batches(env, uneven):
    torch, fire, oracle, ctx = env
    lands, maps, targets = uneven
    mi, params, ign, seeds = _batch(lands, 240, 1)
    res = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds)
    feats = [oracle.Features(L) for L in lands]
    for i in range(len(mi)):
        o, _ = feats[mi[i]].simulate(params[i], tuple(ign[i]), int(seeds[i]),
                                     target=targets[mi[i]], want_steps=False)
        for k in FIELDS:
            assert int(res[k][i]) == o[k], (i, k)
    for j, m in enumerate(maps):
        sel = np.flatnonzero(mi == j)
        r, _ = m.simulate_batch(params[sel], ign[sel], seeds[sel])
        assert np.array_equal(r, res[sel])


def test_multi_graph_replay_with_new_inputs(env, uneven):
    torch, fire, oracle, ctx = env
    lands, maps, targets = uneven
    dev = torch.device("cuda", 0)
    n = 300
    mi, params, ign, seeds = _batch(lands, n, 2)
    t_mi = torch.tensor(mi, device=dev)
    t_p = torch.tensor(params, dtype=torch.float64, device=dev)
    t_g = torch.tensor(ign, device=dev)
    t_s = torch.tensor(seeds.view(np.int64), device=dev)
    out = torch.zeros((n, 6), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    for rep in range(3):
        if rep:
            seeds = seeds + np.uint64(1000 + rep)
            t_s.copy_(torch.tensor(seeds.view(np.int64), device=dev))
            torch.cuda.synchronize()
        fire.fire_simulate_multi(ctx, maps, t_mi, t_p, t_g, t_s, device=True,
                                 out=out, graph=True, sync=True)
        want = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds)
        assert np.array_equal(fire.results_view(out), want), rep
    # the same buffers with the one-uniform-per-cell rule: a new graph, not
    # a replay of the per-neighbour one
    fire.fire_simulate_multi(ctx, maps, t_mi, t_p, t_g, t_s, device=True,
                             out=out, graph=True, sync=True, cell_uniform=True)
    want = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds,
                                    cell_uniform=True)
    assert np.array_equal(fire.results_view(out), want)
    assert not np.array_equal(
        want, fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds))


def test_multi_graph_after_a_map_is_replaced(env):
    """A freed map's memory can come back for a new map of another shape
    (whether it does is up to the allocator): a graph call on the new map
    must give the new map's results, never a replay of the old launch."""
    torch, fire, oracle, ctx = env
    dev = torch.device("cuda", 0)
    results = []
    for shape in ((40, 40), (150, 170)):
        land = synth.landscape(*shape, seed=9, wind_seed=9)
        m = ctx.landscape_upload(land)
        mi, params, ign, seeds = _batch([land], 64, 8)
        t = [torch.tensor(mi, device=dev),
             torch.tensor(params, dtype=torch.float64, device=dev),
             torch.tensor(ign, device=dev),
             torch.tensor(seeds.view(np.int64), device=dev)]
        out = torch.zeros((64, 6), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        fire.fire_simulate_multi(ctx, [m], t[0], t[1], t[2], t[3], device=True,
                                 out=out, graph=True, sync=True)
        want = fire.fire_simulate_multi(ctx, [m], mi, params, ign, seeds)
        assert np.array_equal(fire.results_view(out), want), shape
        m.free()


def test_multi_reports_bad_map_index(env, uneven):
    torch, fire, oracle, ctx = env
    lands, maps, targets = uneven
    mi, params, ign, seeds = _batch(lands, 20, 3)
    bad = mi.copy()
    bad[4] = len(maps)
    with pytest.raises(fire.FireError) as e:
        fire.fire_simulate_multi(ctx, maps, bad, params, ign, seeds)
    assert e.value.code == fire.FIRE_EINVAL
    dev = torch.device("cuda", 0)
    out = torch.zeros((20, 6), dtype=torch.int32, device=dev)
    args = [torch.tensor(a, device=dev) for a in (bad, ign)]
    t_p = torch.tensor(params, dtype=torch.float64, device=dev)
    t_s = torch.tensor(seeds.view(np.int64), device=dev)
    torch.cuda.synchronize()
    fire.fire_simulate_multi(ctx, maps, args[0], t_p, args[1], t_s,
                             device=True, out=out, sync=True)
    r = fire.results_view(out)
    assert r["status"][4] == fire.STATUS_BAD_MAP
    want = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds)
    assert np.array_equal(np.delete(r, 4), np.delete(want, 4))


def test_autotuned_shape_gives_identical_results(env, uneven):
    torch, fire, oracle, ctx = env
    lands, maps, targets = uneven
    mi, params, ign, seeds = _batch(lands, 400, 4)
    before = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds)
    best = fire.fire_autotune(ctx, maps, mi, params, ign, seeds)
    assert best["warps_per_block"] > 0 and best["ms"] > 0
    after = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds)
    assert np.array_equal(before, after)


def test_autotune_in_longest_first_order(env, uneven):
    """Tuning one map in longest-first order (host and device arguments)
    records a shape that leaves fire_simulate_batch's results unchanged;
    longest-first tuning over several maps is rejected."""
    torch, fire, oracle, ctx = env
    lands, maps, targets = uneven
    m = maps[1]
    mi, params, ign, seeds = _batch(lands[1:2], 300, 6)
    before, _ = m.simulate_batch(params, ign, seeds, longest_first=True)
    best = fire.fire_autotune(ctx, [m], None, params, ign, seeds,
                              longest_first=True)
    assert best["warps_per_block"] > 0 and best["ms"] > 0
    after, _ = m.simulate_batch(params, ign, seeds, longest_first=True)
    assert np.array_equal(before, after)
    dev = torch.device("cuda")
    best = fire.fire_autotune(ctx, [m], None, torch.tensor(params, device=dev),
                              torch.tensor(ign, device=dev),
                              torch.tensor(seeds.view(np.int64), device=dev),
                              device=True, longest_first=True)
    assert best["warps_per_block"] > 0
    with pytest.raises(fire.FireError):
        fire.fire_autotune(ctx, maps, mi, params, ign, seeds,
                           longest_first=True)


def test_multi_with_a_global_state_map(env):
    """A 1024 x 1024 map (state beyond shared memory) in the same launch as
    small maps: each simulation equals its single-map batch result."""
    torch, fire, oracle, ctx = env
    lands = [synth.landscape(1024, 1024, seed=3, wind_seed=3),
             synth.landscape(64, 80, seed=4)]
    maps = [ctx.landscape_upload(L) for L in lands]
    mi, params, ign, seeds = _batch(lands, 24, 5)
    res = fire.fire_simulate_multi(ctx, maps, mi, params, ign, seeds)
    for j, m in enumerate(maps):
        sel = np.flatnonzero(mi == j)
        r, _ = m.simulate_batch(params[sel], ign[sel], seeds[sel])
        assert np.array_equal(r, res[sel])
    big = np.flatnonzero(mi == 0)[:2]
    F = oracle.Features(lands[0])
    for i in big:
        o, _ = F.simulate(params[i], tuple(ign[i]), int(seeds[i]),
                          want_steps=False)
        for k in FIELDS:
            assert int(res[k][i]) == o[k], (i, k)
    for m in maps:
        m.free()
