"""Burn-out times on the GPU (fire_simulate_burnout) against the oracle.

* burn_time = 1 everywhere: every result and burn-step map bit-identical to
  fire_simulate_batch (the paper's rule, same keyed draws), both when the call
  hands the batch to the plain kernel and in the burn-time kernel itself;
* per-fuel times: results and burn-step maps bit-identical to the oracle's
  burn-out simulation, host and device argument paths;
* step cap, bad ignition status, and host-side rejection of a zero time.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1701_03549_gb300 import fire, synth  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = fire.fire_create(0, torch.cuda.current_stream())
    yield c
    c.close()


def _per_fuel(veg, times):
    return np.asarray(times, np.uint8)[np.minimum(veg, 4)]


def _batch(L, n, seed):
    rng = np.random.default_rng(seed)
    beta = np.column_stack([rng.uniform(-3, 2, n), rng.uniform(-4, 1, n),
                            rng.uniform(-2, 4, n), rng.uniform(0, 6, n),
                            rng.uniform(-3, 3, n)])
    ign = np.tile(np.array(synth.centre_ignition(L.veg), np.int32), (n, 1))
    seeds = np.arange(1000, 1000 + n, dtype=np.uint64)
    return beta, ign, seeds


def test_unit_times_equal_the_main_kernel(ctx):
    L = synth.landscape(96, 112, seed=3, wind_seed=3)
    m = ctx.landscape_upload(L)
    beta, ign, seeds = _batch(L, 48, 1)
    r0, b0 = m.simulate_batch(beta, ign, seeds, want_steps=True)
    ones = np.ones(L.veg.shape, np.uint8)
    r1, b1 = m.simulate_burnout(beta, ign, seeds, ones, want_steps=True)
    assert np.array_equal(r0, r1)
    assert np.array_equal(b0, b1)
    # the burn-time kernel itself (a time of 2 on one non-burnable cell makes
    # the batch take it; every burnable cell still burns one step)
    rows, cols = np.nonzero(L.veg == 0)
    ones[rows[0], cols[0]] = 2
    r2, b2 = m.simulate_burnout(beta, ign, seeds, ones, want_steps=True)
    assert np.array_equal(r0, r2)
    assert np.array_equal(b0, b2)


@pytest.mark.parametrize("times", [(1, 3, 1, 2, 4), (1, 2, 2, 2, 2),
                                   (1, 1, 5, 1, 1)])
def test_per_fuel_times_match_the_oracle(ctx, oracle_mod, times):
    import oracle

    L = synth.landscape(70, 90, seed=8, wind_seed=8)
    tgt = np.zeros(L.veg.shape, bool)
    tgt[20:50, 30:70] = True
    m = ctx.landscape_upload(L)
    m.target_upload(tgt)
    bt = _per_fuel(L.veg, times)
    beta, ign, seeds = _batch(L, 20, 7)
    res, bs = m.simulate_burnout(beta, ign, seeds, bt, want_steps=True)
    F = oracle.Features(L)
    for i in range(20):
        r, b = F.simulate(beta[i], tuple(ign[i]), int(seeds[i]), target=tgt,
                          burn_time=bt)
        for k in r:
            assert int(res[i][k]) == r[k], (i, k)
        assert np.array_equal(bs[i], b), i
    # device path
    dev = torch.device("cuda")
    out = torch.zeros((20, 6), dtype=torch.int32, device=dev)
    steps = torch.zeros((20,) + L.veg.shape, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    m.simulate_burnout(torch.tensor(beta, device=dev),
                       torch.tensor(ign, device=dev),
                       torch.tensor(seeds.view(np.int64), device=dev),
                       torch.tensor(bt, device=dev), want_steps=True,
                       device=True, out=out, burn_step=steps, sync=True)
    assert np.array_equal(fire.results_view(out), res)
    assert np.array_equal(steps.cpu().numpy(), bs)


def test_cap_status_and_errors(ctx, oracle_mod):
    import oracle

    L = synth.uniform_landscape(40, 40)
    L.veg[5, 5] = 0
    m = ctx.landscape_upload(L)
    bt = np.full(L.veg.shape, 3, np.uint8)
    res, _ = m.simulate_burnout(np.array([[1000.0, 0, 0, 0, 0]]),
                                np.array([[20, 20]], np.int32),
                                np.array([5], np.uint64), bt, max_steps=4)
    F = oracle.Features(L)
    r, _ = F.simulate([1000.0, 0, 0, 0, 0], (20, 20), 5, max_steps=4,
                      burn_time=bt)
    assert res[0]["steps"] == r["steps"] == 4
    assert res[0]["status"] & fire.STATUS_STEP_CAP and r["status"] & 2
    assert res[0]["burnt"] == r["burnt"]
    bad = bt.copy()
    bad[3, 3] = 0
    with pytest.raises(fire.FireError):
        m.simulate_burnout(np.zeros((1, 5)), np.array([[20, 20]], np.int32),
                           np.array([1], np.uint64), bad)
    with pytest.raises(fire.FireError):
        m.simulate_burnout(np.zeros((1, 5)), np.array([[5, 5]], np.int32),
                           np.array([1], np.uint64), bt)
    # device arguments: a bad ignition is a status bit, not an error
    dev = torch.device("cuda")
    out = torch.zeros((1, 6), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    m.simulate_burnout(torch.zeros((1, 5), dtype=torch.float64, device=dev),
                       torch.tensor([[5, 5]], dtype=torch.int32, device=dev),
                       torch.ones(1, dtype=torch.int64, device=dev),
                       torch.tensor(bt, device=dev), device=True, out=out,
                       sync=True)
    assert fire.results_view(out)[0]["status"] & fire.STATUS_BAD_IGNITION


def test_per_cell_times_across_tiles(ctx, oracle_mod):
    """Per-cell burn times 1..12 on a 130 x 161 map (5 x 6 tiles, ragged
    last row and column): fires started on tile corners and edges keep
    cells burning across tile boundaries for many steps; results and
    burn-step maps against the oracle, also under a launch shape with more
    blocks per SM and a small candidate queue (overflow path)."""
    import oracle

    L = synth.landscape(130, 161, seed=21, wind_seed=21)
    rng = np.random.default_rng(5)
    bt = rng.integers(1, 13, L.veg.shape).astype(np.uint8)
    starts = [(31, 31), (32, 63), (64, 0), (95, 160), (129, 96), (0, 127)]
    for r, c in starts:
        L.veg[r, c] = 2
    tgt = rng.random(L.veg.shape) < 0.3
    m = ctx.landscape_upload(L)
    m.target_upload(tgt)
    n = len(starts) * 2
    beta = np.array([[0.5, -1.0, 0.5, 1.5, -0.5], [-1.5, 0.0, 0.5, 2.5, 1.0]]
                    * len(starts))
    ign = np.array([s for s in starts for _ in range(2)], np.int32)
    seeds = np.arange(77, 77 + n, dtype=np.uint64)
    F = oracle.Features(L)
    want = [F.simulate(beta[i], tuple(ign[i]), int(seeds[i]), target=tgt,
                       burn_time=bt) for i in range(n)]
    for shape in ((0, 0, 0, 0), (2, 12, 64, 0)):
        ctx.set_launch(*shape)
        try:
            res, bs = m.simulate_burnout(beta, ign, seeds, bt, want_steps=True)
        finally:
            ctx.set_launch(0, 0)
        for i, (r, b) in enumerate(want):
            for k in r:
                assert int(res[i][k]) == r[k], (shape, i, k)
            assert np.array_equal(bs[i], b), (shape, i)
    assert max(r["steps"] for r, _ in want) > 40


def test_long_burn_times(ctx, oracle_mod):
    """Burn times up to the largest accepted (250) on a small map: cells keep
    trying their neighbours for hundreds of steps; step cap on such a fire."""
    import oracle

    L = synth.landscape(40, 48, seed=22, wind_seed=22)
    g = synth.centre_ignition(L.veg)
    L.veg[g] = 1                       # the ignition cell burns 250 steps
    bt = np.where(L.veg == 1, 250, 37).astype(np.uint8)
    m = ctx.landscape_upload(L)
    beta = np.array([[-4.0, 1.0, 0.0, 0.5, 0.0], [-3.0, -1.0, 0.5, 1.0, 0.0]])
    ign = np.tile(np.array(g, np.int32), (2, 1))
    seeds = np.array([3, 4], np.uint64)
    F = oracle.Features(L)
    for cap in (0, 120):
        res, bs = m.simulate_burnout(beta, ign, seeds, bt, want_steps=True,
                                     max_steps=cap)
        for i in range(2):
            r, b = F.simulate(beta[i], tuple(ign[i]), int(seeds[i]),
                              burn_time=bt, max_steps=cap)
            for k in r:
                assert int(res[i][k]) == r[k], (cap, i, k)
            assert np.array_equal(bs[i], b), (cap, i)
            if cap == 0:
                assert r["steps"] >= 250
