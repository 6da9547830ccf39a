"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Covariates, thresholds and trajectories must match bit for bit; the
single-precision screen's probabilities must agree with double precision to
1e-6 absolute and never change a decision.
"""
import os

import numpy as np
import pytest

from paper_1701_03549_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

TRUTH = np.asarray(synth.TRUTH_BETA)


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1701_03549_gb300 import fire

    c = fire.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _maps(shape_seed_list):
    for (H, W), seed, wind_seed in shape_seed_list:
        yield synth.landscape(H, W, seed=seed, wind_seed=wind_seed)


SHAPES = [((1, 1), 1, None), ((1, 2), 2, None), ((3, 3), 3, 3),
          ((37, 61), 4, 4), ((64, 64), 5, None), ((100, 33), 6, 6),
          ((128, 128), 1, None)]


def _compare_features(ctx, orc, land):
    F = orc.Features(land)
    m = ctx.landscape_upload(land)
    g = m.features()
    assert np.array_equal(g["psi"].view(np.uint32), F.psi.view(np.uint32))
    assert np.array_equal(g["sig"].view(np.uint32), F.sig.view(np.uint32))
    assert np.array_equal(g["cw"].view(np.uint32), F.cw.view(np.uint32))
    assert np.array_equal(g["sw"].view(np.uint32), F.sw.view(np.uint32))
    want = (F.up.astype(np.uint16) | (F.forest.astype(np.uint16) << 8)
            | (F.burnable.astype(np.uint16) << 9))
    assert np.array_equal(g["flags"], want)
    return F, m


def test_covariates_match_oracle(ctx, orc):
    for land in _maps(SHAPES):
        _compare_features(ctx, orc, land)


def test_thresholds_match_oracle_exactly(ctx, orc):
    rng = np.random.default_rng(1)
    betas = [TRUTH, np.zeros(5), [1000.0, 0, 0, 0, 0], [-1000.0, 0, 0, 0, 0]]
    betas += list(rng.normal(0, 5, (4, 5))) + list(rng.uniform(-30, 30, (4, 5)))
    for land in _maps([((37, 61), 4, 4), ((128, 128), 1, None)]):
        F, m = _compare_features(ctx, orc, land)
        for b in betas:
            assert np.array_equal(m.thresholds(b).astype(np.uint64),
                                  F.thresholds(b))


def test_single_precision_probabilities_within_1e6(ctx, orc):
    """The screen's FP32 probability agrees with the double-precision one
    (which equals the oracle's thresholds) within 1e-6 for coefficients in the
    GA's range [-30, 30], and within its stated bound 7.5e-9 |b3| + 5e-7 for
    coefficients up to 200."""
    rng = np.random.default_rng(2)
    worst, worst_ratio = 0.0, 0.0
    for land in _maps([((64, 64), 5, 5), ((128, 128), 1, None)]):
        m = ctx.landscape_upload(land)
        F = orc.Features(land)
        for b in ([TRUTH] + list(rng.uniform(-30, 30, (8, 5))) +
                  list(rng.uniform(-200, 200, (3, 5)))):
            p32, p64 = m.probabilities(b)
            # the double-precision values are the oracle's
            T = F.thresholds(b).astype(np.float64)
            assert np.all(np.floor(p64 * 2.0 ** 32) == T)
            err = float(np.abs(p32.astype(np.float64) - p64).max())
            if np.abs(b).max() <= 30:
                worst = max(worst, err)
            worst_ratio = max(worst_ratio, err / (7.5e-9 * abs(b[3]) + 5e-7))
    assert worst <= 1e-6, worst
    assert worst_ratio < 1.0, worst_ratio


def test_screen_never_flips_a_decision(ctx):
    from paper_1701_03549_gb300 import fire

    r = fire.fire_screen_selftest(ctx, 1 << 30, 12345)
    assert r["cases"] == 1 << 30
    assert r["flips"] == 0
    assert r["max_err_ratio"] < 1.0
    # the double-precision fallback stays rare for uniform draws
    assert r["fallbacks"] < r["cases"]


def test_philox_blocks_match_oracle(ctx, orc):
    from paper_1701_03549_gb300 import fire

    rng = np.random.default_rng(3)
    for _ in range(8):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        ctr[0] = min(int(ctr[0]), 2 ** 32 - 300)
        got = fire.fire_philox_blocks(ctx, 256, ctr, key)
        for i in range(0, 256, 17):
            c = ctr.copy()
            c[0] += i
            assert np.array_equal(got[i], orc.philox4x32_10(c, key))


def test_philox_matches_curand_raw_blocks(ctx, orc, tmp_path):
    """Known-answer check of Philox4x32-10 against a third-party
    implementation: cuRAND's public raw block function, built here into a
    small test library.  The oracle's generator and the library's must both
    equal it on random counters and keys."""
    import ctypes
    import subprocess

    from paper_1701_03549_gb300 import build, fire

    src = os.path.join(os.path.dirname(__file__), "curand_philox_ref.cu")
    so = str(tmp_path / "libcurand_ref.so")
    r = subprocess.run([build._nvcc(), *build.ARCH, "-O2", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-shared", src, "-o", so],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    ref = ctypes.CDLL(so)
    n = 4096
    rng = np.random.default_rng(17)
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = 0
    key[:4] = 0
    key[4:8] = 0xFFFFFFFF
    out = np.zeros((n, 4), np.uint32)
    assert ref.curand_philox_blocks(
        n, ctr.ctypes.data_as(ctypes.c_void_p),
        key.ctypes.data_as(ctypes.c_void_p),
        out.ctypes.data_as(ctypes.c_void_p)) == 0
    for i in range(0, n, 7):
        assert np.array_equal(orc.philox4x32_10(ctr[i], key[i]), out[i]), i
    # the library's device generator on consecutive counters
    base = np.array([5, 0xDEADBEEF, 1, 0], np.uint32)
    k = np.array([0x12345678, 0x9ABCDEF0], np.uint32)
    got = fire.fire_philox_blocks(ctx, 512, base, k)
    cs = np.tile(base, (512, 1))
    cs[:, 0] += np.arange(512, dtype=np.uint32)
    ks = np.tile(k, (512, 1))
    out2 = np.zeros((512, 4), np.uint32)
    assert ref.curand_philox_blocks(
        512, np.ascontiguousarray(cs).ctypes.data_as(ctypes.c_void_p),
        np.ascontiguousarray(ks).ctypes.data_as(ctypes.c_void_p),
        out2.ctypes.data_as(ctypes.c_void_p)) == 0
    assert np.array_equal(got, out2)


def _check_batch(ctx, orc, land, params, ignitions, seeds, target=None,
                 max_steps=0, warps=0, bps=0, state=0):
    F = orc.Features(land)
    m = ctx.landscape_upload(land)
    if target is not None:
        m.target_upload(target)
    ctx.set_launch(warps, bps, 0, state)
    try:
        res, bs = m.simulate_batch(params, ignitions, seeds, want_steps=True,
                                   max_steps=max_steps)
    finally:
        ctx.set_launch(0, 0)
    for i in range(len(seeds)):
        o, obs = F.simulate(params[i], tuple(ignitions[i]), int(seeds[i]),
                            target=target, max_steps=max_steps)
        assert np.array_equal(bs[i], obs), f"trajectory {i}"
        for k in ("burnt", "inter", "target", "steps", "status", "trials"):
            assert int(res[k][i]) == o[k], (i, k, int(res[k][i]), o[k])
    return res, bs


def test_trajectories_single_fire_128(ctx, orc):
    wl = workloads.single_fire_128(replicates=64)
    F = orc.Features(wl.land)
    _, target = workloads.pick_target(
        lambda s: F.simulate(synth.TRUTH_BETA, wl.ignition, s)[1] >= 0,
        int(F.burnable.sum()))
    _check_batch(ctx, orc, wl.land, wl.params, wl.ignitions, wl.seeds,
                 target=target)


@pytest.mark.parametrize("shape,seed", [((1, 1), 1), ((1, 2), 2), ((3, 3), 3),
                                        ((37, 61), 4), ((100, 33), 6),
                                        ((33, 97), 7), ((96, 160), 8)])
def test_trajectories_ragged_grids(ctx, orc, shape, seed):
    land = synth.landscape(*shape, seed=seed, wind_seed=seed)
    rng = np.random.default_rng(seed)
    n = 24
    params = np.concatenate([rng.normal(0, 3, (n - 4, 5)),
                             [TRUTH, [1000.0, 0, 0, 0, 0],
                              [-1000.0, 0, 0, 0, 0], [2.0, 0, 0, 0, 0]]])
    burnable = np.argwhere(land.veg != 0)
    ign = burnable[rng.integers(0, len(burnable), n)].astype(np.int32)
    seeds = rng.integers(1, 2 ** 63, n, dtype=np.uint64)
    target = rng.random(shape) < 0.3
    _check_batch(ctx, orc, land, params, ign, seeds, target=target)


@pytest.mark.parametrize("shape,seed,state", [((96, 160), 21, 0),
                                              ((130, 70), 22, 2)])
def test_trajectories_saturated_thresholds(ctx, orc, shape, seed, state):
    """Parameters whose z reaches the saturated ranges of the threshold
    (z >= 37: 1 + e^-z rounds to 1, T = 2^32 and every draw succeeds;
    z <= -22.5: T = 0 and every draw fails), mixed with Uniform[-30, 30]
    draws, cases next to those bounds and magnitudes up to 2 10^6, in shared
    and global state: trajectories and counts equal the oracle's."""
    land = synth.landscape(*shape, seed=seed, wind_seed=seed)
    rng = np.random.default_rng(seed)
    edge = [[25.0, 10, 5, 8, 0], [30.0, -10, 8, 12, 3], [38.0, 0, 0, 0, 0],
            [36.9, 0, 0, 1.0, 0], [-22.0, 0, 0, 30, 0], [-5.0, 0, 0, 40, 0],
            [9.0e5, 0, 0, 0, 0], [2.0e6, 0, 0, 0, 0]]
    n = 28
    params = np.concatenate([rng.uniform(-30, 30, (n - len(edge), 5)), edge])
    burnable = np.argwhere(land.veg != 0)
    ign = burnable[rng.integers(0, len(burnable), n)].astype(np.int32)
    seeds = rng.integers(1, 2 ** 63, n, dtype=np.uint64)
    target = rng.random(shape) < 0.3
    _check_batch(ctx, orc, land, params, ign, seeds, target=target,
                 state=state)


def test_ignitions_on_edges_and_corners(ctx, orc):
    H, W = 65, 70
    land = synth.landscape(H, W, seed=11, wind_seed=11)
    land.veg[:] = np.maximum(land.veg, 1)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (31, 31), (32, 32),
           (31, 32), (32, 31), (0, 33), (64, 63)]
    n = len(pts)
    params = np.tile([1.0, -0.5, 0.5, 1.5, -1.0], (n, 1))
    _check_batch(ctx, orc, land, params, np.asarray(pts, np.int32),
                 np.arange(1, n + 1, dtype=np.uint64))


def test_p_one_and_p_zero(ctx, orc):
    land = synth.uniform_landscape(70, 75)
    res, bs = _check_batch(ctx, orc, land, np.array([[1000.0, 0, 0, 0, 0],
                                                     [-1000.0, 0, 0, 0, 0]]),
                           np.array([[20, 50], [3, 4]], np.int32),
                           np.array([5, 6], np.uint64))
    rr, cc = np.mgrid[0:70, 0:75]
    assert np.array_equal(bs[0], np.maximum(abs(rr - 20), abs(cc - 50)))
    assert res["burnt"][1] == 1 and res["steps"][1] == 1


def test_step_cap(ctx, orc):
    land = synth.uniform_landscape(40, 40)
    _check_batch(ctx, orc, land, np.array([[1000.0, 0, 0, 0, 0]] * 3),
                 np.array([[20, 20]] * 3, np.int32),
                 np.array([1, 2, 3], np.uint64), max_steps=5)


def test_launch_shape_and_batch_position_do_not_change_results(ctx, orc):
    wl = workloads.single_fire_128(replicates=48)
    m = ctx.landscape_upload(wl.land)
    ref, refbs = m.simulate_batch(wl.params, wl.ignitions, wl.seeds,
                                  want_steps=True)
    for warps, bps in ((1, 1), (2, 0), (8, 3), (16, 1)):
        ctx.set_launch(warps, bps)
        r, b = m.simulate_batch(wl.params, wl.ignitions, wl.seeds,
                                want_steps=True)
        assert np.array_equal(r, ref) and np.array_equal(b, refbs)
    ctx.set_launch(0, 0)
    perm = np.random.default_rng(0).permutation(wl.n)
    r, b = m.simulate_batch(wl.params[perm], wl.ignitions[perm],
                            wl.seeds[perm], want_steps=True)
    assert np.array_equal(r, ref[perm]) and np.array_equal(b, refbs[perm])
    one, oneb = m.simulate_batch(wl.params[7:8], wl.ignitions[7:8],
                                 wl.seeds[7:8], want_steps=True)
    assert np.array_equal(one[0], ref[7]) and np.array_equal(oneb[0], refbs[7])


@pytest.mark.parametrize("queue,state", [(64, 1), (64, 2), (200, 1), (200, 2)])
def test_queue_overflow_decides_in_phase_a(ctx, orc, queue, state):
    """A candidate queue too small for a step makes the tile's warp decide the
    candidates that did not fit itself: same trajectories, step counts and
    step-cap behaviour as the oracle (64 entries, the smallest queue accepted,
    and 200: a wide fire front on the 128 x 128 map overflows either, so most
    steps mix both paths)."""
    from paper_1701_03549_gb300 import fire

    wl = workloads.single_fire_128(replicates=24)
    rng = np.random.default_rng(queue)
    params = np.concatenate([wl.params[:12], rng.normal(0, 3, (10, 5)),
                             [[1000.0, 0, 0, 0, 0], [-0.5, 0, 0, 0, 0]]])
    n = len(params)
    ign = wl.ignitions[:n]
    seeds = wl.seeds[:n]
    F = orc.Features(wl.land)
    m = ctx.landscape_upload(wl.land)
    widest = 0   # most cells ignited in one step (each was a candidate)
    try:
        for cap in (0, 7):
            ctx.set_launch(4, 0, queue, state)
            res, bs = m.simulate_batch(params, ign, seeds, want_steps=True,
                                       max_steps=cap)
            ctx.set_launch(0, 0)
            for i in range(n):
                o, obs = F.simulate(params[i], tuple(ign[i]), int(seeds[i]),
                                    max_steps=cap)
                assert np.array_equal(bs[i], obs), (cap, i)
                for k in ("burnt", "steps", "status", "trials"):
                    assert int(res[k][i]) == o[k], (cap, i, k)
                if obs.max() > 0:
                    widest = max(widest, np.bincount(obs[obs > 0]).max())
    finally:
        ctx.set_launch(0, 0)
        m.free()
    assert widest > queue
    assert fire.STATE_SHARED == 1 and fire.STATE_GLOBAL == 2


def test_ga_generation_512_sample(ctx, orc):
    wl = workloads.ga_generation_512(population=256, replicates=16)
    idx = np.array([0, 1, 2, 17, 100, 2001, 4095])
    F = orc.Features(wl.land)
    _, target = workloads.pick_target(
        lambda s: F.simulate(synth.TRUTH_BETA, wl.ignition, s)[1] >= 0,
        int(F.burnable.sum()))
    m = ctx.landscape_upload(wl.land)
    m.target_upload(target)
    res, _ = m.simulate_batch(wl.params, wl.ignitions, wl.seeds)
    for i in idx:
        o, _ = F.simulate(wl.params[i], wl.ignition, int(wl.seeds[i]),
                          target=target, want_steps=False)
        for k in ("burnt", "inter", "target", "steps", "status", "trials"):
            assert int(res[k][i]) == o[k], (i, k)


def test_global_state_variant_1024(ctx, orc):
    """1024 x 1024 state does not fit in shared memory: the per-block global
    state buffer path must give the same trajectories."""
    land = synth.landscape(1024, 1024, seed=3, wind_seed=3)
    ign = synth.centre_ignition(land.veg)
    params = np.array([TRUTH, [-1.0, 0.5, 0.5, 3.0, -1.0]])
    _check_batch(ctx, orc, land, params, np.array([ign, ign], np.int32),
                 np.array([3, 4], np.uint64))


def test_fitness_matches_oracle(ctx, orc):
    from paper_1701_03549_gb300 import fire

    rng = np.random.default_rng(4)
    r = np.zeros(500, fire.RESULT_DTYPE)
    r["target"] = rng.integers(1, 5000, 500)
    r["burnt"] = rng.integers(1, 5000, 500)
    r["inter"] = np.minimum(r["target"], r["burnt"]) * rng.random(500)
    for kind in (0, 1):
        got = fire.fire_fitness(ctx, r, kind)
        want = [orc.fitness(int(a), int(b), int(c), kind)
                for a, b, c in zip(r["burnt"], r["inter"], r["target"])]
        assert np.array_equal(got, np.asarray(want))


def test_fitness_rejects_overlapping_device_buffers(ctx):
    import torch

    from paper_1701_03549_gb300 import fire

    res = torch.ones((12, 6), dtype=torch.int32, device="cuda")
    res[:, 0] = 2   # |A*| = 2, |A n A*| = 1, |A| = 1: delta = 1
    alias = res.view(torch.float64).view(-1)[:12]   # same bytes as res
    with pytest.raises(fire.FireError):
        fire.fire_fitness(ctx, res, 0, device=True, out=alias)
    out = torch.empty(12, dtype=torch.float64, device="cuda")
    fire.fire_fitness(ctx, res, 0, device=True, out=out)
    ctx.sync()
    assert torch.all(out == 1.0)


def test_mistyped_device_buffers_are_rejected(ctx):
    """A device buffer of the wrong dtype, size or place is refused by the
    binding before any kernel could read past its end."""
    import torch

    from paper_1701_03549_gb300 import fire

    land = synth.landscape(40, 40, seed=1)
    m = ctx.landscape_upload(land)
    n = 4
    ign = synth.centre_ignition(land.veg)
    p = torch.tensor(np.tile(TRUTH, (n, 1)), device="cuda")
    g = torch.tensor(np.tile(np.asarray(ign, np.int32), (n, 1)), device="cuda")
    s = torch.arange(n, dtype=torch.int64, device="cuda")
    out = torch.zeros((n, 6), dtype=torch.int32, device="cuda")
    for args in ((p.float(), g, s, out), (p, g.long(), s, out),
                 (p, g, s[:3], out), (p, g, s, out[:3]),
                 (p, g, s.cpu(), out), (p, g, s, out.t())):
        with pytest.raises(fire.FireError):
            m.simulate_batch(*args[:3], device=True, out=args[3], sync=True)
    assert torch.all(out == 0)
    m.simulate_batch(p, g, s, device=True, out=out, sync=True)
    assert torch.all(out[:, 0] > 0)
    m.free()


def test_empty_batches(ctx):
    """n = 0 on every batch entry point, host and device: nothing runs and
    nothing is written."""
    import torch

    from paper_1701_03549_gb300 import fire

    land = synth.landscape(40, 40, seed=2)
    m = ctx.landscape_upload(land)
    e = np.zeros((0, 5)), np.zeros((0, 2), np.int32), np.zeros(0, np.uint64)
    res, _ = m.simulate_batch(*e)
    assert res.shape == (0,)
    res, _ = m.simulate_burnout(*e, np.ones((40, 40), np.uint8))
    assert res.shape == (0,)
    assert fire.fire_simulate_multi(ctx, [m], np.zeros(0, np.int32),
                                    *e).shape == (0,)
    assert fire.fire_fitness(ctx, np.zeros(0, fire.RESULT_DTYPE)).shape == (0,)
    assert fire.fire_group_mean(ctx, np.zeros(0), 4).shape == (0,)
    d = dict(device="cuda")
    p = torch.zeros((0, 5), dtype=torch.float64, **d)
    g = torch.zeros((0, 2), dtype=torch.int32, **d)
    s = torch.zeros(0, dtype=torch.int64, **d)
    out = torch.zeros((0, 6), dtype=torch.int32, **d)
    m.simulate_batch(p, g, s, device=True, out=out, sync=True)
    m.simulate_batch_noalloc(p, g, s, out)
    fire.fire_simulate_multi(ctx, [m], torch.zeros(0, dtype=torch.int32, **d),
                             p, g, s, device=True, out=out, graph=True,
                             sync=True)
    fire.fire_fitness(ctx, out, 0, device=True,
                      out=torch.zeros(0, dtype=torch.float64, **d))
    ctx.sync()
    m.free()


def test_bad_host_ignition_is_rejected(ctx):
    from paper_1701_03549_gb300 import fire

    land = synth.landscape(40, 40, seed=1)
    land.veg[5, 5] = 0
    m = ctx.landscape_upload(land)
    for ign in ([5, 5], [40, 0], [-1, 3]):
        with pytest.raises(fire.FireError) as e:
            m.simulate_batch([[0.0] * 5], [ign], [1])
        assert e.value.code == fire.FIRE_EIGNITION
    with pytest.raises(fire.FireError) as e:
        m.simulate_batch([[np.nan, 0, 0, 0, 0]], [[1, 1]], [1])
    assert e.value.code == fire.FIRE_EINVAL
    r, _ = m.simulate_batch(np.zeros((0, 5)), np.zeros((0, 2)), np.zeros(0))
    assert r.shape == (0,)


def test_device_pointer_path_matches_host_path(ctx, orc):
    import torch

    from paper_1701_03549_gb300 import fire

    wl = workloads.single_fire_128(replicates=32)
    m = ctx.landscape_upload(wl.land)
    href, hbs = m.simulate_batch(wl.params, wl.ignitions, wl.seeds,
                                 want_steps=True)
    dev = torch.device("cuda", 0)
    p = torch.tensor(wl.params, dtype=torch.float64, device=dev)
    g = torch.tensor(wl.ignitions, dtype=torch.int32, device=dev)
    s = torch.tensor(wl.seeds.view(np.int64), dtype=torch.int64, device=dev)
    out = torch.zeros((wl.n, 6), dtype=torch.int32, device=dev)
    bs = torch.zeros((wl.n, 128, 128), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()  # the context issues work on its own stream
    m.simulate_batch(p, g, s, want_steps=True, device=True, out=out,
                     burn_step=bs, sync=True)
    assert np.array_equal(fire.results_view(out), href)
    assert np.array_equal(bs.cpu().numpy(), hbs)
    # device-side ignition check: an out-of-grid ignition is flagged per sim
    g[3, 0] = 500
    torch.cuda.synchronize()
    m.simulate_batch(p, g, s, device=True, out=out, sync=True)
    r = fire.results_view(out)
    assert r["status"][3] & fire.STATUS_BAD_IGNITION
    assert np.array_equal(np.delete(r, 3), np.delete(href, 3))


@pytest.mark.parametrize("shape,seed", [((37, 61), 4), ((128, 128), 1),
                                        ((3, 3), 3)])
def test_cell_uniform_rule_matches_oracle(ctx, orc, shape, seed):
    """The paper's one-uniform-per-cell update (FIRE_CELL_UNIFORM)."""
    land = synth.landscape(*shape, seed=seed, wind_seed=seed)
    rng = np.random.default_rng(seed + 50)
    n = 24
    params = np.concatenate([rng.normal(0, 3, (n - 3, 5)),
                             [TRUTH, [1000.0, 0, 0, 0, 0],
                              [-1000.0, 0, 0, 0, 0]]])
    burnable = np.argwhere(land.veg != 0)
    ign = burnable[rng.integers(0, len(burnable), n)].astype(np.int32)
    seeds = rng.integers(1, 2 ** 63, n, dtype=np.uint64)
    target = rng.random(shape) < 0.3
    F = orc.Features(land)
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    res, bs = m.simulate_batch(params, ign, seeds, want_steps=True,
                               cell_uniform=True)
    for i in range(n):
        o, obs = F.simulate(params[i], tuple(ign[i]), int(seeds[i]),
                            target=target, mode=1)
        assert np.array_equal(bs[i], obs), i
        for k in ("burnt", "inter", "target", "steps", "status", "trials"):
            assert int(res[k][i]) == o[k], (i, k)


def test_longest_first_order_changes_no_result():
    """FIRE_LONGEST_FIRST only reorders how fires are handed to the blocks:
    every result is the same as in batch order."""
    import torch

    from paper_1701_03549_gb300 import fire, synth, workloads

    ctx = fire.Context(0)
    wl = workloads.ga_generation_512(256, 16)
    m = ctx.landscape_upload(wl.land)
    m.target_upload(np.zeros(wl.land.veg.shape, bool))
    dev = torch.device("cuda")
    p = torch.tensor(wl.params, device=dev)
    g = torch.tensor(wl.ignitions, device=dev)
    s = torch.tensor(wl.seeds.view(np.int64), device=dev)
    a = torch.zeros((4096, 6), dtype=torch.int32, device=dev)
    b = torch.zeros((4096, 6), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    m.simulate_batch(p, g, s, device=True, out=a, sync=True)
    m.simulate_batch(p, g, s, device=True, out=b, sync=True, longest_first=True)
    assert torch.equal(a, b)
    m.free()
    ctx.close()


def test_closing_a_context_frees_its_maps_and_networks_first():
    """The library wants maps and networks freed before their context: the
    binding's close() frees the live ones, and dropping them afterwards is a
    no-op (no use of the destroyed context, no stale CUDA error for the next
    context)."""
    import gc

    from paper_1701_03549_gb300 import fire

    land = synth.landscape(40, 50, seed=1)
    c1 = fire.Context(0)
    m = c1.landscape_upload(land)
    net = fire.Net(c1, 16, 1)
    c1.close()
    assert m.h is None and net.h is None
    del m, net
    gc.collect()
    c2 = fire.Context(0)
    m2 = c2.landscape_upload(land)
    ign = np.array([synth.centre_ignition(land.veg)], np.int32)
    res, _ = m2.simulate_batch(np.array([TRUTH]), ign, np.array([3], np.uint64))
    assert res["status"][0] & fire.STATUS_BAD_IGNITION == 0
    c2.close()
