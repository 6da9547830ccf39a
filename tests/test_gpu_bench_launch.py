"""Parity of the launches the benchmark times, as it times them, against the
oracle on stratified samples of their outputs.

* The nine-fire uneven batch (100,000 simulations, grids up to 2000 x 1500):
  targets of the reference parameters (simulated by the oracle), the launch
  shape the autotuner picks on a stratified tenth of the batch, one
  graph-captured fire_simulate_multi call replayed once; every result field
  of 16 simulations per fire (144), evenly spaced over each fire's block.
* One 512 x 512 GA generation (4096 simulations): the oracle's reference
  target, the shape the autotuner picks in longest-first order, the
  longest-first launch of fire_simulate_batch; every result field of
  replicate 0 of every other parameter vector (128 simulations), and the
  burn-step maps of eight of them from the same launch run again with
  burn-step output (whose results must equal the first launch's).

The oracle runs in a spawn process pool started before any GPU call.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FIELDS = ("burnt", "inter", "target", "steps", "status", "trials")
_W = {}


def _lands(kind):
    from paper_1701_03549_gb300 import synth, workloads

    if kind == "uneven":
        return workloads.uneven_lands()
    return [synth.preset_landscape("ga_generation_512")]


def _init(kind):
    import oracle

    from paper_1701_03549_gb300 import synth

    lands = _lands(kind)
    _W["F"] = [oracle.Features(L) for L in lands]
    _W["ign"] = [synth.centre_ignition(L.veg) for L in lands]
    _W["burnable"] = [int((L.veg != 0).sum()) for L in lands]
    _W["T"] = {}


def _target(j):
    from paper_1701_03549_gb300 import synth, workloads

    F, ign = _W["F"][j], _W["ign"][j]
    seed, burnt = workloads.pick_target(
        lambda s: F.simulate(synth.TRUTH_BETA, ign, s)[1] >= 0,
        _W["burnable"][j])
    return seed, np.packbits(burnt.ravel())


def _sim(args):
    j, packed, beta, ign, seed, steps = args
    F = _W["F"][j]
    if j not in _W["T"]:
        _W["T"][j] = np.unpackbits(packed, count=F.H * F.W).reshape(
            F.H, F.W).astype(bool)
    r, bs = F.simulate(beta, ign, int(seed), target=_W["T"][j],
                       want_steps=steps)
    return r, bs


def _pool(kind):
    return mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1),
                                        initializer=_init, initargs=(kind,))


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


def _unpack(packed, shape):
    return np.unpackbits(packed, count=shape[0] * shape[1]).reshape(
        shape).astype(bool)


def test_uneven_batch_as_benchmarked(env):
    torch = env
    from paper_1701_03549_gb300 import fire, workloads

    pool = _pool("uneven")
    try:
        wl = workloads.uneven_fires()
        targets = pool.map(_target, range(len(wl.lands)), chunksize=1)
        ctx = fire.Context(0)
        maps = [ctx.landscape_upload(L) for L in wl.lands]
        for m, L, (_, p) in zip(maps, wl.lands, targets):
            m.target_upload(_unpack(p, L.veg.shape))
        sub = np.arange(0, wl.n, 10)
        shape = fire.fire_autotune(ctx, maps, wl.map_of_sim[sub],
                                   wl.params[sub], wl.ignitions[sub],
                                   wl.seeds[sub])
        print("autotuned launch:", shape)
        dev = torch.device("cuda")
        t_mi = torch.tensor(wl.map_of_sim, device=dev)
        t_p = torch.tensor(wl.params, dtype=torch.float64, device=dev)
        t_g = torch.tensor(wl.ignitions, device=dev)
        t_s = torch.tensor(wl.seeds.view(np.int64), device=dev)
        out = torch.zeros((wl.n, 6), dtype=torch.int32, device=dev)
        got = []
        for _ in range(2):   # capture, then replay of the same graph
            out.fill_(-1)
            torch.cuda.synchronize()   # the context runs on its own stream
            fire.fire_simulate_multi(ctx, maps, t_mi, t_p, t_g, t_s,
                                     device=True, out=out, graph=True,
                                     sync=True)
            got.append(fire.results_view(out).copy())
        assert np.array_equal(got[0], got[1])
        res = got[0]
        for m in maps:
            m.free()
        ctx.close()
        idx = workloads.stratified_sample(wl.map_of_sim, 16)
        jobs = [(int(wl.map_of_sim[i]), targets[wl.map_of_sim[i]][1],
                 wl.params[i], tuple(int(v) for v in wl.ignitions[i]),
                 int(wl.seeds[i]), False) for i in idx]
        want = pool.map(_sim, jobs, chunksize=1)
    finally:
        pool.close()
        pool.join()
    bad = [(int(i), k, int(res[k][i]), o[k]) for i, (o, _) in zip(idx, want)
           for k in FIELDS if int(res[k][i]) != o[k]]
    assert not bad, bad[:10]
    # the sample spans short and long fires on every map
    steps = np.array([o["steps"] for o, _ in want])
    assert steps.min() <= 2 and steps.max() >= 200


def test_ga_generation_as_benchmarked(env):
    torch = env
    from paper_1701_03549_gb300 import fire, workloads

    pool = _pool("ga512")
    try:
        wl = workloads.ga_generation_512(256, 16)
        (tseed, packed), = pool.map(_target, [0])
        H, W = wl.shape
        ctx = fire.Context(0)
        m = ctx.landscape_upload(wl.land)
        m.target_upload(_unpack(packed, (H, W)))
        shape = fire.fire_autotune(ctx, [m], None, wl.params, wl.ignitions,
                                   wl.seeds, longest_first=True)
        print("autotuned launch:", shape)
        dev = torch.device("cuda")
        p = torch.tensor(wl.params, dtype=torch.float64, device=dev)
        g = torch.tensor(wl.ignitions, dtype=torch.int32, device=dev)
        s = torch.tensor(wl.seeds.view(np.int64), device=dev)
        out = torch.full((wl.n, 6), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()   # the context runs on its own stream
        m.simulate_batch(p, g, s, device=True, out=out, longest_first=True,
                         sync=True)
        res = fire.results_view(out)
        # the same launch with burn-step output (4096 maps, 4.3 GB)
        out2 = torch.full((wl.n, 6), -1, dtype=torch.int32, device=dev)
        bs = torch.empty((wl.n, H, W), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        m.simulate_batch(p, g, s, want_steps=True, device=True, out=out2,
                         burn_step=bs, longest_first=True, sync=True)
        assert np.array_equal(fire.results_view(out2), res)
        idx = np.arange(0, wl.n, 32)            # replicate 0, every other vector
        steps = res["steps"][idx].astype(np.int64)
        order = np.argsort(-steps, kind="stable")
        with_maps = sorted(set(idx[order[:4]].tolist()) |
                           set(idx[[1, 17, 63, 101]].tolist()))
        maps = {int(i): bs[int(i)].cpu().numpy() for i in with_maps}
        del bs
        m.free()
        ctx.close()
        jobs = [(0, packed, wl.params[i], tuple(int(v) for v in wl.ignitions[i]),
                 int(wl.seeds[i]), int(i) in maps) for i in idx]
        want = pool.map(_sim, jobs, chunksize=1)
    finally:
        pool.close()
        pool.join()
    bad = [(int(i), k, int(res[k][i]), o[k]) for i, (o, _) in zip(idx, want)
           for k in FIELDS if int(res[k][i]) != o[k]]
    assert not bad, bad[:10]
    checked = 0
    for i, (_, obs) in zip(idx, want):
        if int(i) in maps:
            assert np.array_equal(maps[int(i)], obs), int(i)
            checked += 1
    assert checked == len(maps) >= 4
    assert max(int(maps[i].max()) for i in maps) >= 100
