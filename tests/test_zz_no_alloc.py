"""fire_simulate_batch_noalloc, the entry point for callers that cannot let
the library allocate device memory (a device-memory budget owned by another
allocator, or a loop that cannot afford cudaMalloc's implicit
synchronisation).  Its results must equal fire_simulate_batch's bit for bit,
on two calls in a row (the shared scratch array keeps the previous call's
contents), for maps whose state lives in shared memory and for maps whose
per-block state buffers live in the fixed scratch array.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.
"""
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

    __graft_entry__.build()
    from paper_1701_03549_gb300 import fire

    ctx = fire.Context(0)
    yield torch, fire, ctx
    ctx.close()


def _device_args(torch, params, ignitions, seeds):
    dev = torch.device("cuda", 0)
    p = torch.tensor(np.asarray(params), dtype=torch.float64, device=dev)
    g = torch.tensor(np.asarray(ignitions, np.int32), dtype=torch.int32,
                     device=dev)
    s = torch.tensor(np.asarray(seeds, np.uint64).view(np.int64), device=dev)
    return p, g, s


def _compare(env, land, params, ignitions, seeds, want_steps):
    torch, fire, ctx = env
    m = ctx.landscape_upload(land)
    n = len(seeds)
    H, W = land.veg.shape
    p, g, s = _device_args(torch, params, ignitions, seeds)
    dev = p.device
    ref = torch.zeros((n, 6), dtype=torch.int32, device=dev)
    refbs = (torch.zeros((n, H, W), dtype=torch.int32, device=dev)
             if want_steps else None)
    torch.cuda.synchronize()
    m.simulate_batch(p, g, s, want_steps=want_steps, device=True, out=ref,
                     burn_step=refbs, sync=True)
    want = fire.results_view(ref)
    for call in range(2):
        out = torch.full((n, 6), -1, dtype=torch.int32, device=dev)
        bs = (torch.full((n, H, W), 7, dtype=torch.int32, device=dev)
              if want_steps else None)
        torch.cuda.synchronize()
        m.simulate_batch_noalloc(p, g, s, out, burn_step=bs,
                                 want_steps=want_steps, sync=True)
        assert np.array_equal(fire.results_view(out), want), call
        if want_steps:
            assert torch.equal(bs, refbs), call
    m.free()


def test_noalloc_matches_batch_shared_memory_state(env):
    wl = workloads.single_fire_128(replicates=64)
    rng = np.random.default_rng(5)
    params = wl.params.copy()
    params[::3] = rng.normal(0, 4, (len(params[::3]), 5))
    _compare(env, wl.land, params, wl.ignitions, wl.seeds, want_steps=True)


def test_noalloc_matches_batch_scratch_array_state(env):
    land = synth.landscape(1024, 1024, seed=3, wind_seed=3)
    ign = synth.centre_ignition(land.veg)
    params = np.array([synth.TRUTH_BETA, [-1.0, 0.5, 0.5, 3.0, -1.0],
                       [0.5, 0, 0, 0, 0], [-3.0, 0, 0, 0, 0]])
    n = len(params)
    _compare(env, land, params, np.tile(np.asarray(ign, np.int32), (n, 1)),
             np.arange(11, 11 + n, dtype=np.uint64), want_steps=False)


def test_noalloc_rejects_state_beyond_its_scratch(env):
    torch, fire, ctx = env
    land = synth.uniform_landscape(3000, 3000)
    m = ctx.landscape_upload(land)
    p, g, s = _device_args(torch, [[0.0] * 5], [[10, 10]], [1])
    out = torch.zeros((1, 6), dtype=torch.int32, device=p.device)
    with pytest.raises(fire.FireError) as e:
        m.simulate_batch_noalloc(p, g, s, out)
    assert e.value.code == fire.FIRE_EINVAL
    assert "no-alloc" in str(e.value)
    m.free()


def test_noalloc_takes_no_device_memory(env):
    """The promise itself: on a context that has never simulated, a call
    whose per-block state lives in the scratch array (1024 x 1024 grid) leaves
    the device's free memory unchanged.  The first call (address lookup,
    module loading) runs before the measurement; every tensor the calls use is
    allocated before it too."""
    torch, fire, _ = env
    ctx = fire.Context(0)
    land = synth.landscape(1024, 1024, seed=3, wind_seed=3)
    m = ctx.landscape_upload(land)
    ign = synth.centre_ignition(land.veg)
    params = np.array([synth.TRUTH_BETA, [0.5, 0, 0, 0, 0]])
    p, g, s = _device_args(torch, params,
                           np.tile(np.asarray(ign, np.int32), (2, 1)),
                           np.array([21, 22], np.uint64))
    out = torch.zeros((2, 6), dtype=torch.int32, device=p.device)
    m.simulate_batch_noalloc(p, g, s, out, sync=True)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(3):
        m.simulate_batch_noalloc(p, g, s, out, sync=True)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)
    assert int(fire.results_view(out)["burnt"][0]) > 1
    m.free()
    ctx.close()
