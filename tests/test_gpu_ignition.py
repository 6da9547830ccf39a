"""GPU parity of the ignition-point search: candidate cells, fitness map and
ensemble estimate against the oracle, bit for bit."""
import numpy as np
import pytest

from paper_1701_03549_gb300 import synth

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
    yield fire, oracle, ctx
    ctx.close()


@pytest.mark.parametrize("shape,lat,reps,kind,cutoff", [
    ((60, 70), (4, 5), 3, 0, 1.5), ((96, 64), (6, 6), 2, 1, 0.4),
    ((33, 47), (3, 2), 4, 0, -1.0), ((128, 128), (8, 8), 2, 0, np.inf)])
def test_ignition_search_matches_oracle(env, shape, lat, reps, kind, cutoff):
    fire, oracle, ctx = env
    H, W = shape
    land = synth.landscape(H, W, seed=H + W, wind_seed=H)
    ign = synth.centre_ignition(land.veg)
    beta = np.array([0.8, -1.0, 0.5, 2.5, -1.0])
    F = oracle.Features(land)
    _, bs = F.simulate(beta, ign, 17)
    target = bs >= 0
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    fm, cells, xy = fire.ignition_search(ctx, m, beta, lat[0], lat[1], reps,
                                         99, kind, cutoff)
    ofm, ocells, oxy = F.ignition_search(target, beta, lat[0], lat[1], reps,
                                         99, kind, cutoff)
    assert np.array_equal(cells, ocells)
    assert np.array_equal(fm, ofm)
    assert np.array_equal(xy, oxy)
    m.free()


def test_ignition_search_rejects_empty_target(env):
    fire, oracle, ctx = env
    land = synth.landscape(40, 40, seed=1)
    m = ctx.landscape_upload(land)
    with pytest.raises(fire.FireError) as e:
        fire.ignition_search(ctx, m, synth.TRUTH_BETA, 2, 2, 1, 1)
    assert e.value.code == fire.FIRE_EINVAL
    m.free()
