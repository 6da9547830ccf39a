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
    ((33, 47), (3, 2), 4, 0, -1.0), ((128, 128), (8, 8), 2, 0, np.inf),
    ((40, 50), (1, 1), 1, 1, 0.5)])
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


def test_single_cell_target(env):
    """A target of one burnable cell: its bounding box is that cell, so
    every lattice point snaps to it and every candidate is the same fire."""
    fire, oracle, ctx = env
    land = synth.landscape(48, 40, seed=5, wind_seed=5)
    r, c = np.argwhere(land.veg != 0)[len(np.argwhere(land.veg != 0)) // 2]
    target = np.zeros(land.veg.shape, bool)
    target[r, c] = True
    beta = np.array([-0.5, 0.5, 0.5, 1.0, -1.0])
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    fm, cells, xy = fire.ignition_search(ctx, m, beta, 3, 3, 2, 5, 0, 1.5)
    F = oracle.Features(land)
    ofm, ocells, oxy = F.ignition_search(target, beta, 3, 3, 2, 5, 0, 1.5)
    assert np.array_equal(cells, ocells) and np.array_equal(fm, ofm)
    assert np.array_equal(xy, oxy)
    assert (cells.reshape(-1, 2) == [r, c]).all()
    m.free()


def test_ignition_search_rejects_empty_target(env):
    fire, oracle, ctx = env
    land = synth.landscape(40, 40, seed=1)
    m = ctx.landscape_upload(land)
    with pytest.raises(fire.FireError) as e:
        fire.ignition_search(ctx, m, synth.TRUTH_BETA, 2, 2, 1, 1)
    assert e.value.code == fire.FIRE_EINVAL
    m.free()


def test_nearest_cell_on_a_wide_map(env):
    """On a 32 x 131072 map the squared distance from the lattice point to a
    target cell exceeds 2^32: the nearest burnt cell must still win (a 64-bit
    key holding the distance above the cell index would wrap here)."""
    fire, oracle, ctx = env
    H, W = 32, 131072
    land = synth.uniform_landscape(H, W)
    target = np.zeros((H, W), bool)
    target[5, 0] = True          # distance^2 = 8^2 + 65536^2 > 2^32
    target[20, W - 1] = True     # distance^2 = 7^2 + 65535^2 < 2^32
    beta = np.array([-1000.0, 0.0, 0.0, 0.0, 0.0])   # burns the ignition only
    m = ctx.landscape_upload(land)
    m.target_upload(target)
    fm, cells, xy = fire.ignition_search(ctx, m, beta, 1, 1, 1, 5, 0, 1.5)
    assert cells[0, 0].tolist() == [20, W - 1]
    F = oracle.Features(land)
    ofm, ocells, oxy = F.ignition_search(target, beta, 1, 1, 1, 5, 0, 1.5)
    assert np.array_equal(cells, ocells)
    assert np.array_equal(fm, ofm)
    assert np.array_equal(xy, oxy)
    m.free()
