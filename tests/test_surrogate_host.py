"""Host-side logic of the surrogate package (no GPU): parameter layout and
initialisation, and the samplers of the training draws."""
import numpy as np
import pytest

from oracle import surrogate as sg
from paper_1701_03549_gb300 import fire, surrogate, synth


def test_layout_matches_the_oracle_and_the_library():
    from paper_1701_03549_gb300 import build

    build.build_library()
    assert surrogate.param_layout() == sg.layer_shapes()
    assert fire.fire_net_param_count() == sg.param_count()


def test_init_params_statistics():
    th = surrogate.init_params(3, head_bias=-1.5)
    assert th.dtype == np.float32 and th.size == sg.param_count()
    P = sg.unflatten(th.astype(np.float64))
    for l in range(8):
        W = P[f"W{l + 1}"]
        want = np.sqrt(2.0 / (9 * W.shape[2]))
        assert W.std() == pytest.approx(want, rel=0.05)
        assert np.all(P[f"b{l + 1}"] == 0)
    assert P["bh"][0] == pytest.approx(-1.5)
    assert np.array_equal(th, surrogate.init_params(3, head_bias=-1.5))
    assert not np.array_equal(th, surrogate.init_params(4, head_bias=-1.5))


def test_training_draws():
    p = surrogate.sample_params(5000, 1)
    assert p.shape == (5000, 5) and p.min() >= -30 and p.max() <= 30
    assert abs(p.std() - 5.0) < 0.2
    L = synth.landscape(64, 80, seed=4)
    g = surrogate.sample_ignitions(L.veg, 300, 2)
    assert g.shape == (300, 2) and g.dtype == np.int32
    assert np.all(L.veg[g[:, 0], g[:, 1]] != 0)
    # inside the central box (one cell of slack for the burnable-cell move)
    assert np.all(np.abs(g[:, 0] - 32) <= 0.25 * 64 + 2)
    assert np.all(np.abs(g[:, 1] - 40) <= 0.25 * 80 + 2)
