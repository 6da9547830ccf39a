"""Pins for the surrogate's CPU oracle (oracle/surrogate.py).

* BF16 rounding against torch's float32 -> bfloat16 conversion and hand-worked
  ties;
* the dilated convolution against scipy.signal.correlate2d with a
  zero-stuffed kernel (a different algorithm and library);
* every gradient (weights, biases, head, the input path through the
  transposed convolution) against central finite differences in float64;
* BCE and Adam closed forms (Adam's bias-corrected first step and constant
  gradients move each weight by exactly lr g / (|g| + eps));
* map planes, inputs and labels on constructed maps with known answers, and
  the expected-size fitness against Eq. 2 on hard (0/1) maps.
"""
import numpy as np
import pytest

from oracle import surrogate as sg

scipy_signal = pytest.importorskip("scipy.signal")


def test_param_count_closed_form():
    want = (128 * 9 * 16 + 128) + 7 * (128 * 9 * 128 + 128) + 128 + 1
    assert sg.param_count() == want == 1051777
    th = np.arange(want, dtype=np.float64)
    assert np.array_equal(sg.flatten(sg.unflatten(th)), th)


def test_bf16_rounding_ties_and_torch():
    one = 1.0
    ulp = 2.0 ** -7
    assert sg.bf16(np.array([one + ulp / 2]))[0] == one            # tie -> even
    assert sg.bf16(np.array([one + 1.5 * ulp]))[0] == one + 2 * ulp
    assert sg.bf16(np.array([one + 0.51 * ulp]))[0] == one + ulp
    assert sg.bf16(np.array([-3.0]))[0] == -3.0
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) *
         np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sg.bf16(x), want)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_conv_matches_correlate2d(d):
    rng = np.random.default_rng(d)
    S, ci, co = 9, 3, 2
    a = rng.standard_normal((1, S, S, ci))
    W = rng.standard_normal((co, 9, ci))
    b = rng.standard_normal(co)
    z = sg.conv(a, W, b, d)
    for o in range(co):
        want = np.full((S, S), b[o])
        for i in range(ci):
            k = np.zeros((2 * d + 1, 2 * d + 1))
            for t in range(9):
                k[(t // 3) * d, (t % 3) * d] = W[o, t, i]
            want += scipy_signal.correlate2d(a[0, :, :, i], k, mode="same",
                                             boundary="fill")
        assert np.allclose(z[0, :, :, o], want, rtol=1e-12, atol=1e-12)


def _fd(f, x, eps=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = x[i]
        x[i] = old + eps
        fp = f()
        x[i] = old - eps
        fm = f()
        x[i] = old
        g[i] = (fp - fm) / (2 * eps)
    return g


@pytest.mark.parametrize("d", [1, 2])
def test_conv_input_and_weight_gradients(d):
    rng = np.random.default_rng(10 + d)
    a = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    R = rng.standard_normal((2, 5, 6, 4))

    def f():
        return float((sg.conv(a, W, b, d) * R).sum())

    assert np.allclose(sg.conv_dgrad(R, W, d), _fd(f, a), atol=1e-7)
    assert np.allclose(sg.conv_wgrad(R, a, d), _fd(f, W), atol=1e-7)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(7)
    C, dil = 4, (1, 2, 1)
    x = rng.standard_normal((2, 6, 6, 3))
    t = rng.uniform(0, 1, (2, 6, 6))
    n = sg.param_count(C, 3, len(dil))
    theta = rng.standard_normal(n) * 0.5
    logits, _ = sg.forward(theta, x, C, dil)
    loss, g = sg.backward(theta, x, t, C=C, dil=dil)
    assert loss == pytest.approx(sg.bce(logits, t), rel=1e-15)

    def f():
        return sg.bce(sg.forward(theta, x, C, dil)[0], t)

    gfd = _fd(f, theta)
    assert np.allclose(g, gfd, rtol=1e-5, atol=1e-8), np.abs(g - gfd).max()


def test_backward_bf16_points_is_close_to_exact():
    rng = np.random.default_rng(8)
    C, dil = 8, (1, 1, 2)
    x = sg.bf16(rng.standard_normal((1, 8, 8, 4)))
    t = rng.uniform(0, 1, (1, 8, 8))
    theta = rng.standard_normal(sg.param_count(C, 4, 3)) * 0.3
    _, g0 = sg.backward(theta, x, t, C=C, dil=dil)
    _, g1 = sg.backward(theta, x, t, bf16_points=True, C=C, dil=dil)
    assert np.linalg.norm(g1 - g0) <= 0.05 * np.linalg.norm(g0)
    assert not np.array_equal(g0, g1)


def test_bce_closed_forms():
    t = np.array([0.0, 0.3, 1.0])
    assert sg.bce(np.zeros(3), t) == pytest.approx(np.log(2.0), rel=1e-15)
    assert sg.bce(np.array([1000.0]), np.array([1.0])) == 0.0
    assert sg.bce(np.array([-1000.0]), np.array([1.0])) == pytest.approx(1000.0)
    z = np.array([0.7])
    p = 1.0 / (1.0 + np.exp(-0.7))
    want = -(0.2 * np.log(p) + 0.8 * np.log(1 - p))
    assert sg.bce(z, np.array([0.2])) == pytest.approx(want, rel=1e-13)
    assert sg.sigmoid(np.array([0.0]))[0] == 0.5


def test_adam_bias_corrected_steps():
    rng = np.random.default_rng(3)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr = 1e-3
    cur = th.copy()
    for k in range(1, 6):
        cur, m, v = sg.adam(cur, m, v, g, lr, k)
        step = lr * g / (np.abs(g) + sg.ADAM_EPS)
        assert np.allclose(cur, th - k * step, rtol=0, atol=1e-12)


def test_planes_on_constructed_maps():
    H = W = 8
    veg = np.zeros((H, W), np.uint8)
    veg[::2, ::2] = 3
    veg[1::2, 1::2] = 7           # counts as class 4
    slope = np.full((H, W), 45.0, np.float32)
    aspect = np.full((H, W), 90.0, np.float32)
    wind = np.zeros((H, W), np.float32)
    wind[:, 4:] = 180.0
    pl = sg.planes(veg, slope, aspect, wind, 4)
    assert np.allclose(pl[..., 0], 0.5) and np.allclose(pl[..., 3], 0.25)
    assert np.allclose(pl[..., 4], 0.25) and np.allclose(pl[..., 1:3], 0)
    assert np.allclose(pl[..., 5], 1.0)
    assert np.allclose(pl[..., 6], 1.0) and np.allclose(pl[..., 7], 0, atol=1e-15)
    assert np.allclose(pl[:, :2, 9], 1.0) and np.allclose(pl[:, 2:, 9], -1.0)
    # against a vectorised block mean
    rng = np.random.default_rng(4)
    veg = rng.integers(0, 6, (12, 18)).astype(np.uint8)
    sl = rng.uniform(0, 40, (12, 18)).astype(np.float32)
    asp = rng.uniform(0, 360, (12, 18)).astype(np.float32)
    wd = rng.uniform(0, 360, (12, 18)).astype(np.float32)
    pl = sg.planes(veg, sl, asp, wd, 6)
    blk = lambda a: a.reshape(6, 2, 6, 3).mean(axis=(1, 3))
    assert np.allclose(pl[..., 5], blk(sl.astype(np.float64)) / 45)
    assert np.allclose(pl[..., 8], blk(np.sin(np.radians(wd.astype(np.float64)))))
    assert np.allclose(pl[..., :5].sum(axis=-1), 1.0)


def test_inputs_and_labels():
    pl = np.random.default_rng(5).uniform(size=(4, 4, 10))
    x = sg.inputs(pl, 16, 8, [[10, 20, 30, 40, 50], [0, 0, 0, 0, -5]],
                  [[5, 3], [15, 7]])
    assert x.shape == (2, 4, 4, 16)
    assert np.array_equal(x[0, :, :, :10], pl)
    assert x[0, 1, 1, 10] == 1 and x[0, :, :, 10].sum() == 1   # (5//4, 3//2)
    assert x[1, 3, 3, 10] == 1 and x[1, :, :, 10].sum() == 1
    assert np.allclose(x[0, :, :, 11:], [1, 2, 3, 4, 5])
    assert np.allclose(x[1, :, :, 15], -0.5)
    bs = -np.ones((4, 4, 6), np.int32)        # 2 groups x 2 replicates
    bs[0, 0, 0] = 0                            # coarse cell (0,0) of group 0
    bs[1, :2, :3] = 3                          # the whole coarse cell (0,0)
    bs[3, 2:, 3:] = -2
    lab = sg.labels(bs, 2, 2)
    assert lab.shape == (2, 2, 2)
    assert lab[0, 0, 0] == pytest.approx((1 + 6) / 12)
    assert lab[0].sum() == pytest.approx(7 / 12) and lab[1].sum() == 0


def test_predicted_fitness_on_hard_maps_is_eq2(oracle_mod):
    rng = np.random.default_rng(6)
    tgt = rng.uniform(size=(10, 10)) < 0.3
    sims = rng.uniform(size=(5, 10, 10)) < 0.4
    for kind in (0, 1):
        pf = sg.predicted_fitness(sims.astype(np.float64), tgt.astype(float),
                                  kind, 1)
        for s in range(5):
            b = int(sims[s].sum())
            i = int((sims[s] & tgt).sum())
            want = oracle_mod.fitness(b, i, int(tgt.sum()), kind)
            assert pf[s] == pytest.approx(want, rel=1e-14)
