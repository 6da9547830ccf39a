"""Surrogate network on the GPU against the float64 CPU oracle
(oracle/surrogate.py), through the C ABI.

* map planes, network inputs, labels (from automaton runs) and target
  fractions against the oracle's definitions (labels from the CPU automaton);
* forward activations of every layer, probabilities, loss and the full
  parameter gradient against the oracle run with BF16 rounding at the
  device's storage points, from the same inputs and weights (tolerances from
  the BF16 rounding: a stored value may differ by one BF16 step where the
  FP32 and float64 sums straddle a rounding boundary);
* the gradient against the exact float64 gradient (mixed-precision error),
  per tensor in norm and element by element;
* Adam's first step against its closed form; training lowers the loss;
* screening (expected-size fitness and ranking) on seeded inputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import surrogate as sg                      # noqa: E402
from paper_1701_03549_gb300 import fire, surrogate, synth  # noqa: E402

S, H, W = 32, 64, 64


@pytest.fixture(scope="module")
def ctx():
    c = fire.fire_create(0, torch.cuda.current_stream())
    yield c
    c.close()


def _dev(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _bf(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def land():
    return synth.landscape(H, W, seed=31, wind_seed=31)


def test_planes_and_inputs(ctx, land):
    pl = torch.empty((S, S, 10), dtype=torch.float32, device="cuda")
    fire.fire_net_planes(ctx, S, _dev(land.veg, torch.uint8),
                         _dev(land.slope, torch.float32),
                         _dev(land.aspect, torch.float32),
                         _dev(land.wind, torch.float32), pl, sync=True)
    ref = sg.planes(land.veg, land.slope, land.aspect, land.wind, S)
    assert np.allclose(pl.cpu().numpy(), ref, rtol=0, atol=2e-6)
    beta = np.array([[-5, -10, 5, 18.1, -5], [1.5, 0.25, -3, 7, 29.9]])
    ign = np.array([[33, 30], [0, 63]], np.int32)
    x = torch.empty((2, S, S, 16), dtype=torch.bfloat16, device="cuda")
    fire.fire_net_inputs(ctx, S, H, W, _dev(ref.astype(np.float32),
                                            torch.float32),
                         _dev(beta, torch.float64), _dev(ign, torch.int32), x,
                         sync=True)
    want = sg.bf16(sg.inputs(ref.astype(np.float32).astype(np.float64), H, W,
                             beta, ign))
    assert np.array_equal(_bf(x), want)


def test_labels_from_the_automaton(ctx, land, oracle_mod):
    import oracle

    m = ctx.landscape_upload(land)
    beta = np.array([[-1.0, -2.0, 1.0, 3.0, -1.0], [0.5, 0, 0, 1.0, 0],
                     [-3.0, 0, 0, 0, 0]])
    ign = np.tile(np.array(synth.centre_ignition(land.veg), np.int32), (3, 1))
    reps, seed = 4, 12345
    lab = torch.empty((3, S, S), dtype=torch.float32, device="cuda")
    res = torch.zeros((12, 6), dtype=torch.int32, device="cuda")
    fire.fire_net_labels(ctx, m, S, _dev(beta, torch.float64),
                         _dev(ign, torch.int32), reps, seed, lab,
                         results=res, sync=True)
    F = oracle.Features(land)
    steps, rres = [], []
    for i in range(12):
        r, bs = F.simulate(beta[i // reps], tuple(ign[0]), seed=seed + i)
        steps.append(bs)
        rres.append(r)
    want = sg.labels(np.stack(steps), S, reps)
    assert np.allclose(lab.cpu().numpy(), want, rtol=1e-7, atol=0)
    got = fire.results_view(res)
    for i in range(12):
        assert got[i]["burnt"] == rres[i]["burnt"]
        assert got[i]["steps"] == rres[i]["steps"]
    # target fractions: the map's target as a single "replicate"
    tb = steps[0] >= 0
    m.target_upload(tb)
    tf = torch.empty((S, S), dtype=torch.float32, device="cuda")
    fire.fire_net_target_frac(ctx, m, S, tf, sync=True)
    assert np.allclose(tf.cpu().numpy(),
                       sg.labels(np.where(tb, 0, -1)[None], S, 1)[0],
                       rtol=1e-7, atol=0)


def _case(seed, n=2):
    rng = np.random.default_rng(seed)
    land = synth.landscape(H, W, seed=40 + seed, wind_seed=40 + seed)
    pl = sg.planes(land.veg, land.slope, land.aspect, land.wind, S)
    beta = rng.normal(0, 5, (n, 5))
    ign = np.stack([rng.integers(0, H, n), rng.integers(0, W, n)], 1)
    x = sg.bf16(sg.inputs(pl, H, W, beta, ign))
    t = rng.uniform(0, 1, (n, S, S)) * (rng.uniform(size=(n, S, S)) < 0.3)
    theta = surrogate.init_params(seed, head_bias=-1.0).astype(np.float64)
    return x, t.astype(np.float32).astype(np.float64), theta


def _close_first_layer(got, x, W, b):
    """Layer 1 from identical inputs: every element is the BF16 rounding
    (relative error <= 2^-8) of the exact ReLU(conv) value up to the FP32
    accumulation error, bounded by K 2^-24 sum|w x| with K = 144 terms (the
    bound matters where the sum nearly cancels); nearly all elements are
    bit-identical to the oracle's rounded value."""
    z = np.maximum(sg.conv(x, W, b, 1), 0.0)
    mag = sg.conv(np.abs(x), np.abs(W), np.abs(b), 1)
    tol = 2.0 ** -8 * np.abs(z) + 2 * 144 * 2.0 ** -24 * mag + 1e-30
    d = np.abs(got - z)
    assert np.all(d <= tol), float((d / tol).max())
    assert np.mean(got == sg.bf16(z)) >= 0.999


def _close_layer(got, want):
    """Deeper layers inherit the one-step rounding differences of the layers
    below and accumulate them with depth: held to a relative norm error of
    2^-7 and a worst element of 2^-5 of the layer's scale (an indexing or
    layout error is O(1))."""
    scale = np.abs(want).max() + 1e-30
    d = np.abs(got - want)
    rel = np.linalg.norm(got - want) / (np.linalg.norm(want) + 1e-30)
    assert rel <= 2.0 ** -7, rel
    assert d.max() <= 2.0 ** -5 * scale, d.max() / scale


def test_forward_backward_match_the_oracle(ctx):
    x, t, theta = _case(1)
    n = x.shape[0]
    net = fire.Net(ctx, S, 4)
    net.set_params(theta.astype(np.float32))
    xd = _dev(x, torch.float32).to(torch.bfloat16)
    td = _dev(t, torch.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    net.backward(xd, td, loss, sync=True)
    logits, cache = sg.forward(theta, x, bf16_points=True)
    for l in range(8):
        h = torch.empty((n, S, S, 128), dtype=torch.bfloat16, device="cuda")
        net.buffer(fire.BUF_ACT, l, n, h)
        if l == 0:
            P0 = sg.unflatten(theta)
            _close_first_layer(_bf(h), x, sg.bf16(P0["W1"]), P0["b1"])
        else:
            _close_layer(_bf(h), cache["hs"][l + 1])
    prob = torch.empty((n, S, S), dtype=torch.float32, device="cuda")
    net.buffer(fire.BUF_PROB, 0, n, prob)
    assert np.allclose(prob.cpu().numpy(), sg.sigmoid(logits), atol=2e-3)
    loss_ref, g_ref = sg.backward(theta, x, t, bf16_points=True)
    assert float(loss.item()) == pytest.approx(loss_ref, rel=2e-3)
    g = net.get(fire.NET_GRAD).astype(np.float64)
    # Rounding to BF16 at the storage points makes the gradient noisy, more so
    # the deeper the layer sits in the backward chain.  The device gradient
    # must be about as close to the exact float64 gradient as the oracle's
    # own BF16-emulated gradient is (same rounding points, float64 sums);
    # a layout or indexing error is far outside that.
    _, g_exact = sg.backward(theta, x, t, bf16_points=False)
    G, R, E = sg.unflatten(g), sg.unflatten(g_ref), sg.unflatten(g_exact)
    rel = lambda a, b: np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
    report = []
    for name in E:
        e_emul = rel(R[name], E[name])
        e_gpu = rel(G[name], E[name])
        report.append((name, round(e_emul, 5), round(e_gpu, 5),
                       round(rel(G[name], R[name]), 5)))
    print("gradient rel. errors (emulated vs exact, device vs exact, "
          "device vs emulated):", report)
    for name, e_emul, e_gpu, _ in report:
        assert e_gpu <= 2.0 * e_emul + 2e-3, (name, e_emul, e_gpu)
    assert rel(g, g_exact) <= 5e-2
    # Element by element: the device and the emulation round the same values
    # to BF16 at the same points and differ only in FP32 against float64
    # sums, so each is a rounding perturbation of the exact gradient of the
    # same kind.  With E = the emulation's largest deviation from the exact
    # gradient over the tensor, the triangle inequality bounds every element
    # of |g_dev - g_emul| by E + (the device's own largest deviation, of the
    # same size): 2 E, held here to 3 E for the spread of that maximum, plus
    # a floor of 2^-20 max |g| for tensors the rounding barely moves.
    worst = []
    for name in E:
        d = np.abs(G[name] - R[name])
        bound = (3.0 * np.abs(R[name] - E[name]).max() +
                 2.0 ** -20 * np.abs(R[name]).max())
        i = int(np.argmax(d))
        worst.append((name, i, float(d.flat[i]), float(bound)))
        assert d.max() <= bound, (name, i, float(d.flat[i]), float(bound))
    print("worst element per tensor (name, flat index, |dev - emul|, bound):",
          [(n, i, f"{v:.3g}", f"{b:.3g}") for n, i, v, b in worst])
    # one Adam step from zero moments moves each weight by lr g/(|g| + eps)
    lr = 1e-3
    net.adam(lr, sync=True)
    th1 = net.get(fire.NET_PARAMS).astype(np.float64)
    step = lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(th1, theta.astype(np.float32) - step, rtol=0,
                       atol=2e-7 + 1e-6 * np.abs(theta).max())
    m1 = net.get(fire.NET_ADAM_M).astype(np.float64)
    assert np.allclose(m1, 0.1 * g, rtol=1e-6, atol=1e-30)
    net.free()


def test_training_lowers_the_loss(ctx):
    x, t, theta = _case(2, n=4)
    net = fire.Net(ctx, S, 4)
    net.set_params(theta.astype(np.float32))
    xd = _dev(x, torch.float32).to(torch.bfloat16)
    td = _dev(t, torch.float32)
    loss = torch.zeros(60, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for s in range(60):
        net.backward(xd, td, loss[s:s + 1])
        net.adam(2e-3)
    ctx.sync()
    L = loss.cpu().numpy()
    assert np.isfinite(L).all()
    assert L[-5:].mean() < 0.8 * L[:3].mean(), L[[0, 1, 2, -3, -2, -1]]
    net.free()


def test_forward_chunks_and_batch_invariance(ctx):
    x, _, theta = _case(3, n=5)
    net = fire.Net(ctx, S, 2)            # forces chunks of 2, 2, 1
    net.set_params(theta.astype(np.float32))
    xd = _dev(x, torch.float32).to(torch.bfloat16)
    p5 = torch.empty((5, S, S), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    net.forward(xd, p5, sync=True)
    p1 = torch.empty((1, S, S), dtype=torch.float32, device="cuda")
    net.forward(xd[4:5].contiguous(), p1, sync=True)
    assert torch.equal(p5[4], p1[0])
    logits, _ = sg.forward(theta, x, bf16_points=True)
    assert np.allclose(p5.cpu().numpy(), sg.sigmoid(logits), atol=2e-3)
    net.free()


def test_screen_against_the_oracle(ctx):
    rng = np.random.default_rng(9)
    n, s2 = 50, 16
    prob = rng.uniform(size=(n, s2, s2)).astype(np.float32)
    prob[7] = np.nan
    tf = (rng.uniform(size=(s2, s2)) * (rng.uniform(size=(s2, s2)) < 0.4)
          ).astype(np.float32)
    for kind in (0, 1):
        pred = torch.empty(n, dtype=torch.float64, device="cuda")
        keep = torch.full((12,), -1, dtype=torch.int32, device="cuda")
        fire.fire_net_screen(ctx, s2, _dev(prob, torch.float32),
                             _dev(tf, torch.float32), 16.0, kind, 12, pred,
                             keep, sync=True)
        want = sg.predicted_fitness(prob.astype(np.float64),
                                    tf.astype(np.float64), kind, 16)
        got = pred.cpu().numpy()
        ok = ~np.isnan(want)
        assert np.isnan(got[7]) and np.allclose(got[ok], want[ok], rtol=1e-12)
        order = np.argsort(np.where(ok, want, np.inf), kind="stable")
        assert np.array_equal(keep.cpu().numpy(), order[:12])


def test_bad_arguments_are_rejected(ctx):
    with pytest.raises(fire.FireError):
        fire.Net(ctx, 48, 1)             # not a power of two
    net = fire.Net(ctx, 16, 1)
    x = torch.zeros((2, 16, 16, 16), dtype=torch.bfloat16, device="cuda")
    t = torch.zeros((2, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(fire.FireError):
        net.backward(x, t)               # n > max_batch
    net.free()


@pytest.mark.parametrize("S5,n,splits", [(128, 5, ((0, 2), (2, 5))),
                                         (256, 3, ((0, 1), (1, 3)))])
def test_row_tiles_and_batch_consistency(S5, n, splits):
    """At S = 128 a 128-pixel tile is one image row and at S = 256 (the
    benchmark's size) half a row (at S = 32 it spans four rows, as in the
    tests above), so the TMA boxes take other shapes: the first two layers
    against the oracle (same criteria as above), and the whole gradient of
    the batch against the sample-weighted gradients of two sub-batches (the
    gradient is a mean over pixels)."""
    ctx = fire.fire_create(0, torch.cuda.current_stream())
    rng = np.random.default_rng(11)
    land = synth.landscape(2 * S5, 2 * S5, seed=12, wind_seed=12)
    pl = sg.planes(land.veg, land.slope, land.aspect, land.wind, S5)
    beta = rng.normal(0, 5, (n, 5))
    ign = np.stack([rng.integers(0, 2 * S5, n), rng.integers(0, 2 * S5, n)], 1)
    x = sg.bf16(sg.inputs(pl, 2 * S5, 2 * S5, beta, ign))
    t = (rng.uniform(0, 1, (n, S5, S5)) *
         (rng.uniform(size=(n, S5, S5)) < 0.3)).astype(np.float32)
    theta = surrogate.init_params(4, head_bias=-1.0)
    net = fire.Net(ctx, S5, n)
    net.set_params(theta)
    xd = _dev(x, torch.float32).to(torch.bfloat16)
    td = _dev(t, torch.float32)
    torch.cuda.synchronize()
    net.backward(xd, td, sync=True)
    g5 = net.get(fire.NET_GRAD).astype(np.float64)
    h = torch.empty((n, S5, S5, 128), dtype=torch.bfloat16, device="cuda")
    P = sg.unflatten(theta.astype(np.float64))
    a1 = sg.bf16(np.maximum(sg.conv(x, sg.bf16(P["W1"]), P["b1"], 1), 0))
    a2 = sg.bf16(np.maximum(sg.conv(a1, sg.bf16(P["W2"]), P["b2"], 1), 0))
    net.buffer(fire.BUF_ACT, 0, n, h)
    _close_first_layer(_bf(h), x, sg.bf16(P["W1"]), P["b1"])
    net.buffer(fire.BUF_ACT, 1, n, h)
    _close_layer(_bf(h), a2)
    net.free()
    gs = []
    for lo, hi in splits:
        sub = fire.Net(ctx, S5, hi - lo)
        sub.set_params(theta)
        sub.backward(xd[lo:hi].contiguous(), td[lo:hi].contiguous(), sync=True)
        gs.append((hi - lo) * sub.get(fire.NET_GRAD).astype(np.float64))
        sub.free()
    want = (gs[0] + gs[1]) / n
    G, R = sg.unflatten(g5), sg.unflatten(want)
    for name in R:
        err = np.linalg.norm(G[name] - R[name]) / (np.linalg.norm(R[name]) + 1e-30)
        assert err <= 2e-2, (name, err)
    ctx.close()
