"""CPU oracle for the learned surrogate of the fire-spread automaton.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA
library never calls it and shares no code with it.

The paper fits its five parameters with a genetic algorithm whose every
fitness evaluation is a batch of automaton runs (Sec. 2.2, App. B).  The
surrogate is not part of the paper: it is a convolutional network that maps
one parameter vector, the landscape and the ignition point to a per-cell
burn probability on a coarse S x S grid, so that a GA can rank offspring
before spending automaton runs on them.  Everything here is plain numpy in
float64, written as the definitions below with ``np.matmul`` as the one
library step; ``bf16=True`` rounds at the points where the device path
stores BF16, so that the two can be compared tightly.

Definitions (the device path follows the same ones):

* coarse grid: S x S cells, each the f_r x f_c block of fine cells with
  f_r = H / S and f_c = W / S (H and W multiples of S);
* map planes (per coarse cell, means over its fine cells): 0..4 the fraction
  of fine cells of vegetation class k (classes above 4 count as 4), 5 slope
  in degrees / 45, 6 and 7 sin and cos of the aspect, 8 and 9 sin and cos of
  the wind bearing;
* network input x[b, y, x, c], 16 channels: the 10 map planes, then 1 at the
  coarse cell holding the ignition (0 elsewhere), then the five parameters
  divided by 10;
* label: the fraction of fine cells burnt, averaged over the replicates;
* network: layer 1 is a 3 x 3 convolution 16 -> C, layers 2..L are 3 x 3
  convolutions C -> C with dilations d_l, each followed by a ReLU; zero
  padding keeps S x S; the head is a 1 x 1 convolution C -> 1 and a
  logistic sigmoid.  Convolution l: z[p, o] = b[o] + sum over taps t = 3 t_y
  + t_x and inputs i of W[o, t, i] in[p + ((t_y - 1) d, (t_x - 1) d), i];
* loss: binary cross-entropy with the label, averaged over all pixels;
* predicted fitness of Eq. 2 with expected set sizes (see
  ``predicted_fitness``);
* Adam (Kingma and Ba, 2015) with the bias corrections of its Algorithm 1.
"""
from __future__ import annotations

import numpy as np

CIN = 16
DILATIONS = (1, 1, 2, 4, 8, 16, 32, 64)   # layer 1 (16 -> C) then 7 more
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


# ---------------------------------------------------------------------------
# BF16 rounding (round to nearest even on the float32 value)

def bf16(a):
    """Round to bfloat16 (via float32, round-to-nearest-even), as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if nan.any():
        out = np.where(nan, np.float32(np.nan), out)
    return out.astype(np.float64)


# ---------------------------------------------------------------------------
# inputs and labels

def planes(veg, slope, aspect, wind, S):
    """Map planes [S, S, 10] (float64) from fine rasters [H, W]."""
    H, W = veg.shape
    fr, fc = H // S, W // S
    assert fr * S == H and fc * S == W
    out = np.zeros((S, S, 10))
    cls = np.minimum(veg.astype(np.int64), 4)
    asp = np.deg2rad(aspect.astype(np.float64))
    wnd = np.deg2rad(wind.astype(np.float64))
    for i in range(S):
        for j in range(S):
            blk = (slice(i * fr, (i + 1) * fr), slice(j * fc, (j + 1) * fc))
            n = fr * fc
            for k in range(5):
                out[i, j, k] = np.count_nonzero(cls[blk] == k) / n
            out[i, j, 5] = slope[blk].astype(np.float64).sum() / n / 45.0
            out[i, j, 6] = np.sin(asp[blk]).sum() / n
            out[i, j, 7] = np.cos(asp[blk]).sum() / n
            out[i, j, 8] = np.sin(wnd[blk]).sum() / n
            out[i, j, 9] = np.cos(wnd[blk]).sum() / n
    return out


def inputs(pl, H, W, beta, ignition):
    """Network input [n, S, S, 16] from map planes, parameters [n, 5] and
    fine-grid ignitions [n, 2] (row, col)."""
    S = pl.shape[0]
    beta = np.asarray(beta, np.float64).reshape(-1, 5)
    ign = np.asarray(ignition, np.int64).reshape(-1, 2)
    n = beta.shape[0]
    x = np.zeros((n, S, S, CIN))
    x[:, :, :, :10] = pl[None]
    for s in range(n):
        x[s, ign[s, 0] // (H // S), ign[s, 1] // (W // S), 10] = 1.0
        x[s, :, :, 11:16] = beta[s] / 10.0
    return x


def labels(burn_step, S, reps):
    """Burn fractions [groups, S, S] from burn steps [groups * reps, H, W]
    (a cell burnt iff its step is >= 0)."""
    n, H, W = burn_step.shape
    fr, fc = H // S, W // S
    burnt = (burn_step >= 0).reshape(n // reps, reps, S, fr, S, fc)
    return burnt.sum(axis=(1, 3, 5)) / float(reps * fr * fc)


# ---------------------------------------------------------------------------
# parameters

def layer_shapes(C=128, cin=CIN, L=len(DILATIONS)):
    """[(name, shape)] in the flat parameter order."""
    out = []
    for l in range(L):
        ci = cin if l == 0 else C
        out.append((f"W{l + 1}", (C, 9, ci)))
        out.append((f"b{l + 1}", (C,)))
    out.append(("wh", (C,)))
    out.append(("bh", (1,)))
    return out


def param_count(C=128, cin=CIN, L=len(DILATIONS)):
    return int(sum(np.prod(s) for _, s in layer_shapes(C, cin, L)))


def unflatten(theta, C=128, cin=CIN, L=len(DILATIONS)):
    theta = np.asarray(theta, np.float64)
    out, o = {}, 0
    for name, shp in layer_shapes(C, cin, L):
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    assert o == theta.size
    return out


def flatten(d, C=128, cin=CIN, L=len(DILATIONS)):
    return np.concatenate([np.asarray(d[name], np.float64).ravel()
                           for name, _ in layer_shapes(C, cin, L)])


# ---------------------------------------------------------------------------
# network

def _shift(a, dy, dx):
    """out[:, y, x] = a[:, y + dy, x + dx], zero outside the grid."""
    n, S1, S2 = a.shape[:3]
    out = np.zeros_like(a)
    ys, ye = max(0, -dy), min(S1, S1 - dy)
    xs, xe = max(0, -dx), min(S2, S2 - dx)
    if ys < ye and xs < xe:
        out[:, ys:ye, xs:xe] = a[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def _taps(d):
    return [((t // 3 - 1) * d, (t % 3 - 1) * d) for t in range(9)]


def conv(a, Wt, b, d):
    """z[n, y, x, o] = b[o] + sum_{t, i} Wt[o, t, i] a[n, y+dy_t, x+dx_t, i]."""
    z = np.zeros(a.shape[:3] + (Wt.shape[0],)) + b
    for t, (dy, dx) in enumerate(_taps(d)):
        z += _shift(a, dy, dx) @ Wt[:, t, :].T
    return z


def conv_dgrad(dz, Wt, d):
    """Gradient with respect to the convolution's input."""
    da = np.zeros(dz.shape[:3] + (Wt.shape[2],))
    for t, (dy, dx) in enumerate(_taps(d)):
        da += _shift(dz @ Wt[:, t, :], -dy, -dx)
    return da


def conv_wgrad(dz, a, d):
    """Gradient with respect to the weights, [o, t, i]."""
    C, ci = dz.shape[3], a.shape[3]
    dW = np.zeros((C, 9, ci))
    dzf = dz.reshape(-1, C)
    for t, (dy, dx) in enumerate(_taps(d)):
        dW[:, t, :] = dzf.T @ _shift(a, dy, dx).reshape(-1, ci)
    return dW


def forward(theta, x, C=128, dil=DILATIONS, bf16_points=False):
    """Returns (logits [n, S, S], cache).  With bf16_points the input, the
    convolution weights and every stored activation are rounded to BF16 as
    on the device (the head weights stay FP32)."""
    P = unflatten(theta, C, x.shape[3], len(dil))
    rnd = bf16 if bf16_points else (lambda v: v)
    a = rnd(x)
    hs = [a]
    for l, d in enumerate(dil):
        z = conv(a, rnd(P[f"W{l + 1}"]), P[f"b{l + 1}"], d)
        a = rnd(np.maximum(z, 0.0))
        hs.append(a)
    logits = a @ P["wh"] + P["bh"][0]
    return logits, dict(P=P, hs=hs, rnd=rnd, dil=dil, C=C)


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def bce(logits, t):
    """Mean binary cross-entropy of sigmoid(logits) against labels t,
    written in the stable form max(z, 0) - t z + log(1 + exp(-|z|))."""
    z = logits
    return float(np.mean(np.maximum(z, 0.0) - t * z +
                         np.log1p(np.exp(-np.abs(z)))))


def backward(theta, x, t, bf16_points=False, C=128, dil=DILATIONS):
    """(loss, flat gradient) of the mean BCE.  With bf16_points the
    activation gradients dz are rounded to BF16 where the device stores
    them."""
    logits, cache = forward(theta, x, C, dil, bf16_points)
    P, hs, rnd = cache["P"], cache["hs"], cache["rnd"]
    loss = bce(logits, t)
    g = (sigmoid(logits) - t) / logits.size
    grads = {"wh": np.einsum("nyx,nyxc->c", g, hs[-1]),
             "bh": np.array([g.sum()])}
    L = len(dil)
    dz = rnd(g[..., None] * P["wh"] * (hs[L] > 0))
    for l in range(L, 0, -1):
        d = dil[l - 1]
        grads[f"W{l}"] = conv_wgrad(dz, hs[l - 1], d)
        grads[f"b{l}"] = dz.sum(axis=(0, 1, 2))
        if l > 1:
            da = conv_dgrad(dz, rnd(P[f"W{l}"]), d)
            dz = rnd(da * (hs[l - 1] > 0))
    return loss, flatten(grads, C, x.shape[3], L)


def adam(theta, m, v, grad, lr, step):
    """One Adam update (step counts from 1); returns (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mh = m / (1.0 - ADAM_B1 ** step)
    vh = v / (1.0 - ADAM_B2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def predicted_fitness(prob, target_frac, kind, cells_per_coarse):
    """Eq. 2 with expected set sizes: for a predicted burn fraction q and the
    target's burnt fraction t per coarse cell of c fine cells,
    E|A*| = c sum q, |A| = c sum t, E|A n A*| = c sum q t (a fine cell of
    the coarse cell is taken to burn independently of being in the target).
    kind 0: (E|A*| + |A| - 2 E|AnA*|) / |A|; kind 1: the same over
    (E|A*| + |A| - E|AnA*|)."""
    q = np.asarray(prob, np.float64).reshape(prob.shape[0], -1)
    tf = np.asarray(target_frac, np.float64).ravel()
    c = float(cells_per_coarse)
    sim = c * q.sum(axis=1)
    tgt = c * tf.sum()
    inter = c * (q * tf).sum(axis=1)
    num = sim + tgt - 2.0 * inter
    den = tgt if kind == 0 else sim + tgt - inter
    return num / den
