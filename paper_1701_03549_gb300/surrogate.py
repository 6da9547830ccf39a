"""The learned surrogate on top of the CUDA library (fire_net_* in
include/fire.h): parameter initialisation, training sets generated by the
automaton, the training loop, and the surrogate-screened genetic algorithm.

The paper has no surrogate.  Here it ranks GA offspring by a predicted Eq. 2
fitness so that only the most promising quarter is simulated; the automaton
stays the judge of every kept candidate.  All network arithmetic (inputs,
forward, backward, Adam, labels, screening) runs in the library's kernels on
device-resident torch tensors; this module sequences the calls, draws the
random numbers (initial weights, mini-batch order, training parameters) and
gathers mini-batches.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import calibrate, fire, synth

CIN, C, LAYERS = fire.NET_CIN, fire.NET_C, fire.NET_LAYERS


def param_layout():
    """[(name, shape)] of the flat parameter vector, in order."""
    out = []
    for l in range(LAYERS):
        ci = CIN if l == 0 else C
        out.append((f"W{l + 1}", (C, 9, ci)))
        out.append((f"b{l + 1}", (C,)))
    out += [("wh", (C,)), ("bh", (1,))]
    return out


def init_params(seed: int, head_bias: float = -2.0) -> np.ndarray:
    """He-normal convolution weights (std sqrt(2 / (9 C_in))), zero biases,
    head weights N(0, 0.01 / C) and head bias `head_bias` (a low initial burn
    probability); float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in param_layout():
        if name.startswith("W"):
            parts.append(rng.standard_normal(shp) * np.sqrt(2.0 / (9 * shp[2])))
        elif name == "wh":
            parts.append(rng.standard_normal(shp) * (0.1 / np.sqrt(C)))
        elif name == "bh":
            parts.append(np.full(shp, head_bias))
        else:
            parts.append(np.zeros(shp))
    theta = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    assert theta.size == fire.fire_net_param_count()
    return theta


def _torch():
    import torch
    return torch


@dataclass
class Dataset:
    """One map's training samples, device-resident."""
    H: int
    W: int
    planes: object          # (S, S, 10) float32
    params: object          # (G, 5) float64
    ign: object             # (G, 2) int32
    labels: object          # (G, S, S) float32

    def __len__(self):
        return int(self.params.shape[0])


class Surrogate:
    """A fire_net with its context, input size S and mini-batch size."""

    def __init__(self, ctx: fire.Context, S: int = 256, max_batch: int = 8,
                 seed: int = 1):
        self.ctx, self.S = ctx, int(S)
        self.net = fire.Net(ctx, S, max_batch)
        self.max_batch = int(max_batch)
        self.net.set_params(init_params(seed))
        self.step = 0

    # -- inputs
    def planes(self, land):
        torch = _torch()
        dev = torch.device("cuda", self.ctx.device)
        t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt,
                                       device=dev)
        veg = t(land.veg, torch.uint8)
        out = torch.empty((self.S, self.S, 10), dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        fire.fire_net_planes(self.ctx, self.S, veg, t(land.slope, torch.float32),
                             t(land.aspect, torch.float32),
                             t(land.wind, torch.float32), out, sync=True)
        return out

    def inputs(self, planes, H, W, params, ign, out=None):
        torch = _torch()
        n = int(params.shape[0])
        if out is None:
            out = torch.empty((n, self.S, self.S, CIN), dtype=torch.bfloat16,
                              device=params.device)
        fire.fire_net_inputs(self.ctx, self.S, H, W, planes, params, ign, out)
        return out

    def predict(self, planes, H, W, params, ign, chunk=64):
        """Burn probabilities (n, S, S) for parameter rows `params` (device
        float64) and ignitions `ign` (device int32 (n, 2))."""
        torch = _torch()
        n = int(params.shape[0])
        prob = torch.empty((n, self.S, self.S), dtype=torch.float32,
                           device=params.device)
        x = torch.empty((min(n, chunk), self.S, self.S, CIN),
                        dtype=torch.bfloat16, device=params.device)
        for s0 in range(0, n, chunk):
            s1 = min(n, s0 + chunk)
            xs = x[: s1 - s0]
            self.inputs(planes, H, W, params[s0:s1], ign[s0:s1], out=xs)
            self.net.forward(xs, prob[s0:s1])
        self.ctx.sync()
        return prob

    # -- training
    def train(self, data, steps: int, lr: float = 1e-3, batch: int | None = None,
              seed: int = 0, lr_final: float | None = None):
        """`steps` Adam steps on mini-batches drawn uniformly (without
        replacement within an epoch) from the datasets `data`; cosine decay
        from lr to lr_final.  Returns the per-step losses."""
        torch = _torch()
        batch = batch or self.max_batch
        rng = np.random.default_rng(seed)
        sizes = [len(d) for d in data]
        index = np.concatenate([np.stack([np.full(s, k), np.arange(s)], 1)
                                for k, s in enumerate(sizes)])
        dev = data[0].params.device
        x = torch.empty((batch, self.S, self.S, CIN), dtype=torch.bfloat16,
                        device=dev)
        tgt = torch.empty((batch, self.S, self.S), dtype=torch.float32,
                          device=dev)
        loss = torch.zeros(steps, dtype=torch.float64, device=dev)
        order = rng.permutation(len(index))
        pos = 0
        lr_final = lr if lr_final is None else lr_final
        for s in range(steps):
            if pos + batch > len(order):
                order = rng.permutation(len(index))
                pos = 0
            pick = index[order[pos:pos + batch]]
            pos += batch
            # group the mini-batch by dataset; inputs are built per map
            row = 0
            for k in np.unique(pick[:, 0]):
                ids = torch.as_tensor(pick[pick[:, 0] == k, 1], device=dev)
                d = data[k]
                m = int(ids.numel())
                self.inputs(d.planes, d.H, d.W, d.params[ids].contiguous(),
                            d.ign[ids].contiguous(), out=x[row:row + m])
                tgt[row:row + m] = d.labels[ids]
                row += m
            torch.cuda.synchronize(dev)
            self.net.backward(x, tgt, loss[s:s + 1])
            c = 0.5 * (1 + np.cos(np.pi * s / max(1, steps)))
            self.net.adam(lr_final + (lr - lr_final) * c)
            self.step += 1
        self.ctx.sync()
        return loss.cpu().numpy()


def sample_params(n: int, seed: int, sd: float = 5.0, lo=-30.0, hi=30.0):
    """Training parameter vectors: N(0, sd^2) per gene (the GA's initial
    prior), clipped to the GA bounds."""
    rng = np.random.default_rng(seed)
    return np.clip(rng.normal(0.0, sd, (n, 5)), lo, hi)


def sample_ignitions(veg: np.ndarray, n: int, seed: int, spread: float = 0.25):
    """Burnable ignition cells drawn uniformly from the central box of side
    2 spread (H, W) around the centre (the nearest burnable cell if the drawn
    one is not)."""
    rng = np.random.default_rng(seed)
    H, W = veg.shape
    burn = np.argwhere(veg != 0)
    out = np.zeros((n, 2), np.int32)
    for i in range(n):
        r = int(H / 2 + rng.uniform(-spread, spread) * H)
        c = int(W / 2 + rng.uniform(-spread, spread) * W)
        r, c = min(max(r, 0), H - 1), min(max(c, 0), W - 1)
        if veg[r, c] == 0:
            d = ((burn - [r, c]) ** 2).sum(1)
            r, c = burn[int(np.argmin(d))]
        out[i] = (r, c)
    return out


def make_dataset(ctx, m, land, sur: Surrogate, groups: int, reps: int,
                 seed: int, params=None, ign=None, sim_seed: int = 1 << 40):
    """Automaton-generated training set on map `m` (a fire.Map of `land`):
    `groups` (parameters, ignition) draws, each simulated `reps` times; the
    label is the burn fraction per coarse cell."""
    torch = _torch()
    dev = torch.device("cuda", ctx.device)
    if params is None:
        params = sample_params(groups, seed)
    if ign is None:
        ign = sample_ignitions(land.veg, groups, seed + 1)
    p = torch.tensor(np.asarray(params, np.float64), device=dev)
    g = torch.tensor(np.asarray(ign, np.int32), device=dev)
    labels = torch.empty((groups, sur.S, sur.S), dtype=torch.float32,
                         device=dev)
    torch.cuda.synchronize(dev)
    fire.fire_net_labels(ctx, m, sur.S, p, g, reps, sim_seed + seed * 1000003,
                         labels, sync=True)
    return Dataset(land.veg.shape[0], land.veg.shape[1], sur.planes(land), p, g,
                   labels)


@dataclass
class ScreenedHistory(calibrate.History):
    predicted: list = field(default_factory=list)  # per generation (pool,)


def _evaluate_with_labels(ctx, m, sur, genes, ign_dev, seed0, reps, kind):
    """Mean fitness over `reps` replicates of each row of `genes` (as
    calibrate.evaluate, seeds seed0 + i R + r) and the burn fractions of the
    same runs (the surrogate's labels), from one fire_net_labels call."""
    torch = _torch()
    dev = genes.device
    P = int(genes.shape[0])
    res = torch.zeros((P * reps, 6), dtype=torch.int32, device=dev)
    lab = torch.empty((P, sur.S, sur.S), dtype=torch.float32, device=dev)
    fit = torch.empty(P * reps, dtype=torch.float64, device=dev)
    mean = torch.empty(P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    fire.fire_net_labels(ctx, m, sur.S, genes, ign_dev[:P].contiguous(), reps,
                         seed0, lab, results=res)
    fire.fire_fitness(ctx, res, kind, device=True, out=fit)
    fire.fire_group_mean(ctx, fit, reps, device=True, out=mean)
    ctx.sync()
    return mean, lab


def run_screened_ga(ctx, m, land, sur: Surrogate, ignition, pop=256, pool=1024,
                    reps=16, generations=50, ga_seed=1, sim_seed=1,
                    kind=fire.FITNESS_JACCARD, lo=-30.0, hi=30.0, init=None,
                    finetune_steps=32, finetune_lr=3e-4, replay_cap=8192,
                    explore=0.25):
    """The GA with surrogate screening: each generation breeds `pool`
    candidates from the `pop` evaluated parents (ga_step over the parents
    tiled pool / pop times), ranks them by predicted fitness, and simulates
    only `pop` of them (pool = 4 pop simulates a quarter): the best
    (1 - explore) pop by predicted fitness and explore pop drawn uniformly
    from the rest (seeded), so that candidates the surrogate wrongly rejects
    still reach the automaton; generation 0 screens `pool` draws of the
    initial prior the same way.  The automaton runs of the simulated
    candidates also yield their burn fractions, which join a replay buffer
    the surrogate is fine-tuned on for `finetune_steps` Adam steps per
    generation (0: no fine-tuning), so that it stays accurate where the GA
    is searching."""
    torch = _torch()
    dev = torch.device("cuda", ctx.device)
    H, W = land.veg.shape
    S = sur.S
    cells = (H // S) * (W // S)
    assert pool % pop == 0
    rep = pool // pop
    planes = sur.planes(land)
    tfrac = torch.empty((S, S), dtype=torch.float32, device=dev)
    fire.fire_net_target_frac(ctx, m, S, tfrac, sync=True)
    ign = torch.tensor(np.tile(np.asarray(ignition, np.int32), (pool, 1)),
                       device=dev)
    if init is None:
        init = synth.gauss_population(pool, ga_seed)
    cand = torch.tensor(np.clip(np.asarray(init, np.float64), lo, hi),
                        device=dev)
    tlo = torch.full((5,), float(lo), dtype=torch.float64, device=dev)
    thi = torch.full((5,), float(hi), dtype=torch.float64, device=dev)
    pred = torch.empty(pool, dtype=torch.float64, device=dev)
    rank = torch.empty(pool, dtype=torch.int32, device=dev)
    n_top = pop - int(round(explore * pop))
    rng = np.random.default_rng(ga_seed + 7919)
    nxt = torch.empty_like(cand)
    replay = None
    hist = ScreenedHistory()
    for g in range(generations):
        t0 = time.perf_counter()
        prob = sur.predict(planes, H, W, cand, ign)
        fire.fire_net_screen(ctx, S, prob, tfrac, cells, kind, pool, pred,
                             rank)
        ctx.sync()
        order = rank.cpu().numpy()
        rest = order[n_top:]
        pick = np.concatenate([order[:n_top],
                               rng.choice(rest, pop - n_top, replace=False)])
        genes = cand[torch.as_tensor(pick, device=dev).long()].contiguous()
        seed0 = sim_seed + g * pop * reps
        f, lab = _evaluate_with_labels(ctx, m, sur, genes, ign, seed0, reps,
                                       kind)
        hist.params.append(genes.cpu().numpy())
        hist.fitness.append(f.cpu().numpy())
        hist.predicted.append(pred.cpu().numpy())
        if finetune_steps:
            chunk = Dataset(H, W, planes, genes, ign[:pop].contiguous(), lab)
            if replay is None:
                replay = chunk
            else:
                start = max(0, len(replay) + pop - replay_cap)
                replay = Dataset(
                    H, W, planes,
                    torch.cat([replay.params[start:], genes]),
                    torch.cat([replay.ign[start:], chunk.ign]),
                    torch.cat([replay.labels[start:], lab]))
            sur.train([replay], steps=finetune_steps, lr=finetune_lr,
                      seed=g + 1)
        if g + 1 < generations:
            torch.cuda.synchronize(dev)
            fire.ga_step(ctx, genes.repeat(rep, 1).contiguous(),
                         f.repeat(rep).contiguous(), g, generations, ga_seed,
                         tlo, thi, device=True, out=nxt)
            ctx.sync()
            cand, nxt = nxt, cand
        hist.seconds.append(time.perf_counter() - t0)
    return hist
