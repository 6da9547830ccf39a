"""What the trained surrogate gains over the method without it.

A small surrogate (S = 32 on a 128 x 128 landscape) is trained on burn
fractions from automaton runs with parameters drawn from the GA's initial
prior.  On a fresh pool of candidates from the same prior, each scored by
the automaton itself (16 replicates), the surrogate's top quarter must

* have a clearly lower true mean fitness than the pool (what a plain GA, or
  a random quarter, would simulate), and
* hold most of the pool's true best tenth;

and on held-out samples its cross-entropy must beat the best
parameter-blind predictor (the training labels' per-cell mean).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1701_03549_gb300 import calibrate, fire, surrogate, synth  # noqa

TRUTH = np.array(synth.TRUTH_BETA)


def _bce(p, t):
    p = np.clip(p, 1e-6, 1 - 1e-6)
    return float(np.mean(-(t * np.log(p) + (1 - t) * np.log(1 - p))))


def test_screening_gain():
    ctx = fire.fire_create(0, torch.cuda.current_stream())
    H = W = 128
    land = synth.landscape(H, W, seed=77, wind_seed=None)
    m = ctx.landscape_upload(land)
    ign = synth.centre_ignition(land.veg)
    res, bs = m.simulate_batch(TRUTH[None], np.array([ign], np.int32),
                               np.array([2024], np.uint64), want_steps=True)
    m.target_upload(bs[0] >= 0)
    sur = surrogate.Surrogate(ctx, S=32, max_batch=32, seed=3)
    ngroups, ntrain = 4608, 4096
    params = surrogate.sample_params(ngroups, 11)
    igns = np.tile(np.array(ign, np.int32), (ngroups, 1))
    data = surrogate.make_dataset(ctx, m, land, sur, ngroups, 8, 11,
                                  params=params, ign=igns)
    train = surrogate.Dataset(H, W, data.planes, data.params[:ntrain],
                              data.ign[:ntrain], data.labels[:ntrain])
    hold = slice(ntrain, ngroups)
    losses = sur.train([train], steps=1200, lr=2e-3, lr_final=1e-4, seed=5)
    assert np.isfinite(losses).all()

    # held-out cross-entropy against the parameter-blind predictor
    prob = sur.predict(data.planes, H, W, data.params[hold].contiguous(),
                       data.ign[hold].contiguous()).cpu().numpy()
    lab = data.labels[hold].cpu().numpy()
    blind = train.labels.mean(0).cpu().numpy()
    assert _bce(prob, lab) < 0.8 * _bce(np.broadcast_to(blind, lab.shape), lab)

    # screening a fresh candidate pool, judged by the automaton
    pool = 256
    cand = surrogate.sample_params(pool, 99)
    cd = torch.tensor(cand, device="cuda")
    cign = torch.tensor(np.tile(np.array(ign, np.int32), (pool, 1)),
                        device="cuda")
    pr = sur.predict(data.planes, H, W, cd, cign)
    tf = torch.empty((32, 32), dtype=torch.float32, device="cuda")
    fire.fire_net_target_frac(ctx, m, 32, tf, sync=True)
    pred = torch.empty(pool, dtype=torch.float64, device="cuda")
    keep = torch.empty(pool // 4, dtype=torch.int32, device="cuda")
    fire.fire_net_screen(ctx, 32, pr, tf, 16.0, fire.FITNESS_JACCARD,
                         pool // 4, pred, keep, sync=True)
    true_f = calibrate.evaluate(
        ctx, m, cd, ign, calibrate.sim_seeds(7, 0, pool, 16), 16,
        fire.FITNESS_JACCARD, torch).cpu().numpy()
    kept = keep.cpu().numpy()
    best10 = set(np.argsort(true_f, kind="stable")[: pool // 10].tolist())
    caught = len(best10 & set(kept.tolist())) / len(best10)
    pr_all = pred.cpu().numpy()
    rk = lambda a: np.argsort(np.argsort(a, kind="stable"), kind="stable")
    rho = np.corrcoef(rk(pr_all), rk(true_f))[0, 1]
    print(f"pool mean {true_f.mean():.3f} kept mean {true_f[kept].mean():.3f} "
          f"best-tenth caught {caught:.2f} spearman {rho:.3f} "
          f"loss {losses[:5].mean():.4f}->{losses[-20:].mean():.4f} "
          f"heldout bce {_bce(prob, lab):.4f} blind "
          f"{_bce(np.broadcast_to(blind, lab.shape), lab):.4f}")
    assert true_f[kept].mean() < true_f.mean() - 0.05
    assert caught >= 0.5
    sur.net.free()
    ctx.close()
