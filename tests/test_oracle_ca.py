"""Pins for the oracle's automaton (Sec. 2.1 rules, Sec. 2.3) and fitness.

* p = 0 and p = 1 closed forms (only the ignition burns; the 8-connected
  burnable component burns with burn step equal to the Chebyshev or BFS
  distance);
* exact enumeration of burn probabilities on grids of at most 3 x 3 cells
  against the oracle's Monte Carlo frequencies, within a binomial bound;
* structural invariants of every trajectory; D4 symmetry of isotropic fires;
* the fitness of Eq. 2 against set arithmetic.
"""
import json
import math
import os
from collections import deque

import numpy as np
import pytest

from paper_1701_03549_gb300 import synth
from tests.exact_enum import exact_burn_probability

DIRS = ((-1, 0), (-1, 1), (0, 1), (1, 1), (1, 0), (1, -1), (0, -1), (-1, -1))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bfs(burnable, src):
    H, W = burnable.shape
    dist = np.full((H, W), -1, np.int64)
    dist[src] = 0
    q = deque([src])
    while q:
        r, c = q.popleft()
        for dr, dc in DIRS:
            rr, cc = r + dr, c + dc
            if 0 <= rr < H and 0 <= cc < W and burnable[rr, cc] and \
                    dist[rr, cc] < 0:
                dist[rr, cc] = dist[r, c] + 1
                q.append((rr, cc))
    return dist


def test_p_zero_burns_only_the_ignition(oracle_mod):
    L = synth.landscape(40, 50, seed=2)
    F = oracle_mod.Features(L)
    ign = synth.centre_ignition(L.veg)
    res, bs = F.simulate([-1000.0, 0, 0, 0, 0], ign, seed=5)
    assert res["burnt"] == 1 and res["steps"] == 1
    assert bs[ign] == 0 and np.count_nonzero(bs >= 0) == 1


def test_p_one_chebyshev_distance_on_uniform_terrain(oracle_mod):
    L = synth.uniform_landscape(37, 53)
    F = oracle_mod.Features(L)
    ign = (11, 29)
    res, bs = F.simulate([1000.0, 0, 0, 0, 0], ign, seed=9)
    rr, cc = np.mgrid[0:37, 0:53]
    cheb = np.maximum(abs(rr - ign[0]), abs(cc - ign[1]))
    assert np.array_equal(bs, cheb)
    assert res["burnt"] == 37 * 53
    assert res["steps"] == cheb.max() + 1
    assert res["status"] & 1


def test_p_one_bfs_distance_with_obstacles(oracle_mod):
    L = synth.landscape(45, 38, seed=12)
    rng = np.random.default_rng(0)
    L.veg[rng.random(L.veg.shape) < 0.35] = 0
    F = oracle_mod.Features(L)
    ign = synth.centre_ignition(L.veg)
    res, bs = F.simulate([1000.0, 0, 0, 0, 0], ign, seed=1)
    dist = _bfs(L.veg != 0, ign)
    want = np.where(L.veg == 0, -2, dist)
    assert np.array_equal(bs, want)
    assert res["burnt"] == int((dist >= 0).sum())


def test_single_trial_probability_on_a_1x2_grid(oracle_mod):
    """Two cells: the second burns iff its only trial succeeds, P = T/2^32."""
    L = synth.uniform_landscape(1, 2)
    F = oracle_mod.Features(L)
    beta = [0.3, 0, 0, 0, 0]
    T = F.thresholds(beta)[6, 0, 0]   # target (0,0), source (0,1): west step
    n = 40000
    cnt = F.burn_frequency(beta, (0, 1), 1, n)
    p = T / 2 ** 32
    assert abs(cnt[0, 0] / n - p) <= 5 * math.sqrt(p * (1 - p) / n) + 1 / n


def _z_with_threshold(oracle_mod, T):
    """The least z whose threshold floor(p(z) 2^32) is >= T (bisection; the
    threshold is non-decreasing in z)."""
    lo, hi = -40.0, 40.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if oracle_mod.threshold_of_z(mid) >= T:
            hi = mid
        else:
            lo = mid
    return hi


def test_a_draw_equal_to_its_threshold_fails(oracle_mod):
    """A trial succeeds iff its draw is strictly below its threshold.  On a
    1 x 2 flat grid (z = beta_0 exactly) beta_0 is set so that the only
    trial's threshold equals its draw: the fire stays at the ignition; with
    the threshold one above the draw it spreads.  (A statistical pin cannot
    see this boundary: it decides one trial in 2^32.)"""
    L = synth.uniform_landscape(1, 2)
    F = oracle_mod.Features(L)
    seed = 12345
    # target (0, 1), burning source (0, 0) to its west: direction E, d = 2
    u = oracle_mod.draw(seed, 1, 0, 2)
    assert 1000 < u < 2 ** 32 - 1000
    for T, burnt in ((u, 1), (u + 1, 2)):
        z = _z_with_threshold(oracle_mod, T)
        assert oracle_mod.threshold_of_z(z) == T
        assert int(F.thresholds([z, 0, 0, 0, 0])[2, 0, 1]) == T
        res, _ = F.simulate([z, 0, 0, 0, 0], (0, 0), seed)
        assert res["burnt"] == burnt and res["trials"] == 1


@pytest.mark.parametrize("shape,seed", [((1, 1), 0), ((1, 2), 1), ((2, 2), 2),
                                        ((2, 3), 3), ((3, 3), 4),
                                        ((3, 3), 5)])
def test_exact_enumeration_matches_monte_carlo(oracle_mod, shape, seed):
    H, W = shape
    rng = np.random.default_rng(100 + seed)
    L = synth.landscape(H, W, seed=seed, wind_seed=None,
                        wind_deg=float(rng.uniform(0, 360)))
    L.slope[:] = rng.uniform(0, 30, (H, W)).astype(np.float32)
    L.aspect[:] = rng.uniform(0, 360, (H, W)).astype(np.float32)
    L.elev[:] = rng.uniform(0, 100, (H, W)).astype(np.float32)
    L.veg[:] = rng.integers(1, 3, (H, W)).astype(np.uint8)
    if H * W == 9:
        L.veg[0, 2] = 0
    F = oracle_mod.Features(L)
    beta = rng.uniform(-3, 3, 5)
    for ign in [(r, c) for r in range(H) for c in range(W) if L.veg[r, c]]:
        T = F.thresholds(beta)
        p = exact_burn_probability(L.veg != 0, T, ign)
        n = 60000 if H * W > 4 else 20000
        cnt = F.burn_frequency(beta, ign, 1000 * seed + 1, n)
        ph = cnt / n
        bound = 5 * np.sqrt(p * (1 - p) / n) + 1.0 / n
        assert np.all(np.abs(ph - p) <= bound), (ign, p, ph)


def test_trajectory_invariants(oracle_mod):
    L = synth.landscape(96, 80, seed=21, wind_seed=21)
    F = oracle_mod.Features(L)
    ign = synth.centre_ignition(L.veg)
    dist = _bfs(L.veg != 0, ign)
    rng = np.random.default_rng(1)
    for s in range(6):
        beta = rng.uniform(-4, 6, 5)
        res, bs = F.simulate(beta, ign, seed=s + 1)
        H, W = bs.shape
        assert bs[ign] == 0
        burnt = bs >= 0
        assert res["burnt"] == int(burnt.sum())
        assert np.all(dist[burnt] >= 0)          # inside the component
        assert np.all(bs[burnt] >= dist[burnt])  # never faster than BFS
        assert np.all(bs[L.veg == 0] == -2)
        assert res["steps"] == bs.max() + 1
        # every ignited cell had a neighbour burning one step before, and the
        # trial count equals the (unburnt target, burning source) pairs
        trials = 0
        for r in range(H):
            for c in range(W):
                k = bs[r, c]
                nb = [bs[r + dr, c + dc] for dr, dc in DIRS
                      if 0 <= r + dr < H and 0 <= c + dc < W]
                if k > 0:
                    assert (k - 1) in nb
                if L.veg[r, c]:
                    last = k if k >= 0 else res["steps"]
                    trials += sum(1 for v in nb if 0 <= v < last)
        assert res["trials"] == trials


def test_isotropic_fire_is_d4_symmetric(oracle_mod):
    """Only beta_0 set on flat uniform terrain: burn frequencies are invariant
    under the rotations and reflections of the square."""
    n = 9
    L = synth.uniform_landscape(n, n)
    F = oracle_mod.Features(L)
    N = 4000
    cnt = F.burn_frequency([-0.4, 0, 0, 0, 0], (4, 4), 77, N) / N
    for g in (np.rot90(cnt), np.rot90(cnt, 2), np.fliplr(cnt), cnt.T):
        sd = np.sqrt(np.maximum(cnt * (1 - cnt), 1e-4) * 2 / N)
        assert np.all(np.abs(g - cnt) <= 6 * sd + 2.0 / N)


def test_wind_elongates_the_scar_downwind(oracle_mod):
    L = synth.uniform_landscape(41, 41, wind_deg=90.0)
    F = oracle_mod.Features(L)
    cnt = F.burn_frequency([-1.2, 0, 0, 2.5, 0], (20, 20), 5, 300)
    rows, cols = np.nonzero(cnt)
    w = cnt[rows, cols]
    assert (w * (cols - 20)).sum() / w.sum() > 1.0   # mass east of ignition


def test_step_cap_and_bad_ignition(oracle_mod):
    L = synth.uniform_landscape(20, 20)
    F = oracle_mod.Features(L)
    res, _ = F.simulate([1000.0, 0, 0, 0, 0], (10, 10), 1, max_steps=3)
    assert res["status"] & 2 and res["steps"] == 3
    L.veg[3, 3] = 0
    F = oracle_mod.Features(L)
    with pytest.raises(ValueError):
        F.simulate([0.0] * 5, (3, 3), 1)
    with pytest.raises(ValueError):
        F.simulate([0.0] * 5, (20, 3), 1)


def test_fitness_against_set_arithmetic(oracle_mod):
    rng = np.random.default_rng(2)
    for _ in range(200):
        A = set(rng.choice(400, rng.integers(1, 120), replace=False).tolist())
        As = set(rng.choice(400, rng.integers(0, 120), replace=False).tolist())
        b, i, t = len(As), len(A & As), len(A)
        sym = len(A ^ As)
        assert oracle_mod.fitness(b, i, t, 0) == pytest.approx(sym / len(A),
                                                               rel=1e-15)
        assert oracle_mod.fitness(b, i, t, 1) == pytest.approx(
            sym / len(A | As), rel=1e-15)


def test_fitness_golden_cases(oracle_mod):
    with open(os.path.join(GOLDEN, "fitness_eq2.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        got = oracle_mod.fitness(c["burnt"], c["inter"], c["target"],
                                 c["kind"])
        assert got == pytest.approx(c["fitness"], rel=1e-15), c


def test_target_map_counts(oracle_mod):
    L = synth.landscape(30, 30, seed=8)
    F = oracle_mod.Features(L)
    ign = synth.centre_ignition(L.veg)
    _, tb = F.simulate([1.0, 0, 0, 0, 0], ign, seed=3)
    tgt = tb >= 0
    res, bs = F.simulate([1.0, 0, 0, 0, 0], ign, seed=4, target=tgt)
    assert res["target"] == int(tgt.sum())
    assert res["inter"] == int(((bs >= 0) & tgt).sum())


# --- the paper's one-uniform-per-cell update (Sec. 2.3), oracle mode 1 -----

def test_cell_uniform_p_zero_and_p_one(oracle_mod):
    L = synth.uniform_landscape(31, 29)
    F = oracle_mod.Features(L)
    res, bs = F.simulate([-1000.0, 0, 0, 0, 0], (10, 10), 3, mode=1)
    assert res["burnt"] == 1 and res["steps"] == 1
    res, bs = F.simulate([1000.0, 0, 0, 0, 0], (10, 10), 3, mode=1)
    rr, cc = np.mgrid[0:31, 0:29]
    assert np.array_equal(bs, np.maximum(abs(rr - 10), abs(cc - 10)))


@pytest.mark.parametrize("shape,seed", [((2, 2), 7), ((3, 3), 8), ((2, 3), 9)])
def test_cell_uniform_matches_the_per_neighbour_distribution(oracle_mod, shape,
                                                             seed):
    """One uniform against 1 - prod(1 - p_i) and one trial per neighbour give
    the same ignition probability (up to threshold rounding, far below the
    Monte Carlo error), so the per-neighbour exact enumeration pins the
    cell-uniform rule too."""
    H, W = shape
    rng = np.random.default_rng(200 + seed)
    L = synth.landscape(H, W, seed=seed, wind_deg=float(rng.uniform(0, 360)))
    L.slope[:] = rng.uniform(0, 30, (H, W)).astype(np.float32)
    L.elev[:] = rng.uniform(0, 100, (H, W)).astype(np.float32)
    L.veg[:] = rng.integers(1, 3, (H, W)).astype(np.uint8)
    F = oracle_mod.Features(L)
    beta = rng.uniform(-2, 2, 5)
    T = F.thresholds(beta)
    ign = (0, 0)
    p = exact_burn_probability(L.veg != 0, T, ign)
    n = 60000
    cnt = F.burn_frequency(beta, ign, 5000 + seed, n, mode=1)
    ph = cnt / n
    assert np.all(np.abs(ph - p) <= 5 * np.sqrt(p * (1 - p) / n) + 2.0 / n)
