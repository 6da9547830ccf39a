"""Pins for the oracle's burn-out times (a cell burns burn_time steps once
ignited; the paper's rule, Sec. 2.1, is one step for every fuel).

* burn_time = 1 everywhere reproduces the paper's rule exactly;
* p = 0: the ignition burns alone for its burn time (steps = burn_time);
  p = 1 on uniform terrain: burn steps stay the Chebyshev distance and the
  fire lasts max distance + burn time steps;
* closed forms on lines, where a target is tried once per step of its
  burning neighbour: P(second cell of 1x2 burns) = 1 - (1 - p)^k, and on
  1x3 with per-cell times the product over the two links, against Monte
  Carlo within a binomial bound;
* on random maps with per-fuel times: every ignited cell had a neighbour
  burning in the step before, the fire lasts max(burn step + burn time)
  steps, and the trial count equals the overlaps of each neighbour's burning
  window with the target's unburnt window.
"""
import math

import numpy as np
import pytest

from paper_1701_03549_gb300 import synth

DIRS = ((-1, 0), (-1, 1), (0, 1), (1, 1), (1, 0), (1, -1), (0, -1), (-1, -1))


def _per_fuel(veg, times):
    """Burn time per cell from a per-class table (class = min(veg, 4))."""
    return np.asarray(times, np.uint8)[np.minimum(veg, 4)]


def test_unit_burn_time_is_the_papers_rule(oracle_mod):
    rng = np.random.default_rng(0)
    L = synth.landscape(48, 40, seed=5, wind_seed=5)
    F = oracle_mod.Features(L)
    ign = synth.centre_ignition(L.veg)
    ones = np.ones(L.veg.shape, np.uint8)
    for s in range(5):
        beta = rng.uniform(-3, 6, 5)
        r0, b0 = F.simulate(beta, ign, seed=s + 1)
        r1, b1 = F.simulate(beta, ign, seed=s + 1, burn_time=ones)
        assert r0 == r1 and np.array_equal(b0, b1)


def test_p_zero_and_p_one(oracle_mod):
    L = synth.uniform_landscape(21, 27)
    F = oracle_mod.Features(L)
    bt = np.full(L.veg.shape, 3, np.uint8)
    r, bs = F.simulate([-1000.0, 0, 0, 0, 0], (10, 10), 2, burn_time=bt)
    assert r["burnt"] == 1 and r["steps"] == 3
    r, bs = F.simulate([1000.0, 0, 0, 0, 0], (10, 10), 2, burn_time=bt)
    rr, cc = np.mgrid[0:21, 0:27]
    cheb = np.maximum(abs(rr - 10), abs(cc - 10))
    assert np.array_equal(bs, cheb)
    assert r["steps"] == cheb.max() + 3


@pytest.mark.parametrize("k", [2, 3, 5])
def test_line_of_two_closed_form(oracle_mod, k):
    L = synth.uniform_landscape(1, 2)
    F = oracle_mod.Features(L)
    beta = [-1.2, 0, 0, 0, 0]
    p = F.thresholds(beta)[2, 0, 1] / 2 ** 32     # (0,1) from its west source
    bt = np.array([[k, 1]], np.uint8)
    n = 40000
    cnt = F.burn_frequency(beta, (0, 0), 11, n, burn_time=bt)
    want = 1 - (1 - p) ** k
    assert abs(cnt[0, 1] / n - want) <= 5 * math.sqrt(want * (1 - want) / n) + 1 / n


def test_line_of_three_per_cell_times(oracle_mod):
    L = synth.uniform_landscape(1, 3, wind_deg=90.0)
    F = oracle_mod.Features(L)
    beta = [-1.5, 0, 0, 0.8, 0]
    T = F.thresholds(beta)
    pa = T[2, 0, 1] / 2 ** 32
    pb = T[2, 0, 2] / 2 ** 32
    bt = np.array([[3, 2, 4]], np.uint8)
    n = 60000
    cnt = F.burn_frequency(beta, (0, 0), 77, n, burn_time=bt) / n
    p1 = 1 - (1 - pa) ** 3
    p2 = p1 * (1 - (1 - pb) ** 2)
    for got, want in ((cnt[0, 1], p1), (cnt[0, 2], p2)):
        assert abs(got - want) <= 5 * math.sqrt(want * (1 - want) / n) + 1 / n


def test_trajectory_invariants_with_per_fuel_times(oracle_mod):
    L = synth.landscape(40, 36, seed=9, wind_seed=9)
    F = oracle_mod.Features(L)
    bt = _per_fuel(L.veg, [1, 3, 1, 2, 4])
    ign = synth.centre_ignition(L.veg)
    rng = np.random.default_rng(4)
    H, W = L.veg.shape
    for s in range(5):
        beta = rng.uniform(-4, 4, 5)
        res, bs = F.simulate(beta, ign, seed=100 + s, burn_time=bt)
        burnt = bs >= 0
        assert res["burnt"] == int(burnt.sum())
        assert res["steps"] == int((bs + bt.astype(np.int64))[burnt].max())
        trials = 0
        for r in range(H):
            for c in range(W):
                if not L.veg[r, c]:
                    continue
                last = bs[r, c] if bs[r, c] >= 0 else res["steps"]
                for dr, dc in DIRS:
                    sr, sc = r - dr, c - dc
                    if not (0 <= sr < H and 0 <= sc < W) or bs[sr, sc] < 0:
                        continue
                    lo = bs[sr, sc]
                    hi = bs[sr, sc] + int(bt[sr, sc]) - 1
                    trials += max(0, min(hi, last - 1) - lo + 1)
                if bs[r, c] > 0:
                    ok = False
                    for dr, dc in DIRS:
                        sr, sc = r - dr, c - dc
                        if 0 <= sr < H and 0 <= sc < W and bs[sr, sc] >= 0 and \
                                bs[sr, sc] <= bs[r, c] - 1 <= \
                                bs[sr, sc] + int(bt[sr, sc]) - 1:
                            ok = True
                    assert ok, (r, c)
        assert res["trials"] == trials


def test_zero_burn_time_is_rejected(oracle_mod):
    L = synth.uniform_landscape(5, 5)
    F = oracle_mod.Features(L)
    bt = np.ones((5, 5), np.uint8)
    bt[1, 1] = 0
    with pytest.raises(ValueError):
        F.simulate([0.0] * 5, (2, 2), 1, burn_time=bt)
