"""Pins for the covariates of Eq. 1 (Sec. 2.1) as the oracle computes them.

Each test builds a map whose covariates have a closed form from the paper's
definitions (vegetation indicator, relative aspect, relative wind, slope
only when going uphill) and checks the oracle's values and thresholds
against that closed form, evaluated with scipy's logistic.
"""
import math

import numpy as np
import pytest
from scipy.special import expit

from paper_1701_03549_gb300 import synth

DIRS = ((-1, 0), (-1, 1), (0, 1), (1, 1), (1, 0), (1, -1), (0, -1), (-1, -1))
N, NE, E, SE, S, SW, W, NW = range(8)


def _land(H=6, W=7, veg=2, slope=0.0, aspect=0.0, wind=0.0, elev=None):
    L = synth.uniform_landscape(H, W, veg_code=veg, wind_deg=wind)
    L.slope[:] = slope
    L.aspect[:] = aspect
    if elev is not None:
        L.elev[:] = elev
    return L


def _T(p):
    return math.floor(p * 2 ** 32)


def test_vegetation_indicator_and_burnable(oracle_mod):
    L = _land()
    L.veg[:] = np.array([0, 1, 2, 3, 4, 1, 0])[None, :]
    F = oracle_mod.Features(L)
    assert F.forest[0].tolist() == [0, 1, 0, 0, 0, 1, 0]
    assert F.burnable[0].tolist() == [0, 1, 1, 1, 1, 1, 0]


@pytest.mark.parametrize("aspect,want", [(315.0, 1.0), (135.0, -1.0),
                                         (45.0, 0.0), (225.0, 0.0),
                                         (0.0, math.sqrt(0.5))])
def test_relative_aspect(oracle_mod, aspect, want):
    """psi = cos(aspect - 315 deg): +1 facing NW, -1 facing SE (Sec. 2.1)."""
    F = oracle_mod.Features(_land(slope=20.0, aspect=aspect))
    assert abs(float(F.psi[2, 2]) - want) < 1e-7


def test_relative_aspect_is_zero_on_gentle_slopes(oracle_mod):
    F = oracle_mod.Features(_land(slope=5.0, aspect=315.0))
    assert np.all(F.psi == 0.0)
    F = oracle_mod.Features(_land(slope=5.01, aspect=315.0))
    assert np.all(F.psi == 1.0)


def test_slope_term_is_slope_over_100(oracle_mod):
    F = oracle_mod.Features(_land(slope=37.5))
    assert np.all(F.sig == np.float32(0.375))


def test_relative_wind_equals_cosine_of_bearing_difference(oracle_mod):
    """omega = cos(phi_w - phi_c) with phi_c the bearing source -> target."""
    rng = np.random.default_rng(1)
    for phi_w in rng.uniform(0, 360, 200).astype(np.float32):
        F = oracle_mod.Features(_land(H=3, W=3, wind=float(phi_w)))
        for d in range(8):
            om = oracle_mod.omega(float(F.cw[1, 1]), float(F.sw[1, 1]), d)
            assert abs(om - math.cos(math.radians(phi_w - 45 * d))) < 3e-7


def test_wind_sign_is_plus_one_downwind(oracle_mod):
    """Wind blowing toward the east: a fire stepping east (source west of the
    target) is downwind (+1), stepping west is upwind (-1), N/S crosswind."""
    F = oracle_mod.Features(_land(H=3, W=3, wind=90.0))
    cw, sw = float(F.cw[1, 1]), float(F.sw[1, 1])
    assert oracle_mod.omega(cw, sw, E) == 1.0
    assert oracle_mod.omega(cw, sw, W) == -1.0
    assert oracle_mod.omega(cw, sw, N) == 0.0
    assert oracle_mod.omega(cw, sw, S) == 0.0


def test_uphill_mask_on_an_eastward_ramp(oracle_mod):
    """Elevation rising to the east: a step east goes uphill (sigma used),
    a step west goes downhill, north/south steps are level (sigma ignored)."""
    H, W = 5, 6
    elev = np.tile(np.arange(W, dtype=np.float32) * 10.0, (H, 1))
    F = oracle_mod.Features(_land(H, W, elev=elev, slope=18.0))
    up = F.up[2, 3]
    for d, want in ((E, 1), (NE, 1), (SE, 1), (W, 0), (NW, 0), (SW, 0),
                    (N, 0), (S, 0)):
        assert (up >> d) & 1 == want, d


def test_up_mask_ignores_out_of_grid_sources(oracle_mod):
    elev = np.zeros((3, 3), np.float32)
    elev[0, 0] = 5.0
    F = oracle_mod.Features(_land(3, 3, elev=elev))
    # corner cell: only sources inside the grid can set bits
    assert F.up[0, 0] == 0b11111111 & sum(
        1 << d for d, (dr, dc) in enumerate(DIRS)
        if 0 <= -dr < 3 and 0 <= -dc < 3)


def test_thresholds_baseline_only(oracle_mod):
    """beta = (b0, 0, 0, 0, 0): every threshold is floor(2^32 expit(b0))."""
    L = synth.landscape(20, 24, seed=3)
    F = oracle_mod.Features(L)
    for b0 in (-3.0, 0.7, 2.5):
        T = F.thresholds([b0, 0, 0, 0, 0])
        assert np.all(T == _T(expit(b0)))


def test_thresholds_forest_term(oracle_mod):
    L = synth.landscape(16, 16, seed=4)
    F = oracle_mod.Features(L)
    T = F.thresholds([-1.0, 2.0, 0, 0, 0])
    forest = F.forest.astype(bool)
    assert np.all(T[:, forest] == _T(expit(1.0)))
    assert np.all(T[:, ~forest] == _T(expit(-1.0)))


def test_thresholds_wind_term_by_direction(oracle_mod):
    F = oracle_mod.Features(_land(4, 4, wind=90.0))
    T = F.thresholds([-0.5, 0, 0, 1.5, 0])
    assert np.all(T[E] == _T(expit(1.0)))
    assert np.all(T[W] == _T(expit(-2.0)))
    assert np.all(T[N] == _T(expit(-0.5)))
    assert np.all(T[S] == _T(expit(-0.5)))


def test_thresholds_slope_term_only_uphill(oracle_mod):
    H, W = 4, 5
    elev = np.tile(np.arange(W, dtype=np.float32), (H, 1))
    F = oracle_mod.Features(_land(H, W, elev=elev, slope=40.0))
    T = F.thresholds([0.0, 0, 0, 0, 2.0])
    inner = (slice(None), slice(1, None))
    assert np.all(T[E][inner] == _T(expit(2.0 * float(np.float32(0.4)))))
    assert np.all(T[W] == 1 << 31)
    assert np.all(T[N] == 1 << 31)


def test_thresholds_aspect_term(oracle_mod):
    F = oracle_mod.Features(_land(slope=30.0, aspect=135.0))
    T = F.thresholds([1.0, 0, 2.0, 0, 0])
    assert np.all(T == _T(expit(-1.0)))


def test_threshold_sums_terms_in_equation_order(oracle_mod):
    """Spot check of a full z against an independent float64 evaluation."""
    L = synth.landscape(12, 12, seed=9, wind_seed=9)
    F = oracle_mod.Features(L)
    beta = [-5.0, -10.0, 5.0, 18.1, -5.0]
    for i in range(0, 144, 7):
        r, c = divmod(i, 12)
        for d in range(8):
            om = math.cos(math.radians(float(L.wind[r, c]) - 45 * d))
            sr, sc = r - DIRS[d][0], c - DIRS[d][1]
            upd = (0 <= sr < 12 and 0 <= sc < 12
                   and L.elev[r, c] > L.elev[sr, sc])
            psi = (math.cos(math.radians(float(L.aspect[r, c]) - 315.0))
                   if L.slope[r, c] > 5.0 else 0.0)
            z = (beta[0] + beta[1] * (L.veg[r, c] == 1) + beta[2] * psi
                 + beta[3] * om + beta[4] * (float(L.slope[r, c]) / 100.0
                                             if upd else 0.0))
            assert abs(F.z(beta, i, d) - z) < 2e-5
