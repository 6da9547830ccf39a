"""Pins for the oracle's ignition-point search: lattice placement and
snapping checked on hand-built scars, fitness against the p = 0 closed form,
and the ensemble statistics against numpy."""
import numpy as np
import pytest

from paper_1701_03549_gb300 import synth


def _flat(H, W):
    return synth.uniform_landscape(H, W)


def test_lattice_on_a_rectangular_scar(oracle_mod):
    """Scar = rows 5..14, columns 10..29 of a 20 x 30 grid: a 2 x 4 lattice
    falls at rows 5 + floor((2a + 1) 10 / 4) = 7, 12 and columns
    10 + floor((2b + 1) 20 / 8) = 12, 17, 22, 27, all inside the scar."""
    F = oracle_mod.Features(_flat(20, 30))
    tg = np.zeros((20, 30), np.uint8)
    tg[5:15, 10:30] = 1
    _, cells, _ = F.ignition_search(tg, [-1000.0, 0, 0, 0, 0], 2, 4, 1, 1)
    assert cells[:, :, 0].tolist() == [[7] * 4, [12] * 4]
    assert cells[:, :, 1].tolist() == [[12, 17, 22, 27]] * 2


def test_lattice_point_in_a_hole_snaps_to_the_nearest_burnt_cell(oracle_mod):
    """Ring scar around a 3 x 3 hole centred at (10, 10): a 1 x 1 lattice
    sits at the hole's centre, at distance^2 = 4 from (8,10), (10,8), (10,12),
    (12,10); the lowest row-major index, (8, 10), wins."""
    F = oracle_mod.Features(_flat(21, 21))
    tg = np.zeros((21, 21), np.uint8)
    tg[6:15, 6:15] = 1
    tg[9:12, 9:12] = 0
    _, cells, _ = F.ignition_search(tg, [-1000.0, 0, 0, 0, 0], 1, 1, 1, 1)
    assert cells[0, 0].tolist() == [8, 10]


def test_non_burnable_scar_cells_are_not_ignitions(oracle_mod):
    land = _flat(10, 10)
    land.veg[5, 5] = 0
    F = oracle_mod.Features(land)
    tg = np.zeros((10, 10), np.uint8)
    tg[5, 5] = 1
    tg[5, 8] = 1
    _, cells, _ = F.ignition_search(tg, [-1000.0, 0, 0, 0, 0], 1, 1, 1, 1)
    assert cells[0, 0].tolist() == [5, 8]


def test_fitness_map_for_p_zero_is_the_closed_form(oracle_mod):
    """p = 0 burns only the ignition, which lies inside the scar A, so every
    candidate scores (|A| - 1) / |A| under Eq. 2."""
    land = synth.landscape(40, 40, seed=2)
    F = oracle_mod.Features(land)
    tg = np.zeros((40, 40), np.uint8)
    tg[8:30, 5:33] = 1
    tg &= (land.veg != 0)
    A = int(tg.sum())
    fm, _, _ = F.ignition_search(tg, [-1000.0, 0, 0, 0, 0], 3, 3, 2, 7,
                                 kind=0, cutoff=10.0)
    assert np.all(fm == (A - 1) / A)


def test_ensemble_statistics(oracle_mod):
    land = synth.landscape(50, 50, seed=6, wind_seed=6)
    F = oracle_mod.Features(land)
    ign = synth.centre_ignition(land.veg)
    beta = [0.5, -0.5, 0.3, 2.5, -0.5]
    _, bs = F.simulate(beta, ign, 3)
    tg = (bs >= 0).astype(np.uint8)
    fm, cells, xy = F.ignition_search(tg, beta, 4, 4, 2, 11, kind=0,
                                      cutoff=np.inf)
    x = cells[:, :, 1].ravel().astype(float)
    y = cells[:, :, 0].ravel().astype(float)
    assert np.allclose(xy, [x.mean(), x.std(ddof=1), y.mean(), y.std(ddof=1)],
                       rtol=1e-12, atol=1e-12)
    cut = float(np.sort(fm.ravel())[5])
    fm2, cells2, xy2 = F.ignition_search(tg, beta, 4, 4, 2, 11, kind=0,
                                         cutoff=cut)
    sel = fm2.ravel() <= cut
    xs = cells2[:, :, 1].ravel()[sel].astype(float)
    ys = cells2[:, :, 0].ravel()[sel].astype(float)
    assert np.allclose(xy2, [xs.mean(), xs.std(ddof=1), ys.mean(),
                             ys.std(ddof=1)], rtol=1e-12, atol=1e-12)
    # a cutoff below every candidate: the best candidate alone
    fm3, cells3, xy3 = F.ignition_search(tg, beta, 4, 4, 2, 11, kind=0,
                                         cutoff=-1.0)
    b = int(np.argmin(fm3.ravel()))
    assert xy3.tolist() == [cells3.reshape(-1, 2)[b, 1], 0.0,
                            cells3.reshape(-1, 2)[b, 0], 0.0]


# ---------------------------------------------------------------------------
# The ignition point as two more genes (Sec. 3, Table 3): gene x (column) and
# y (row) clamped to the grid, rounded half up, moved to the nearest burnable
# cell of the target burnt area (ties to the lower row-major index).

def _snap_scene():
    """9 x 11 burnable map; target cells (2, 2), (2, 6), (6, 4), (5, 9) and a
    burnt but non-burnable cell (4, 4)."""
    land = synth.uniform_landscape(9, 11)
    land.veg[4, 4] = 0
    t = np.zeros((9, 11), bool)
    for rc in ((2, 2), (2, 6), (6, 4), (5, 9), (4, 4)):
        t[rc] = True
    return land, t


# (x, y) -> (row, col), worked out by hand on the scene above
SNAP_CASES = [
    ((4.0, 2.0), (2, 2)),    # (2,2) and (2,6) both at d^2 = 4: lower index
    ((4.0, 4.0), (6, 4)),    # (4,4) is at 0 but non-burnable; (6,4) at 4
    ((4.5, 2.0), (2, 6)),    # half up: column 5, d^2 1 against 9
    ((50.0, 0.0), (2, 6)),   # clamped to column 10: (2,6) 20, (5,9) 26
    ((9.0, 5.0), (5, 9)),    # exactly on a target cell
    ((-7.0, 100.0), (6, 4)), # clamped to (8, 0): (6,4) 20, (2,2) 40
]


def test_snap_ignition_worked_cases(oracle_mod):
    land, t = _snap_scene()
    F = oracle_mod.Features(land)
    for xy, want in SNAP_CASES:
        assert F.snap_ignition(t, *xy) == want, xy


def test_snap_ignition_nan_and_empty_target(oracle_mod):
    land, t = _snap_scene()
    F = oracle_mod.Features(land)
    assert F.snap_ignition(t, float("nan"), float("nan")) == (2, 2)
    with pytest.raises(ValueError):
        F.snap_ignition(np.zeros_like(t), 3.0, 3.0)
    only_blocked = np.zeros_like(t)
    only_blocked[4, 4] = True
    with pytest.raises(ValueError):
        F.snap_ignition(only_blocked, 3.0, 3.0)


def test_snap_ignition_is_the_nearest_by_brute_force(oracle_mod):
    """Random tiny maps and points: the cell is burnable and burnt, and no
    burnable burnt cell is nearer to the rounded point, nor equally near with
    a lower row-major index."""
    rng = np.random.default_rng(8)
    for case in range(40):
        H, W = rng.integers(2, 8, 2)
        land = synth.noise_landscape(int(H), int(W), 100 + case)
        t = rng.random((H, W)) < 0.3
        ok = t & (land.veg != 0)
        if not ok.any():
            continue
        F = oracle_mod.Features(land)
        for _ in range(6):
            x, y = rng.uniform(-2, W + 1), rng.uniform(-2, H + 1)
            r, c = F.snap_ignition(t, x, y)
            assert ok[r, c]
            C = np.floor(min(max(x, 0.0), W - 1) + 0.5)
            R = np.floor(min(max(y, 0.0), H - 1) + 0.5)
            d = (r - R) ** 2 + (c - C) ** 2
            rows, cols = np.nonzero(ok)
            dd = (rows - R) ** 2 + (cols - C) ** 2
            assert d == dd.min()
            assert r * W + c == (rows * W + cols)[dd == d].min()
