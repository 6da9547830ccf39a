"""Seeded synthetic inputs shaped like the paper's landscapes.

This module produces raster maps (vegetation, elevation, slope, aspect,
wind direction), parameter populations, ignition points and replicate
seeds.  It holds none of the fire-spread method's arithmetic: no ignition
probability, no random draw of the cellular automaton, no fitness.  Both the
CUDA library's callers and the CPU oracle take their inputs from here.

The paper fits its model on 801 x 801 rasters of a Patagonian landscape at
30 m resolution (Section 2.1, Fig. 1).  Those rasters are not available, so
seeded synthetic maps stand in for them:

* elevation: a sum of 20 Gaussian hills (centres uniform over the extent,
  widths uniform in [0.05, 0.25] x extent, amplitudes uniform in [0, 1]),
  rescaled to 0-2000 m on 30 m cells;
* slope and aspect: central differences of the elevation (one-sided at the
  edges) in float64, cast to float32.  Aspect is the compass bearing of the
  downslope direction, clockwise from north (0 on flat cells);
* vegetation: Gaussian-smoothed white noise (sigma 4 cells) split at its
  quartiles into codes 1..4, then 10 % of the cells, chosen uniformly, set to
  code 0 (non-burnable).  Code 1 is forest (Section 2.1: the indicator I_f);
* wind direction: constant (45 degrees, blowing toward the north-east) or a
  smooth seeded field scaled to [0, 360).

Row 0 is the northern edge and column 0 the western edge of every raster.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CELL_M = 30.0
RELIEF_M = 2000.0
N_HILLS = 20

# Reference-fire parameters (beta_0 .. beta_4) of the paper's synthetic
# experiment, Table 2 ("Reference value" column).
TRUTH_BETA = (-5.0, -10.0, 5.0, 18.1, -5.0)
# Seed of the replicate that produces a workload's target (reference) fire.
TARGET_SEED = 0x7A96E7
# Initial distributions of Table 1.
GAUSS_PRIOR_SD = 5.0
UNIFORM_BOUNDS = (-30.0, 30.0)


@dataclass
class Landscape:
    """Raster inputs of one fire, all row-major (H, W)."""

    veg: np.ndarray        # uint8, 0 non-burnable, 1 forest, 2..4 other fuels
    elev: np.ndarray       # float32 metres
    slope: np.ndarray      # float32 degrees
    aspect: np.ndarray     # float32 degrees, bearing of downslope direction
    wind: np.ndarray       # float32 degrees, bearing the wind blows toward
    cell_m: float = CELL_M
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.veg.shape


def _gaussian_smooth(a: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter

    return gaussian_filter(a, sigma=sigma, mode="reflect")


def hills_elevation(H: int, W: int, seed: int, n_hills: int = N_HILLS,
                    relief_m: float = RELIEF_M) -> np.ndarray:
    """Sum of seeded Gaussian hills rescaled to [0, relief_m] (float64)."""
    rng = np.random.default_rng([seed, 0xE1E7])
    ext = float(max(H, W))
    cy = rng.uniform(0.0, H, n_hills)
    cx = rng.uniform(0.0, W, n_hills)
    sd = rng.uniform(0.05, 0.25, n_hills) * ext
    amp = rng.uniform(0.0, 1.0, n_hills)
    rows = np.arange(H, dtype=np.float64)[:, None]
    cols = np.arange(W, dtype=np.float64)[None, :]
    z = np.zeros((H, W), dtype=np.float64)
    for i in range(n_hills):
        z += amp[i] * np.exp(-(((rows - cy[i]) ** 2) + ((cols - cx[i]) ** 2))
                             / (2.0 * sd[i] * sd[i]))
    lo, hi = z.min(), z.max()
    if hi > lo:
        z = (z - lo) / (hi - lo) * relief_m
    else:
        z = np.zeros_like(z)
    return z


def slope_aspect(elev: np.ndarray, cell_m: float = CELL_M):
    """Slope (degrees) and aspect (bearing of the downslope direction)."""
    H, W = elev.shape
    if H > 1:
        dz_drow = np.gradient(elev, cell_m, axis=0)
    else:
        dz_drow = np.zeros_like(elev)
    if W > 1:
        dz_dcol = np.gradient(elev, cell_m, axis=1)
    else:
        dz_dcol = np.zeros_like(elev)
    # rows grow southward: the northward gradient is -dz/drow
    g_east = dz_dcol
    g_north = -dz_drow
    slope = np.degrees(np.arctan(np.hypot(g_east, g_north)))
    # downslope direction is -grad; bearing = atan2(east, north)
    aspect = np.degrees(np.arctan2(-g_east, -g_north)) % 360.0
    flat = (g_east == 0.0) & (g_north == 0.0)
    aspect[flat] = 0.0
    return slope.astype(np.float32), aspect.astype(np.float32)


def vegetation(H: int, W: int, seed: int, non_burnable_frac: float = 0.10,
               smooth_sigma: float = 4.0) -> np.ndarray:
    rng = np.random.default_rng([seed, 0x7E6])
    noise = rng.standard_normal((H, W))
    sm = _gaussian_smooth(noise, smooth_sigma) if min(H, W) > 1 else noise
    q = np.quantile(sm, [0.25, 0.5, 0.75])
    veg = (1 + np.searchsorted(q, sm.ravel(), side="right")).reshape(H, W)
    veg = veg.astype(np.uint8)
    n_block = int(round(non_burnable_frac * H * W))
    if n_block:
        idx = rng.choice(H * W, size=n_block, replace=False)
        veg.ravel()[idx] = 0
    return veg


def wind_field(H: int, W: int, seed: int | None, constant_deg: float = 45.0):
    """Constant wind (seed None) or smooth seeded field in [0, 360)."""
    if seed is None:
        return np.full((H, W), constant_deg, dtype=np.float32)
    rng = np.random.default_rng([seed, 0x317D])
    noise = rng.standard_normal((H, W))
    sm = _gaussian_smooth(noise, max(H, W) / 16.0)
    lo, hi = sm.min(), sm.max()
    w = (sm - lo) / (hi - lo) * 360.0 if hi > lo else np.zeros_like(sm)
    w = np.minimum(w, np.nextafter(360.0, 0.0))
    return w.astype(np.float32)


def landscape(H: int, W: int, seed: int, wind_seed: int | None = None,
              wind_deg: float = 45.0, cell_m: float = CELL_M) -> Landscape:
    elev64 = hills_elevation(H, W, seed)
    slope, aspect = slope_aspect(elev64, cell_m)
    return Landscape(
        veg=vegetation(H, W, seed),
        elev=elev64.astype(np.float32),
        slope=slope,
        aspect=aspect,
        wind=wind_field(H, W, wind_seed, wind_deg),
        cell_m=cell_m,
        meta={"H": H, "W": W, "seed": seed, "wind_seed": wind_seed,
              "wind_deg": wind_deg},
    )


def noise_landscape(H: int, W: int, seed: int) -> Landscape:
    """Independent random rasters (no spatial structure), cheap at any size:
    fuel codes 1..4 with 10 % of cells non-burnable, elevation in [0, 2000)
    m, slope in [0, 45) degrees, aspect and wind bearings in [0, 360).  For
    size and edge cases, where the hills of landscape() would take longer
    to generate than the fires take to run."""
    rng = np.random.default_rng(seed)
    veg = rng.integers(1, 5, (H, W), dtype=np.uint8)
    veg[rng.random((H, W)) < 0.1] = 0
    f32 = np.float32
    return Landscape(
        veg=veg,
        elev=(rng.random((H, W), dtype=f32) * f32(2000.0)),
        slope=(rng.random((H, W), dtype=f32) * f32(45.0)),
        aspect=(rng.random((H, W), dtype=f32) * f32(360.0)),
        wind=(rng.random((H, W), dtype=f32) * f32(360.0)),
        meta={"H": H, "W": W, "seed": seed, "kind": "noise"},
    )


def uniform_landscape(H: int, W: int, veg_code: int = 2, wind_deg: float = 0.0,
                      elev: float = 100.0) -> Landscape:
    """Flat, fully burnable terrain (for closed-form checks)."""
    z = np.full((H, W), elev, dtype=np.float32)
    return Landscape(
        veg=np.full((H, W), veg_code, dtype=np.uint8),
        elev=z,
        slope=np.zeros((H, W), dtype=np.float32),
        aspect=np.zeros((H, W), dtype=np.float32),
        wind=np.full((H, W), wind_deg, dtype=np.float32),
    )


def centre_ignition(veg: np.ndarray):
    """Burnable cell nearest the grid centre; ties go to the lower index."""
    H, W = veg.shape
    rows, cols = np.nonzero(veg != 0)
    if rows.size == 0:
        raise ValueError("no burnable cell")
    cr, cc = (H - 1) / 2.0, (W - 1) / 2.0
    d2 = (rows - cr) ** 2 + (cols - cc) ** 2
    best = np.flatnonzero(d2 == d2.min())
    lin = rows[best] * W + cols[best]
    k = best[np.argmin(lin)]
    return int(rows[k]), int(cols[k])


def gauss_population(n: int, seed: int, genes: int = 5,
                     sd: float = GAUSS_PRIOR_SD) -> np.ndarray:
    rng = np.random.default_rng([seed, 0x6A55])
    return rng.normal(0.0, sd, size=(n, genes)).astype(np.float64)


def uniform_population(n: int, seed: int, genes: int = 5,
                       lo: float = UNIFORM_BOUNDS[0],
                       hi: float = UNIFORM_BOUNDS[1]) -> np.ndarray:
    rng = np.random.default_rng([seed, 0x0F0F])
    return rng.uniform(lo, hi, size=(n, genes)).astype(np.float64)


def burnt_area_points(area: np.ndarray, n: int, seed: int) -> np.ndarray:
    """n points (x = column, y = row) drawn uniformly from the cells set in
    `area` (the initial ignition genes of the variable-ignition GA: the
    paper starts those fires from random points of the reference fire's
    burnt area), as float64 (n, 2)."""
    rows, cols = np.nonzero(np.asarray(area))
    if rows.size == 0:
        raise ValueError("empty area")
    rng = np.random.default_rng([seed, 0x16A1])
    k = rng.integers(0, rows.size, n)
    return np.stack([cols[k], rows[k]], axis=1).astype(np.float64)


def replicate_seeds(n: int, first: int = 1) -> np.ndarray:
    return np.arange(first, first + n, dtype=np.uint64)


# Workload presets.  Sizes follow the five configurations the library is
# measured on; the map seed of preset i is i + 1.
PRESETS = {
    "single_fire_128": dict(H=128, W=128, map_seed=1, wind_seed=None,
                            n_sims=64),
    "ga_generation_512": dict(H=512, W=512, map_seed=2, wind_seed=None,
                              population=256, replicates=16),
    "ignition_search_1024": dict(H=1024, W=1024, map_seed=3, wind_seed=3,
                                 lattice=32, replicates=64),
}


def uneven_fire_shapes():
    """Grid shapes of the nine-fire uneven batch: 200x300 ... 2000x1500."""
    return [(200 + 225 * i, 300 + 150 * i) for i in range(9)]


def preset_landscape(name: str) -> Landscape:
    p = PRESETS[name]
    return landscape(p["H"], p["W"], p["map_seed"], wind_seed=p["wind_seed"])
