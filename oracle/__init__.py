"""CPU oracle for the stochastic fire-spread automaton (arXiv:1701.03549).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it.

The arithmetic lives in ``fire_oracle.c`` (plain single-threaded C, double
precision, compiled with ``-ffp-contract=off``); this module compiles it on
first use and exposes it through ctypes.  See ``fire_oracle.c`` for the
paper passages each function follows (Eq. 1, Sec. 2.1 covariates, the
synchronous update of Sec. 2.1/2.3, the Philox generator of Sec. 2.3 and the
fitness of Eq. 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fire_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_BORDER = 1
STATUS_STEP_CAP = 2
KIND_PAPER_DELTA = 0
KIND_JACCARD = 1

# direction offsets off(d) = (drow, dcol), bearing 45 d degrees
DIRS = ((-1, 0), (-1, 1), (0, 1), (1, 1), (1, 0), (1, -1), (0, -1), (-1, -1))


def build(force: bool = False) -> str:
    """Compile fire_oracle.c into liboracle.so (in place)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class _Map(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32),
                ("psi", C.c_void_p), ("sig", C.c_void_p),
                ("cw", C.c_void_p), ("sw", C.c_void_p),
                ("up", C.c_void_p), ("forest", C.c_void_p),
                ("burnable", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C")
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.orc_draw.restype = C.c_uint32
        L.orc_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int]
        for f in ("orc_exp", "orc_cosd", "orc_sind", "orc_logistic"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_double]
        L.orc_threshold_of_z.restype = C.c_uint64
        L.orc_threshold_of_z.argtypes = [C.c_double]
        L.orc_omega.restype = C.c_double
        L.orc_omega.argtypes = [C.c_float, C.c_float, C.c_int]
        L.orc_features.restype = C.c_int
        L.orc_features.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 12
        L.orc_z.restype = C.c_double
        L.orc_z.argtypes = [C.POINTER(_Map), C.c_void_p, C.c_long, C.c_int]
        L.orc_thresholds.argtypes = [C.POINTER(_Map), C.c_void_p, C.c_void_p]
        L.orc_simulate.restype = C.c_int
        L.orc_simulate.argtypes = [C.POINTER(_Map), C.c_void_p, C.c_void_p,
                                   C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                   C.c_void_p, C.c_void_p]
        L.orc_simulate_mode.restype = C.c_int
        L.orc_simulate_mode.argtypes = [C.POINTER(_Map), C.c_void_p,
                                        C.c_void_p, C.c_int, C.c_int,
                                        C.c_uint64, C.c_uint32, C.c_int,
                                        C.c_void_p, C.c_void_p]
        L.orc_simulate_burnout.restype = C.c_int
        L.orc_simulate_burnout.argtypes = [C.POINTER(_Map), C.c_void_p,
                                           C.c_void_p, C.c_int, C.c_int,
                                           C.c_uint64, C.c_uint32, C.c_void_p,
                                           C.c_void_p, C.c_void_p]
        L.orc_burn_frequency_burnout.restype = C.c_int
        L.orc_burn_frequency_burnout.argtypes = [C.POINTER(_Map), C.c_void_p,
                                                 C.c_int, C.c_int, C.c_uint64,
                                                 C.c_long, C.c_void_p,
                                                 C.c_void_p]
        L.orc_burn_frequency_mode.restype = C.c_int
        L.orc_burn_frequency_mode.argtypes = [C.POINTER(_Map), C.c_void_p,
                                              C.c_int, C.c_int, C.c_uint64,
                                              C.c_long, C.c_int, C.c_void_p]
        L.orc_burn_frequency.restype = C.c_int
        L.orc_burn_frequency.argtypes = [C.POINTER(_Map), C.c_void_p, C.c_int,
                                         C.c_int, C.c_uint64, C.c_long,
                                         C.c_void_p]
        L.orc_fitness.restype = C.c_double
        L.orc_fitness.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
        L.orc_ga_step.restype = C.c_int
        L.orc_ga_step.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_int, C.c_uint64, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
        L.orc_group_mean.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.orc_ignition_search.restype = C.c_int
        L.orc_ignition_search.argtypes = [C.POINTER(_Map), C.c_void_p,
                                          C.c_void_p, C.c_int, C.c_int,
                                          C.c_int, C.c_uint64, C.c_int,
                                          C.c_double, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
        L.orc_snap_ignition.restype = C.c_int
        L.orc_snap_ignition.argtypes = [C.POINTER(_Map), C.c_void_p,
                                        C.c_double, C.c_double, C.c_void_p,
                                        C.c_void_p]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# scalar helpers

def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32),
                            np.asarray(key, np.uint32), out)
    return out


def philox4x64_10(ctr, key):
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(np.asarray(ctr, np.uint64),
                            np.asarray(key, np.uint64), out)
    return out


def draw(seed: int, cell: int, step: int, d: int) -> int:
    return int(lib().orc_draw(seed, cell, step, d))


def spec_exp(x: float) -> float:
    return lib().orc_exp(x)


def cosd(x: float) -> float:
    return lib().orc_cosd(x)


def sind(x: float) -> float:
    return lib().orc_sind(x)


def logistic(z: float) -> float:
    return lib().orc_logistic(z)


def threshold_of_z(z: float) -> int:
    return int(lib().orc_threshold_of_z(z))


def omega(cw: float, sw: float, d: int) -> float:
    return lib().orc_omega(cw, sw, d)


def fitness(burnt: int, inter: int, target: int, kind: int = 0) -> float:
    return lib().orc_fitness(burnt, inter, target, kind)


def ga_step(genes, fitness, generation, total_gens, seed, lo, hi):
    """One generation of the Appendix B genetic algorithm (see
    fire_oracle.c for the reading of its unspecified constants)."""
    g = np.ascontiguousarray(genes, np.float64)
    P, G = g.shape
    f = np.ascontiguousarray(fitness, np.float64).reshape(P)
    lo = np.ascontiguousarray(lo, np.float64).reshape(G)
    hi = np.ascontiguousarray(hi, np.float64).reshape(G)
    out = np.zeros_like(g)
    rc = lib().orc_ga_step(P, G, _p(g), _p(f), int(generation),
                           int(total_gens), int(seed), _p(lo), _p(hi), _p(out))
    if rc:
        raise ValueError(f"orc_ga_step failed ({rc})")
    return out


def group_mean(values, per_group):
    v = np.ascontiguousarray(values, np.float64)
    groups = v.size // per_group
    out = np.zeros(groups, np.float64)
    lib().orc_group_mean(_p(v), groups, per_group, _p(out))
    return out


# ---------------------------------------------------------------------------
# maps

class Features:
    """Per-cell covariates of Eq. 1 computed by the oracle."""

    def __init__(self, land):
        veg = np.ascontiguousarray(land.veg, np.uint8)
        H, W = veg.shape
        self.H, self.W = H, W
        f32 = lambda a: np.ascontiguousarray(a, np.float32)
        elev, slope = f32(land.elev), f32(land.slope)
        aspect, wind = f32(land.aspect), f32(land.wind)
        self.psi = np.zeros((H, W), np.float32)
        self.sig = np.zeros((H, W), np.float32)
        self.cw = np.zeros((H, W), np.float32)
        self.sw = np.zeros((H, W), np.float32)
        self.up = np.zeros((H, W), np.uint8)
        self.forest = np.zeros((H, W), np.uint8)
        self.burnable = np.zeros((H, W), np.uint8)
        rc = lib().orc_features(H, W, _p(veg), _p(elev), _p(slope),
                                _p(aspect), _p(wind), _p(self.psi),
                                _p(self.sig), _p(self.cw), _p(self.sw),
                                _p(self.up), _p(self.forest),
                                _p(self.burnable))
        if rc:
            raise ValueError("bad map shape")
        self._m = _Map(H, W, _p(self.psi).value, _p(self.sig).value,
                       _p(self.cw).value, _p(self.sw).value,
                       _p(self.up).value, _p(self.forest).value,
                       _p(self.burnable).value)

    def z(self, beta, i: int, d: int) -> float:
        b = np.ascontiguousarray(beta, np.float64)
        return lib().orc_z(C.byref(self._m), _p(b), i, d)

    def thresholds(self, beta) -> np.ndarray:
        """uint64 table T[d, row, col] (Eq. 1 thresholds)."""
        b = np.ascontiguousarray(beta, np.float64)
        T = np.zeros((8, self.H, self.W), np.uint64)
        lib().orc_thresholds(C.byref(self._m), _p(b), _p(T))
        return T

    def simulate(self, beta, ignition, seed: int, target=None,
                 want_steps: bool = True, max_steps: int = 0, mode: int = 0,
                 burn_time=None):
        """Run one fire; returns (result dict, burn-step map or None).
        mode 0: one trial per burning neighbour; mode 1: one uniform per
        cell against 1 - prod(1 - p_i) (see fire_oracle.c).  burn_time
        (uint8 (H, W), mode 0 only): steps each cell burns once ignited."""
        b = np.ascontiguousarray(beta, np.float64)
        res = np.zeros(6, np.uint32)
        bs = np.zeros((self.H, self.W), np.int32) if want_steps else None
        tg = None if target is None else np.ascontiguousarray(target,
                                                              np.uint8)
        if burn_time is not None:
            if mode != 0:
                raise ValueError("burn times apply to the per-neighbour rule")
            bt = np.ascontiguousarray(burn_time, np.uint8).reshape(self.H,
                                                                   self.W)
            rc = lib().orc_simulate_burnout(
                C.byref(self._m), None if tg is None else _p(tg), _p(b),
                int(ignition[0]), int(ignition[1]), int(seed), int(max_steps),
                _p(bt), None if bs is None else _p(bs), _p(res))
            if rc == -1:
                raise ValueError("burn time 0 on a burnable cell")
        else:
            rc = lib().orc_simulate_mode(C.byref(self._m),
                                         None if tg is None else _p(tg), _p(b),
                                         int(ignition[0]), int(ignition[1]),
                                         int(seed), int(max_steps), int(mode),
                                         None if bs is None else _p(bs),
                                         _p(res))
        if rc == -4:
            raise ValueError("ignition outside the grid or non-burnable")
        if rc:
            raise RuntimeError(f"oracle simulate failed ({rc})")
        out = dict(burnt=int(res[0]), inter=int(res[1]), target=int(res[2]),
                   steps=int(res[3]), status=int(res[4]), trials=int(res[5]))
        return out, bs

    def ignition_search(self, target, beta, lat_h, lat_w, reps, seed,
                        kind=KIND_PAPER_DELTA, cutoff=1.5):
        """Lattice ignition search (see fire_oracle.c): returns
        (fitness map (lat_h, lat_w), cells (lat_h, lat_w, 2) as (row, col),
        [x mean, x sd, y mean, y sd])."""
        b = np.ascontiguousarray(beta, np.float64)
        tg = np.ascontiguousarray(target, np.uint8)
        fm = np.zeros((lat_h, lat_w), np.float64)
        cells = np.zeros((lat_h, lat_w, 2), np.int32)
        xy = np.zeros(4, np.float64)
        rc = lib().orc_ignition_search(C.byref(self._m), _p(tg), _p(b),
                                       int(lat_h), int(lat_w), int(reps),
                                       int(seed), int(kind), float(cutoff),
                                       _p(fm), _p(cells), _p(xy))
        if rc:
            raise ValueError("target has no burnable burnt cell")
        return fm, cells, xy

    def snap_ignition(self, target, x: float, y: float):
        """Ignition cell (row, col) of the genes x (column) and y (row): the
        burnable target cell nearest to the clamped, rounded point (see
        fire_oracle.c)."""
        tg = np.ascontiguousarray(target, np.uint8)
        r = np.zeros(1, np.int32)
        c = np.zeros(1, np.int32)
        rc = lib().orc_snap_ignition(C.byref(self._m), _p(tg), float(x),
                                     float(y), _p(r), _p(c))
        if rc:
            raise ValueError("target has no burnable burnt cell")
        return int(r[0]), int(c[0])

    def burn_frequency(self, beta, ignition, seed0: int, nseeds: int,
                       mode: int = 0, burn_time=None):
        b = np.ascontiguousarray(beta, np.float64)
        counts = np.zeros((self.H, self.W), np.uint32)
        if burn_time is not None:
            bt = np.ascontiguousarray(burn_time, np.uint8).reshape(self.H,
                                                                   self.W)
            rc = lib().orc_burn_frequency_burnout(
                C.byref(self._m), _p(b), int(ignition[0]), int(ignition[1]),
                int(seed0), int(nseeds), _p(bt), _p(counts))
        else:
            rc = lib().orc_burn_frequency_mode(C.byref(self._m), _p(b),
                                               int(ignition[0]),
                                               int(ignition[1]), int(seed0),
                                               int(nseeds), int(mode),
                                               _p(counts))
        if rc:
            raise RuntimeError(f"oracle burn_frequency failed ({rc})")
        return counts
