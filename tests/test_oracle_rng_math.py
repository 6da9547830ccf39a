"""Pins for the oracle's random numbers and elementary functions.

Each check ties the oracle to something other than itself: numpy's Philox
implementation, cuRAND's Philox4x32-10 block function compiled for the host,
the platform libm, mpmath at high precision, closed forms and distributional
properties.
"""
import math
import os

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")


# --- Philox (Sec. 2.3; Salmon et al. SC'11) --------------------------------

def test_philox_round_structure_matches_numpy_4x64(oracle_mod):
    """The generic Philox round structure, instantiated for 64-bit words,
    reproduces numpy's Philox4x64-10 (numpy increments its counter before
    generating a block, so its first block is that of counter + 1)."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        bg = np.random.Philox(counter=ctr, key=key)
        want = bg.random_raw(4)
        c1 = ctr.copy()
        c1[0] += np.uint64(1)
        got = oracle_mod.philox4x64_10(c1, key)
        assert np.array_equal(got, want)


_CURAND_HDR = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"),
                           "include", "curand_philox4x32_x.h")


def _curand_host_blocks(tmp_path):
    """cuRAND's public Philox4x32-10 block function compiled for the host
    (tests/curand_philox_host.cpp): a third-party known answer, no GPU."""
    import ctypes
    import subprocess

    if not os.path.exists(_CURAND_HDR):
        pytest.skip("CUDA headers not installed")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                       "curand_philox_host.cpp")
    so = str(tmp_path / "libcurand_philox_host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I" + os.path.dirname(_CURAND_HDR), src, "-o", so],
                   check=True)
    lib = ctypes.CDLL(so)

    def blocks(ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32)
        key = np.ascontiguousarray(key, np.uint32)
        out = np.zeros((len(ctr), 4), np.uint32)
        lib.curand_philox_blocks_host(len(ctr), ctr.ctypes.data,
                                      key.ctypes.data, out.ctypes.data)
        return out
    return blocks


def test_philox4x32_equals_curand_on_the_host(oracle_mod, tmp_path):
    """Blocks equal those of cuRAND's raw block function (built for the CPU
    from its public header) on 4096 random counters and keys and on the
    all-zero and all-one corners: multipliers, Weyl increments and the
    round count are pinned without a GPU."""
    ref = _curand_host_blocks(tmp_path)
    rng = np.random.default_rng(17)
    ctr = rng.integers(0, 2 ** 32, (4096, 4), dtype=np.uint32)
    key = rng.integers(0, 2 ** 32, (4096, 2), dtype=np.uint32)
    ones = np.uint32(0xFFFFFFFF)
    ctr[:4] = [[0, 0, 0, 0], [ones] * 4, [0, 0, 0, 0], [ones] * 4]
    key[:4] = [[0, 0], [0, 0], [ones, ones], [ones, ones]]
    want = ref(ctr, key)
    got = np.array([oracle_mod.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(got, want)


def test_philox4x32_outputs_are_uniform(oracle_mod):
    """Chi-square of the top byte and per-bit frequencies over 2^16 blocks."""
    n = 1 << 14
    outs = np.array([oracle_mod.philox4x32_10([i, 7, 0, 0], [123, 456])
                     for i in range(n)], dtype=np.uint32).ravel()
    top = outs >> 24
    hist = np.bincount(top, minlength=256)
    exp = outs.size / 256.0
    chi2 = ((hist - exp) ** 2 / exp).sum()
    # 255 dof: mean 255, sd 22.6; 6 sd bound
    assert chi2 < 255 + 6 * 22.6
    bits = ((outs[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(0)
    assert np.all(np.abs(bits - 0.5) < 6 * 0.5 / math.sqrt(outs.size))


def test_draws_differ_across_every_key_component(oracle_mod):
    base = oracle_mod.draw(5, 100, 3, 2)
    assert oracle_mod.draw(6, 100, 3, 2) != base           # seed
    assert oracle_mod.draw(5, 101, 3, 2) != base           # cell
    assert oracle_mod.draw(5, 100, 4, 2) != base           # step
    assert oracle_mod.draw(5, 100, 3, 6) != base           # other block
    assert oracle_mod.draw(5, 100, 3, 3) != base           # other word
    assert oracle_mod.draw(5 + (1 << 32), 100, 3, 2) != base  # seed high


def test_draw_is_the_keyed_block_word(oracle_mod):
    """Draw for (cell, step, d) is word d % 4 of block (cell, step, d / 4)."""
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for d in range(8):
        blk = oracle_mod.philox4x32_10([77, 9, d >> 2, 0], key)
        assert oracle_mod.draw(seed, 77, 9, d) == int(blk[d & 3])


# --- exp, cos, sin written from the mathematics ----------------------------

def _ulp_err(a, b):
    return abs(a - b) / math.ulp(b)


def test_spec_exp_within_two_ulp_of_libm(oracle_mod):
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-40, 40, 200000),
                         rng.uniform(-700, 700, 20000),
                         np.arange(-40, 41, dtype=np.float64)])
    worst = max(_ulp_err(oracle_mod.spec_exp(float(x)), math.exp(x))
                for x in xs)
    assert worst <= 2.0
    assert oracle_mod.spec_exp(0.0) == 1.0


def test_spec_exp_against_mpmath(oracle_mod):
    mpmath.mp.prec = 200
    rng = np.random.default_rng(4)
    for x in rng.uniform(-40, 40, 500):
        exact = mpmath.exp(mpmath.mpf(float(x)))
        got = oracle_mod.spec_exp(float(x))
        assert abs(mpmath.mpf(got) - exact) <= 2 * mpmath.mpf(
            math.ulp(float(exact)))


def test_degree_trig_against_libm_and_exact_points(oracle_mod):
    rng = np.random.default_rng(5)
    for a in rng.uniform(-720, 720, 50000).astype(np.float32):
        a = float(a)
        assert abs(oracle_mod.cosd(a) - math.cos(math.radians(a))) < 2e-15
        assert abs(oracle_mod.sind(a) - math.sin(math.radians(a))) < 2e-15
    for k in range(-8, 9):
        assert abs(oracle_mod.cosd(90.0 * k)) == abs(round(math.cos(
            k * math.pi / 2)))
        assert abs(oracle_mod.sind(90.0 * k)) == abs(round(math.sin(
            k * math.pi / 2)))
    r2 = math.sqrt(0.5)
    for a in (45.0, 135.0, 225.0, 315.0, -45.0):
        assert abs(abs(oracle_mod.cosd(a)) - r2) < 2e-16
        assert abs(abs(oracle_mod.sind(a)) - r2) < 2e-16


# --- threshold of Eq. 1 ------------------------------------------------------

def _exact_threshold(z):
    mpmath.mp.prec = 200
    p = 1 / (1 + mpmath.exp(-mpmath.mpf(z)))
    v = p * 2 ** 32
    return int(mpmath.floor(v)), float(v - mpmath.floor(v))


def test_threshold_matches_high_precision_logistic(oracle_mod):
    """floor(2^32 / (1 + e^-z)) agrees with a 200-bit evaluation except where
    the exact value lies within 1e-6 of an integer (rounding ties)."""
    rng = np.random.default_rng(6)
    zs = np.concatenate([rng.uniform(-30, 30, 3000), rng.normal(0, 3, 2000),
                         [-22.0, -21.0, -5.0, 0.0, 5.0, 21.0, 22.0, 35.0]])
    near = 0
    for z in zs:
        want, frac = _exact_threshold(float(z))
        got = oracle_mod.threshold_of_z(float(z))
        if min(frac, 1 - frac) < 1e-6:
            near += 1
            assert abs(got - want) <= 1
        else:
            assert got == want, (z, got, want)
    assert near < 10


def test_threshold_special_values_and_monotonicity(oracle_mod):
    t = oracle_mod.threshold_of_z
    assert t(0.0) == 1 << 31
    assert t(40.0) == 1 << 32 and t(1000.0) == 1 << 32
    assert t(-40.0) == 0 and t(-1000.0) == 0
    assert t(-23.0) == 0  # 2^32 e^-23 < 1
    zs = np.sort(np.random.default_rng(7).uniform(-45, 45, 20000))
    ts = [t(float(z)) for z in zs]
    assert all(a <= b for a, b in zip(ts, ts[1:]))
    # symmetry of the logistic: T(z) + T(-z) is 2^32 or 2^32 - 1
    for z in np.random.default_rng(8).uniform(-20, 20, 2000):
        s = t(float(z)) + t(float(-z))
        assert s in ((1 << 32) - 1, 1 << 32)
