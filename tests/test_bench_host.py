"""Host logic of the benchmark on CPU: the clock-sample summary, the memory
roofline arithmetic from a committed ncu record, the staleness rule for that
record (a record whose source hash differs from the kernel sources gives no
traffic), and the dense-sweep reference rate."""
import json

import numpy as np

import pytest

import bench


def _row(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active",
         cap="Not Active", power="812.40"):
    return f"{sm}, {smax}, {power}, {hw}, {hwt}, {swt}, {cap}\n"


def test_clock_summary_median_max_and_reasons():
    lines = [_row(1965, 2070), _row(1950, 2070, cap="Active"),
             _row(1980, 2070), "garbage line\n",
             "1, 2, 3\n", _row("[N/A]", 2070)]
    c = bench.Clocks.summarise(lines)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 1965
    assert c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_empty():
    c = bench.Clocks.summarise([_row(1400, 2070, hwt="Active"),
                                _row(1410, 2070, swt="Active")])
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.Clocks.summarise([]) is None
    assert bench.Clocks.summarise(["not, a, clock\n"]) is None


def _record(tmp_path, sha):
    d = {"source_sha256": sha, "dram_bytes_per_launch": 2.0e8,
         "l2_bytes_per_launch": 8.0e10, "ncu_duration_ms": 20.0,
         "l2_pct_of_peak_sectors": 10.0}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "rec.json").write_text(json.dumps(d))
    return d


def test_memory_roofs_from_record(tmp_path, monkeypatch):
    _record(tmp_path, "abc")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "abc")
    r = bench._memory_roofs(0.025, {"hbm_gbs": 8000.0}, "measured", "rec.json")
    assert r["dram_gbs"] == pytest.approx(2.0e8 / 0.025 / 1e9)
    assert r["dram_frac"] == pytest.approx(8.0 / 8000.0)
    # the L2 peak is the record's own rate over its fraction of peak sectors
    l2_peak = 8.0e10 / 0.020 / 1e9 / 0.10
    assert r["l2_peak_gbs"] == pytest.approx(l2_peak)
    assert r["l2_frac"] == pytest.approx(8.0e10 / 0.025 / 1e9 / l2_peak)


def test_stale_record_gives_no_traffic(tmp_path, monkeypatch):
    _record(tmp_path, "abc")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "changed")
    assert bench._committed_profile("rec.json") is None
    assert bench._memory_roofs(0.025, {}, "measured", "rec.json") is None
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "abc")
    assert bench._committed_profile("rec.json")["dram_bytes_per_launch"] == 2.0e8


def test_missing_record_gives_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._committed_profile("rec.json") is None


def test_dense_sweep_reference_rate():
    r = bench._dense_sweep_roof(1.0e13, {"hbm_gbs": 6000.0}, "measured")
    assert r["dense_rate"] == pytest.approx(6000.0e9 / 0.5)
    assert r["ratio"] == pytest.approx(1.0e13 / 1.2e13)


def test_trial_op_count():
    # a quarter of one Philox4x32-10 block: 10 rounds of (two 32x32->64
    # multiplies as 4 operations, two 3-way xors as 4, two key additions)
    # over 4 words = 25 integer operations; Eq. 1 in one direction, the
    # logistic and the comparison with the draw: about 15 single-precision
    # operations
    assert bench.OPS_PER_TRIAL == 10 * (4 + 4 + 2) // 4 + 15


def test_oracle_extrapolation_is_per_fire():
    """Batch time = sum over fires of (simulations of the fire x mean
    single-core seconds of its sampled simulations) / cores."""
    res = [(0, 1.0, 5), (0, 3.0, 9), (1, 10.0, 40)]
    est = bench._extrapolate(res, {0: 100, 1: 10}, 4)
    assert est == pytest.approx((100 * 2.0 + 10 * 10.0) / 4)


def test_both_arms_name_the_same_config():
    """The native line and the oracle arm print the same config object (the
    launch shape sits outside it), so the two lines compare like for like."""
    for kind in ("uneven", "ga512"):
        a, b = bench._config(kind, 1), bench._config(kind, 1)
        assert a == b and "launch" not in a
        assert a["l2"] == bench.L2_NOTE
    assert bench._config("uneven", 1)["sims_per_step"] == 100_000
    assert bench._config("uneven", 1)["cells_total"] == sum(
        H * W for H, W in bench.synth.uneven_fire_shapes())


def test_stratified_sample_of_the_uneven_batch():
    """16 simulations per fire, evenly spaced within each fire's block of
    the batch, ordered so that every prefix of 9 covers the nine fires."""
    from paper_1701_03549_gb300 import workloads

    counts = [11112] + [11111] * 8
    mos = np.repeat(np.arange(9), counts)
    idx = workloads.stratified_sample(mos, 16)
    assert idx.size == 144 and len(set(idx.tolist())) == 144
    assert np.array_equal(np.bincount(mos[idx], minlength=9), [16] * 9)
    for k in range(16):
        assert sorted(mos[idx[9 * k:9 * k + 9]].tolist()) == list(range(9))
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    for j in range(9):
        pos = np.sort(idx[mos[idx] == j]) - starts[j]
        assert pos[0] == 0 and np.all(np.diff(pos) >= counts[j] // 16)


def test_recovery_errors_and_times():
    """The recovery report: ensemble = mean of the best tenth of a
    generation; a parameter is recovered once its relative error is within
    5 %; the time is the GA's cumulative seconds through that generation."""
    from paper_1701_03549_gb300 import calibrate

    truth = np.array([-5.0, -10.0, 5.0, 18.1, -5.0])
    P = np.tile(truth, (20, 1))
    P[:2] *= 1.2                           # the two best are 20 % off
    h = calibrate.History([P, np.tile(truth, (20, 1))],
                          [np.arange(20.0), np.arange(20.0)], [1.5, 2.0])
    ens, errs = bench._param_errors(h, truth)
    assert np.allclose(errs[0], 0.2) and np.allclose(errs[1], 0.0)
    rec, per = bench._time_to_recover(errs, h.seconds)
    assert rec == 3.5 and per == [3.5] * 5
    rec, per = bench._time_to_recover(errs[:1], h.seconds[:1])
    assert rec is None and per == [None] * 5


def test_crossover_side_interpolates_log_log():
    """The crossover side is read off the measured per-simulation times by
    straight-line interpolation in log(side) against log(time)."""
    sides = (512, 1024, 2048)
    per = (0.01, 0.04, 0.16)
    assert bench._crossover_side(sides, per, 0.02) == pytest.approx(512 * 2 ** 0.5)
    assert bench._crossover_side(sides, per, 0.04) == pytest.approx(1024)
    assert bench._crossover_side(sides, per, 0.005) is None
    assert bench._crossover_side(sides, per, 0.2) is None


def test_nearest_burnable_cell_and_tie_rule():
    """Scar ignitions of the multi-scar recovery: the burnable cell nearest a
    point, ties to the lower (row-major) index."""
    veg = np.zeros((7, 9), np.uint8)
    veg[2, 3] = veg[2, 5] = veg[6, 8] = 1
    assert bench._nearest_burnable(veg, 2, 4) == (2, 3)   # tie: lower index
    assert bench._nearest_burnable(veg, 2, 5) == (2, 5)
    assert bench._nearest_burnable(veg, 6, 6) == (6, 8)



def test_kernel_hash_ignores_comments_only():
    """The key of the committed ncu records hashes the kernel's code with its
    comments stripped: editing a comment keeps it, editing code changes it,
    and comment markers inside literals are code."""
    a = "int f(int x) {  // add one\n    return x + 1; /* done */\n}\n"
    b = "/* header */\nint f(int x) {\n\n    return x + 1;   // changed note\n}\n"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench._strip_comments(a) == bench._strip_comments(b)
    assert bench._strip_comments(a) != bench._strip_comments(c)
    s = 'const char *p = "// kept"; char q = \'/\';'
    assert bench._strip_comments(s) == s


def test_forced_launch_option():
    """--launch W,B,Q,S sets that shape on the context in place of the
    autotuner's pick; without it the autotuner decides."""
    class Ctx:
        def __init__(self):
            self.shape = None

        def set_launch(self, *a):
            self.shape = a

    class Args:
        launch = "8,4,3072,2"

    c = Ctx()
    t = bench._forced_launch(Args(), c)
    assert c.shape == (8, 4, 3072, 2)
    assert (t["warps_per_block"], t["blocks_per_sm"], t["queue_entries"],
            t["state_mode"], t["forced"]) == (8, 4, 3072, 2, True)
    Args.launch = ""
    assert bench._forced_launch(Args(), Ctx()) is None
