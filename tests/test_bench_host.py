"""Host logic of the benchmark on CPU: the clock-sample summary, the memory
roofline arithmetic from a committed ncu record, the staleness rule for that
record (a record whose source hash differs from the kernel sources gives no
traffic), and the dense-sweep reference rate."""
import json

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
    # one Philox4x32-10 word: 10 rounds x 8 ops over 4 words; Eq. 1 and the
    # comparison: 4 FMAs, exp 2, 1 + e 1, reciprocal 1, draw to float 2,
    # compare 1
    assert bench.OPS_PER_TRIAL == 10 * 8 // 4 + (4 + 2 + 1 + 1 + 2 + 1)
