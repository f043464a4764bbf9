"""Host logic of bench.py on the CPU: the peak and traffic lookups behind the
roofline object, the kernel-source hash that keeps stale DRAM counters out
of it, and the parsing of the clock samples taken during the timed region.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_hash_ignores_comments_but_not_code():
    src = open(os.path.join(ROOT, bench.KERNEL_SOURCES[0])).read()
    base = bench._code_only(src)
    edited = src.replace("\n", "\n// a remark\n", 3) + "\n/* block\n comment */\n   \n"
    assert bench._code_only(edited) == base
    assert bench._code_only(src.replace("kLanes", "kLanez", 1)) != base
    # a comment marker inside a code token is not a comment
    assert bench._code_only("a = b / c; // x\nd = e /* y */ * f;") == "a = b / c; d = e * f;"


def test_traffic_is_reported_only_for_the_current_kernel(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"kernel_hash": bench.kernel_hash(), "dram_bytes_per_launch": 123456789}
    data = {"moving-cylinder:f32": entry,
            "moving-cylinder:f16": dict(entry, kernel_hash="0" * 16),
            "moving-cylinder:f32:aa": dict(entry, dram_bytes_per_launch=42)}
    (prof / "fused_step_dram_moving_cylinder_16384x4096.json").write_text(json.dumps(data))
    h = bench.kernel_hash()  # of the real sources, before ROOT moves to the fixture
    monkeypatch.setattr(bench, "kernel_hash", lambda: h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch("moving-cylinder", "f32") == 123456789.0
    assert bench.traffic_per_launch("moving-cylinder", "f16") is None  # other kernel code
    assert bench.traffic_per_launch("moving-cylinder", "bf16") is None  # never captured
    assert bench.traffic_per_launch("moving-cylinder", "f32", "aa") == 42.0


def test_committed_counters_name_the_workload_and_their_command():
    d = json.load(open(os.path.join(ROOT, "profiles",
                                    "fused_step_dram_moving_cylinder_16384x4096.json")))
    for key, e in d.items():
        if key.startswith("_"):
            continue
        assert key.startswith("moving-cylinder:")
        assert e["dram_bytes_per_launch"] == e["dram_bytes_read"] + e["dram_bytes_write"]
        assert "--clock-control none" in e["command"] and "python bench.py" in e["command"]
        # no re-reads: DRAM traffic within a few percent of the algorithmic bytes
        assert 0.95 < e["dram_bytes_per_launch"] / e["algorithmic_bytes_per_launch"] < 1.05


def test_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6666.6}))
    assert bench.hbm_peak() == (6666.6, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.proc = _Done()
    c.lines = [
        "2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "2055, 2070, 1201.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
    ]
    r = c.stop()
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    c2 = bench.ClockSampler(0)
    c2.proc = _Done()
    c2.lines = ["1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active"]
    assert c2.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).stop() is None  # never started


@pytest.mark.parametrize("storage,expected", [("f32", 73.0), ("f16", 37.0), ("bf16", 37.0),
                                              ("f64", 145.0)])
def test_algorithmic_bytes_per_node(storage, expected):
    """9 populations read and written in the storage type plus the 1-byte mask."""
    size = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}[storage]
    assert bench.ALGO_BYTES[storage] == expected == 2 * 9 * size + 1


def test_clock_records_that_disqualify_a_run():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9}
    assert bench.clocks_rejected(ok) is None
    assert bench.clocks_rejected(None) is None  # nvidia-smi unavailable: nothing to judge
    capped = dict(ok, sm_mhz=1500.0, reasons=["sw_power_cap"])
    assert bench.clocks_rejected(capped) is None  # kept, and noted by its reasons
    assert bench.clocks_rejected(dict(ok, reasons=["hw_slowdown"])) == "hw_slowdown"
    assert bench.clocks_rejected(dict(ok, reasons=["sw_power_cap", "sw_thermal_slowdown"])) \
        == "sw_thermal_slowdown"
    assert "no reason" in bench.clocks_rejected(dict(ok, sm_mhz=1200.0))  # a leftover clock lock


@pytest.mark.parametrize("name,nx,ny,collision", [
    ("circular-couette", 128, 128, "srt"), ("cylinder-re100", 1024, 256, "mrt"),
    ("cylinder-re1000", 4096, 1024, "mrt"), ("moving-cylinder", 16384, 4096, "mrt")])
def test_workloads_are_the_configurations_and_take_the_storage(name, nx, ny, collision):
    w = bench.make_workload(name, "bf16")
    assert (w.nx, w.ny, w.collision, w.storage) == (nx, ny, collision, "bf16")
