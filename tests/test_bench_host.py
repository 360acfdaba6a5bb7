"""Host-side parts of bench.py, without a GPU: the reference arm's JSON line
(the CPU oracle timed on a bounded sample), the clock-record parser, the
algorithmic-bytes formula and the rule that a stored DRAM-traffic figure is
only reported for the sources it was measured on."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1",
                          "--steps", "2", "--warmup", "1"], check=True, capture_output=True, text=True,
                         cwd=ROOT, timeout=600).stdout.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "queries/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["config"]["workload"].startswith(bench.WORKLOAD_NAMES[1])


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1",
                          "--steps", "1", "--warmup", "0"], check=True, capture_output=True, text=True,
                         cwd=ROOT, env=env, timeout=600).stdout
    assert out.strip() == ""


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_parser():
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = [
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbled line",
        "[N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = s.stop()
    assert c["samples"] == 3 and c["sm_mhz"] == 2055.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    s.lines.append("1200, 2070, 800, 0x48, Not Active, Active, Not Active, Not Active")
    assert bench.ClockSampler.stop(s)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_bytes():
    cnt = {"extracted": 3, "edges": 10, "relaxed": 4, "pushed": 5, "touched": 7}
    # X (offsets 8 + distance W) + E (target 4 + weight 4 + W) + R (W) + P (queue write + read) + touched (W)
    assert bench.algorithmic_bytes(cnt, 4, False) == 3 * 12 + 10 * 12 + 4 * 4 + 5 * 8 + 7 * 4
    # A*: coordinates of every extracted and every improved vertex
    assert bench.algorithmic_bytes(cnt, 4, True) == 3 * 20 + 10 * 12 + 4 * 12 + 5 * 8 + 7 * 4
    assert bench.algorithmic_bytes(cnt, 8, False) == 3 * 16 + 10 * 16 + 4 * 8 + 5 * 8 + 7 * 8


def test_traffic_only_for_the_measured_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2506_16488_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "engine.cu").write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.engine_source_hash()
    (tmp_path / "profiles" / "engine_traffic.json").write_text(
        json.dumps({"source_hash": h, "workload": "w", "dram_bytes_per_launch": 123}))
    assert bench.read_traffic("w") == 123
    assert bench.read_traffic("another workload") is None
    (csrc / "engine.cu").write_text("kernel v2\n")
    assert bench.engine_source_hash() != h
    assert bench.read_traffic("w") is None


def test_peaks_from_measured_file_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6658.6}))
    assert bench.read_peaks() == (6658.6, "measured")


def test_group_time_stats():
    import numpy as np

    from paper_2506_16488_gb300 import ppsp

    class P:
        def __init__(self, ns):
            self.ns = ns

        def group_times(self):
            if self.ns is None:
                raise ppsp.PPSPError(ppsp.ERR_INVALID_ARG)
            return np.asarray(self.ns, dtype=np.uint64)

    st = bench.group_time_stats(P([1_000_000, 4_000_000, 0, 16_000_000]))
    assert st["groups"] == 3 and st["max"] == 16.0 and st["p50"] == 4.0
    assert abs(st["geomean"] - 4.0) < 1e-12  # (1 * 4 * 16) ** (1/3)
    assert bench.group_time_stats(P([0, 0])) is None
    assert bench.group_time_stats(P(None)) is None
