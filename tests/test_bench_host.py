"""Host-side helpers of bench.py, on the CPU: the DRAM traffic figure the roofline
object takes from the committed ncu summary of the substep kernel, the peak it
divides by, and the parser of the clock samples taken during the timed region
(fed canned nvidia-smi lines; no GPU, no nvidia-smi)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_comes_from_the_committed_profile():
    # the summary's per-atom-substep figure times the atom count of a launch
    path = os.path.join(ROOT, "profiles", "substep_tile_track_2M.md")
    rows = [ln for ln in open(path) if ln.startswith("| traffic_bytes_per_atom_substep |")]
    assert len(rows) == 1
    per_atom = float(rows[0].split("|")[2])
    assert 30.0 < per_atom < 116.0          # below the int32-ELL algorithmic 116 B
    assert bench._traffic_from_profile(4_000_000) == per_atom * 4_000_000


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench._peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("\n".join(lines) + "\n")
    return s.stop()


def test_clock_parser_median_max_and_reasons():
    idle = "Not Active"
    got = _sampler([
        f"0, 2070, 2070, 900.5, 0x0, {idle}, {idle}, {idle}, {idle}",
        f"0, 1965, 2070, 1390.2, 0x4, {idle}, {idle}, {idle}, Active",
        f"0, 2055, 2070, 1201.0, 0x0, {idle}, {idle}, {idle}, {idle}",
        "garbled line",
        "0, [N/A], 2070, 1.0, 0x0, a, b, c, d",
    ])
    assert got == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_parser_reports_thermal_reasons():
    got = _sampler(["0, 1500, 2070, 1000, 0x0, Not Active, Active, Active, Not Active"])
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_parser_without_samples():
    assert _sampler([]) is None
    assert bench.ClockSampler(0).stop() is None   # never started (no nvidia-smi)


def test_job_value_counts_every_replica():
    # 2 replicas x 4M atoms x 100 substeps x 20 steps in 10.08 ms per step
    v = bench.job_value(2, 4_000_000, 100, 20, 20 * 10.08)
    assert abs(v - 2 * 4e6 * 100 / 10.08e-3) < 1e-3 * v
