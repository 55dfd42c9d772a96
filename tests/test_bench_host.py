"""Host-side logic of bench.py, on the CPU: the capture-hash gate of the
reported DRAM traffic and binary64 issue counts, the binary64-pipe roofline
arithmetic, the peak lookup and the parsing of nvidia-smi clock samples."""
import json
import os

import pytest

import bench


def test_captures_apply_only_to_their_sources():
    good = dict(bench.TRAFFIC_CAPTURE)
    if not bench._sources_match(good):
        pytest.skip("the kernel sources changed since the committed capture (the bench reports null)")
    assert bench._captured_traffic() == good["dram_bytes_per_launch"]
    bad = dict(good, sha256="0" * 64)
    assert not bench._sources_match(bad)
    moved = dict(good, sources=good["sources"][:-1])
    assert not bench._sources_match(moved)


def test_fp64_roofline_counts_issue_slots():
    if not bench._sources_match(bench.FP64_OPS_CAPTURE):
        pytest.skip("the kernel sources changed since the committed capture")
    r = bench._fp64_roofline(1.0e8, 0.25)
    per = bench.FP64_OPS_CAPTURE["warp_instructions_per_segment"]
    assert r["achieved"] == pytest.approx(per * 1.0e8 / 0.25 / 1e9)
    assert r["peak"] == pytest.approx(4 * 152 * 2.070e9 / 64 / 1e9)
    assert r["frac"] == pytest.approx(per * 1.0e8 / 0.25 / (4 * 152 * 2.070e9 / 64))
    assert r["bound"] == "alu"


def test_peak_is_the_measured_hbm_copy_bandwidth():
    peak, kind = bench._peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert peak == pytest.approx(float(json.load(f)["hbm_gbs"]))
        assert kind == "measured"
    else:
        assert kind == "fallback"


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_give_median_clock_and_throttle_reasons():
    cs = bench.ClockSampler(0)
    cs.proc = _Done()
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1300.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] == 3


def test_clock_sampler_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
