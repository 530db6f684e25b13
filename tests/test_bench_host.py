"""Host-side logic of the benchmark on CPU: the clock-record summary (median
SM clock, throttle reasons), the DRAM-traffic lookup in the committed ncu
summaries (taken only on matching kernel sources), the optional report parts
and the mixed workload switch."""
import os
import sys
from pathlib import Path

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_median_and_reasons(work_dir):
    p = Path(work_dir) / "clocks.csv"
    p.write_text("0, 2070, 2070, 400.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 610.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2040, 2070, 590.2, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n")
    c = bench.ClockSampler(0)
    c.path = str(p)
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert s["power_w_max"] == 610.0
    assert not p.exists()


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.path = None
    assert c.summary()["reasons"] == ["unavailable"]


def test_profile_traffic_needs_matching_sources(work_dir, monkeypatch):
    tmp_path = Path(work_dir)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2302_11825_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_FILES["wost_walk"]:
        (csrc / f).write_text("// " + f)
    h = bench.kernel_source_hash("wost_walk")
    prof = tmp_path / "profiles" / "wost_walk_demo.md"
    prof.write_text(f"# demo\n\n- kernel_source_hash: {h}\n- dram_bytes_per_launch_full_size: 12345\n")
    assert bench.profile_traffic("wost_walk", "demo") == 12345.0
    assert bench.profile_traffic("wost_walk", "other") is None
    (csrc / "bvc_wost.cu").write_text("// changed")
    assert bench.profile_traffic("wost_walk", "demo") is None


def test_committed_profiles_name_their_sources():
    # every kernel summary states the hash of the sources it was taken on
    for f in os.listdir(os.path.join(ROOT, "profiles")):
        if f.startswith(tuple(bench.KERNEL_FILES)):
            text = open(os.path.join(ROOT, "profiles", f)).read()
            assert "kernel_source_hash" in text and "ncu " in text, f


def test_optional_part_records_failures():
    assert bench.optional_part(lambda: {"a": 1}) == {"a": 1}

    def boom():
        raise ValueError("no GPU")

    assert bench.optional_part(boom) == {"error": "ValueError: no GPU"}


@pytest.mark.parametrize("name, expect", [("mixed", "star_mixed_20kseg"), ("mixed3d", "tunnel_mixed_3d")])
def test_mixed_workload_switch(name, expect):
    w = bench.mixed_workload(name, samples=1024)
    assert w.name == expect and w.n_samples == 1024
    gap = w.meta.get("silhouette_gap", 0.0)
    assert (gap > 0.0) == (name == "mixed3d")


def test_device_info_never_breaks_the_line():
    # on a GPU: name, SM count, compute capability; without one: an error entry
    d = bench.optional_part(lambda: bench.device_info(0))
    assert isinstance(d, dict) and ("name" in d or "error" in d)
