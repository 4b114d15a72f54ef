"""Host logic of bench.py (no GPU): which kernel a configuration reports,
the DRAM traffic taken from a committed ncu summary only while the kernel's
sources are the ones it was captured on, the peak's source, and the sysfs CPU
list parser used to place the pinned host buffers."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402


def test_kernel_routing():
    assert bench.uses_paired_kernel(4, 14) and bench.uses_paired_kernel(4, 16)
    assert not bench.uses_paired_kernel(4, 13) and not bench.uses_paired_kernel(4, 17)
    assert not bench.uses_paired_kernel(2, 16)
    assert bench.kernel_name(4, 16).startswith("paired-region")
    assert bench.kernel_name(2, 16).startswith("fused")
    assert bench.kernel_name(4, 18).startswith("multi-pass")


def test_source_sha_follows_the_sources():
    # paired and fused configurations hash different files
    assert bench.kernel_source_sha(4, 16) != bench.kernel_source_sha(2, 16)
    assert bench.kernel_source_sha(4, 14) == bench.kernel_source_sha(4, 16)
    assert len(bench.kernel_source_sha(4, 16)) == 16


def _recorded_lines():
    out = []
    for name in sorted(os.listdir(os.path.join(bench.ROOT, "profiles"))):
        if name.endswith(".md"):
            for line in open(os.path.join(bench.ROOT, "profiles", name)):
                if line.startswith("bench-traffic:"):
                    out.append(dict(kv.split("=") for kv in line.split()[1:]))
    return out


def test_recorded_traffic_scales_by_batch():
    recs = [r for r in _recorded_lines() if r["source_sha"] == bench.kernel_source_sha(int(r["variant"]),
                                                                                          int(r["log2n"]))]
    if not recs:
        pytest.skip("no summary matches the current kernel sources")
    r = recs[0]
    v, ln, b, per = int(r["variant"]), int(r["log2n"]), int(r["batch"]), int(r["bytes_per_launch"])
    assert bench.recorded_traffic(v, ln, b) == per
    assert bench.recorded_traffic(v, ln, 8 * b) == 8 * per
    # the DRAM bytes of a launch are of the order of its algorithmic bytes
    algo = bench.BYTES_PER_POINT * b * (1 << ln)
    assert 0.5 * algo < per < 2.0 * algo


def test_recorded_traffic_is_none_once_the_kernel_changed(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_sha", lambda variant=4, log2n=16: "0" * 16)
    assert bench.recorded_traffic(4, 16, 4096) is None
    assert bench.recorded_traffic(4, 15, 4096) is None


def test_measured_peak_source(monkeypatch, tmp_path):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (1234.5, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "absent"))
    assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, "fallback")


@pytest.mark.parametrize("text,want", [
    ("0-3,8,10-11\n", {0, 1, 2, 3, 8, 10, 11}),
    ("5", {5}),
    ("", set()),
    ("0-71,144-215", set(range(72)) | set(range(144, 216))),
])
def test_cpulist(text, want):
    assert bench._cpulist(text) == want
