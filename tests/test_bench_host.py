"""Host-side pieces of bench.py that need no GPU: the recorded DRAM traffic of
the FP32 formal-solution kernel is used only while the kernel's sources match
the hash recorded with it, and the refinement-precision names."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402


def test_committed_profile_is_used_only_for_its_sources():
    # the committed summary records a hash and a positive byte count; the
    # bench takes the count only while the kernel sources still hash the same
    vals = {}
    with open(os.path.join(os.path.dirname(HERE), bench.FS_PROFILE)) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    assert len(vals["source_sha256"]) == 64
    assert float(vals["dram_bytes_per_launch"]) > 1e6
    t = bench.recorded_traffic()
    if vals["source_sha256"] == bench.fs_source_hash():
        assert t == float(vals["dram_bytes_per_launch"])
    else:
        assert t is None


def test_traffic_is_dropped_when_the_sources_changed(tmp_path, monkeypatch):
    prof = tmp_path / "profile.md"
    prof.write_text("source_sha256: " + "0" * 64 + "\ndram_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "FS_PROFILE", str(prof))
    assert bench.recorded_traffic() is None
    prof.write_text("source_sha256: " + bench.fs_source_hash() + "\ndram_bytes_per_launch: 123\n")
    assert bench.recorded_traffic() == 123.0


def test_precision_names():
    from paper_2102_01734_gb300 import rt3d

    assert bench.precision_of("ff") == rt3d.FP32_FS_FF_REFINE
    assert bench.precision_of("mixed") == rt3d.FP32_FS_FP64_ALI
    assert bench.precision_of("fp64") == rt3d.FP64
