"""bench.py reports the profiled DRAM traffic of the bench kernel only while
the kernel sources are the ones the counters were taken from: the committed
summary carries a hash of the sources, and any change to them turns the
traffic into null."""
import json
import os
import shutil

import bench


def _fake_root(tmp_path):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2605_09882_gb300", "csrc"),
                    root / "paper_2605_09882_gb300" / "csrc")
    (root / "profiles").mkdir()
    return root


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.kernel_source_sha()
    (root / "profiles" / "trace_f32k_uniform512.json").write_text(
        json.dumps({"kernel_source_sha": sha, "dram_bytes_per_full_launch": 123.0}))
    assert bench.profiled_traffic() == 123.0
    # any edit of the kernel sources invalidates the profiled traffic
    f = root / "paper_2605_09882_gb300" / "csrc" / "rt_device.cuh"
    f.write_text(f.read_text() + "\n")
    assert bench.kernel_source_sha() != sha
    assert bench.profiled_traffic() is None


def test_missing_profile_gives_null_traffic(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic() is None
