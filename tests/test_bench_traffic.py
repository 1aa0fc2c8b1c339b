"""bench.py reports the profiled counters of the bench kernel (warp
instructions and DRAM bytes per segment) only while the kernel sources are the
ones the counters were taken from: the committed summary carries a hash of the
forward kernel's sources, and any change to them turns the figures into null."""
import json
import os
import shutil

import bench


def _fake_root(tmp_path):
    root = tmp_path / "repo"
    for n in bench.FORWARD_SOURCES:
        os.makedirs(os.path.dirname(root / n), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, n), root / n)
    (root / "profiles").mkdir()
    return root


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.kernel_source_sha()
    (root / "profiles" / "trace_f32k_uniform512.json").write_text(
        json.dumps({"kernel_source_sha": sha, "warp_inst_per_segment": 2.5, "dram_bytes_per_segment": 0.5}))
    assert bench.profiled_traffic(1000) == 500.0
    assert bench.kernel_profile()["warp_inst_per_segment"] == 2.5
    # any edit of the kernel's sources invalidates the profiled figures
    f = root / "paper_2605_09882_gb300" / "csrc" / "rt_device.cuh"
    f.write_text(f.read_text() + "\n")
    assert bench.kernel_source_sha() != sha
    assert bench.profiled_traffic(1000) is None and bench.kernel_profile() is None


def test_missing_profile_gives_null_traffic(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic(1000) is None
