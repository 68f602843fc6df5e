"""Host logic of bench.py that needs no GPU: the lookup of the step kernel's
measured DRAM traffic, which must describe the kernel the run times."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_match_the_current_sources():
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    entries = {k: v for k, v in d.items() if not k.startswith("_")}
    assert entries
    for key, e in entries.items():
        workload, collision, storage = key.split(":")
        assert workload in bench.WORKLOADS and storage in ("f16", "bf16", "f32")
        # reads cover at least the algorithmic bytes: 9 populations in, 2 or 4 B each
        assert e["read_bytes_per_node"] >= 9 * {"f32": 4, "f16": 2, "bf16": 2}[storage]
        assert e["dram_bytes_per_node"] == pytest.approx(
            e["read_bytes_per_node"] + e["write_bytes_per_node"], abs=2e-3)
        if e["source_hash"] == bench.kernel_source_hash():
            assert bench.traffic_per_node(key, e["kind"]) == e["dram_bytes_per_node"]


def test_traffic_is_null_for_another_shape_or_rule(tmp_path, monkeypatch):
    import bench
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "step_kernel_traffic.json").write_text(json.dumps({
        "ensemble64:minxent4:f16": {"kind": "smem_deep", "dram_bytes_per_node": 34.0,
                                    "read_bytes_per_node": 18.0, "write_bytes_per_node": 16.0,
                                    "source_hash": h},
        "ensemble64:srt:f16": {"kind": "smem_deep", "dram_bytes_per_node": 34.0,
                               "read_bytes_per_node": 18.0, "write_bytes_per_node": 16.0,
                               "source_hash": "0" * 16}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.traffic_per_node("ensemble64:minxent4:f16", "smem_deep") == 34.0
    assert bench.traffic_per_node("ensemble64:minxent4:f16", "smem_wide") is None
    assert bench.traffic_per_node("ensemble64:minxent2:f16", "smem_deep") is None
    assert bench.traffic_per_node("ensemble64:minxent4:f32", "smem_deep") is None
    assert bench.traffic_per_node("ensemble64:srt:f16", "smem_deep") is None  # stale sources
