"""Host logic of bench.py (CPU): traffic figures are only reported for an ncu
capture of the current kernel source and the same launch shape."""
import json

import bench


def _write(tmp_path, entries):
    p = tmp_path / "ncu_traffic.json"
    p.write_text(json.dumps(entries))
    return str(p)


def test_profiled_traffic_matches_source_and_launch_shape(tmp_path, monkeypatch):
    h = bench.kernel_source_hash("ens_stage")
    path = _write(tmp_path, {
        "ens_stage_fp32": {"source_hash": h, "threads_per_node": 1, "dram_per_algorithmic_byte": 1.02},
        "ns_stage_fp32_hex25": {"source_hash": "0" * 16, "threads_per_node": 1, "dram_bytes_per_launch": 5},
        "persistent_fp32_hex100": {"source_hash": bench.kernel_source_hash("persistent"), "persistent_lanes": 1,
                                   "persistent_ctas": 152, "dram_bytes_per_launch": 7},
    })
    monkeypatch.setattr(bench, "TRAFFIC_JSON", path)
    assert bench.profiled_traffic("ens_stage_fp32", algorithmic=1000.0, threads_per_node=1) == 1020.0
    assert bench.profiled_traffic("ens_stage_fp32", algorithmic=1000.0, threads_per_node=2) is None
    assert bench.profiled_traffic("ns_stage_fp32_hex25", threads_per_node=1) is None      # stale source
    assert bench.profiled_traffic("persistent_fp32_hex100", persistent_lanes=1, persistent_ctas=152) == 7
    assert bench.profiled_traffic("persistent_fp32_hex100", persistent_lanes=2, persistent_ctas=152) is None
    assert bench.profiled_traffic("missing_key") is None


def test_committed_traffic_entries_name_their_captures():
    """Every committed traffic figure points at an ncu summary under
    profiles/ and records the launch shape it was taken with."""
    import os
    with open(bench.TRAFFIC_JSON) as f:
        d = json.load(f)
    assert d
    for key, e in d.items():
        assert len(e["source_hash"]) == 16, key
        assert ("dram_bytes_per_launch" in e) != ("dram_per_algorithmic_byte" in e), key
        capture = e["capture"].split()[0]
        assert capture.startswith("profiles/") and os.path.exists(os.path.join(bench.ROOT, capture)), key
        assert "threads_per_node" in e or "persistent_lanes" in e, key
