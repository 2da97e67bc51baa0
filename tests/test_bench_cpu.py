"""Host-side arithmetic of bench.py: the wavefront frame's algorithmic bytes from its device counts,
and the committed ncu figures used only when they were taken on the current kernel sources (a
changed kernel reports traffic null until it is profiled again)."""
import json

import bench


def test_wavefront_frame_bytes_counts_every_stage():
    st = {"active": [100, 60, 30], "shadow_rays": 120}
    n_paths, n_pixels = 100, 50
    b = bench.BYTES_PER_UNIT
    expect = (190 * (b["extend"] + b["shade"]) + 120 * b["shadow"] + n_paths * (b["raygen"] + b["reduce"])
              + n_pixels * 12)
    assert bench.wavefront_frame_bytes(st, n_paths, n_pixels) == expect
    # per ray of the frame: (extend + shade) bytes per extension ray, shadow bytes per shadow ray
    assert b["extend"] == 40 and b["shadow"] == 80 and b["shade"] == 184


def test_traffic_only_for_the_current_kernel_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    entry = {"kernel_hash": bench.kernel_hash(), "dram_bytes_per_unit": 60.0, "counters": {"issue_active": 0.7}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"extend": entry}))
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "kernel_hash", lambda: entry["kernel_hash"])
    assert bench.load_traffic("extend")["dram_bytes_per_unit"] == 60.0
    assert bench.load_traffic("shadow") is None
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.load_traffic("extend") is None

