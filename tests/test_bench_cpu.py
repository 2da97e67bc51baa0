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



def test_traversal_ceilings_arithmetic():
    """The traversal kernels' ceilings: fetched node/triangle records against the L1 data path, and
    (with committed ncu counts) warp instructions against the issue rate and L2 bytes against the L2
    peak; achieved = work per unit x units per launch / live launch time."""
    prof = {"inst_per_unit": 100.0, "l2_bytes_per_unit": 500.0, "l2_peak_gbs": 20000.0,
            "utilisation": {"l1tex_throughput": 0.5}}
    c = bench.traversal_ceilings(1e6, 0.5, nodes_per_unit=40.0, tris_per_unit=10.0, sms=152, sm_mhz=2000.0,
                                 prof=prof)
    clk_s = 2000e6
    f = c["traversal_fetch"]
    assert f["bytes_per_unit"] == 40 * 64 + 10 * 48
    assert abs(f["achieved"] - (40 * 64 + 10 * 48) * 1e6 / 0.5e-3 / 1e9) < 1e-9
    assert abs(f["peak"] - 152 * 128 * clk_s / 1e9) < 1e-9 and abs(f["frac"] - f["achieved"] / f["peak"]) < 1e-12
    i = c["issue"]
    assert abs(i["peak"] - 152 * 4 * clk_s / 1e9) < 1e-9
    assert abs(i["achieved"] - 100.0 * 1e6 / 0.5e-3 / 1e9) < 1e-9
    assert abs(c["l2"]["frac"] - 500.0 * 1e6 / 0.5e-3 / 1e9 / 20000.0) < 1e-12
    assert c["ncu_utilisation"] == {"l1tex_throughput": 0.5}
    # without committed counts only the device-counted fetch ceiling remains
    assert set(bench.traversal_ceilings(1e6, 0.5, 40.0, 10.0, 152, 2000.0, None)) == {"traversal_fetch"}
