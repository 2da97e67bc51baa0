"""The benchmark's JSON line: `bench.py` with its default workload prints exactly one line with the
keys, types and units the measurement contract fixes, and its numbers hang together (whole-step
throughput from the same rays and time, the roofline fraction from its own achieved and peak, the
end-to-end figure counted from the bytes it copies, the oracle baseline on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def line():
    out = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3"], cwd=ROOT,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_contract_keys_and_types(line):
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict), ("e2e", dict), ("gpu_launches", int),
                 ("clocks", dict), ("roofline", dict), ("cpu_baseline", dict)):
        assert isinstance(line[k], t), k
    assert "vs_baseline" in line
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3
    assert line["unit"] == "Mrays/s" and line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["data"] == "synthetic" and "workload" in line["config"]
    assert line["gpu_launches"] > 0


def test_numbers_hang_together(line):
    wf, mk = line["wavefront"], line["megakernel"]
    assert wf["ms_per_frame"] > 0 and mk["ms_per_frame"] > 0
    assert abs(line["wf_over_mk_speedup"] - mk["ms_per_frame"] / wf["ms_per_frame"]) < 1e-6
    # the step is one wavefront frame, one megakernel frame and one adjoint pass
    parts = wf["ms_per_frame"] + mk["ms_per_frame"] + line["adjoint"]["ms_per_pass"]
    assert abs(line["ms_per_step"] - parts) <= 1e-3 * parts
    rays = wf["rays_per_frame"] + 2 * mk["rays_per_frame"]
    assert abs(line["value"] - rays / (line["ms_per_step"] * 1e-3) / 1e6) <= 1e-3 * line["value"]
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert 0.0 < r["frac"] < 1.0
    shares = r["share_of_step_kernel_time"]
    assert abs(sum(shares.values()) - 1.0) < 1e-3 and shares["extend"] > 0.1
    e = line["e2e"]
    assert e["unit"] == line["unit"] and 0 < e["value"] <= line["value"] * 1.05
    cam_px = line["config"]["resolution"][0] * line["config"]["resolution"][1]
    assert e["h2d_bytes_per_step"] == cam_px * 12                 # the gradient image
    assert e["d2h_bytes_per_step"] >= 2 * cam_px * 12             # both images (+ the gradients)
    f = line["wavefront_frame_roofline"]
    assert f["unit"] == "GB/s" and 0.0 < f["frac"] < 1.0 and abs(f["frac"] - f["achieved"] / f["peak"]) < 1e-9
    assert f["bytes_per_ray"] > 40 and f["mrays_s_bound"] > wf["mrays_s"]
    px = line["config"]["resolution"][0] * line["config"]["resolution"][1] * line["config"]["spp"]
    assert abs(wf["mpaths_s"] - px / (wf["ms_per_frame"] * 1e-3) / 1e6) <= 1e-6 * wf["mpaths_s"]
    c = line["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["unit"] == line["unit"]
    assert line["clocks"]["sm_mhz"] > 0


def test_ceilings_and_extra_workloads(line):
    """The traversal ceilings (device-counted node and triangle fetches against the L1 data path, for
    extend and the megakernel), the device counters' agreement between the two integrators, and the
    batched and inverse-rendering summaries the default run carries."""
    r = line["roofline"]
    t = r["traversal_per_ray"]
    assert t["megakernel_counts_equal_wavefront"] is True
    assert t["extension_ray"]["nodes"] >= 1 and t["shadow_ray"]["nodes"] >= 1
    for k in ("extend", "megakernel"):
        f = r["ceilings"][k]["traversal_fetch"]
        assert f["unit"] == "GB/s" and 0.0 < f["frac"] < 2.0 and abs(f["frac"] - f["achieved"] / f["peak"]) < 1e-9
    d = line["inverse_rendering"]
    assert d["paths"] == 512 * 512 * 64 and d["forward_ms"] > 0 and d["backward_ms"] > 0
    assert abs(d["bwd_over_fwd"] - d["backward_ms"] / d["forward_ms"]) < 1e-9 and d["bwd_over_fwd"] <= 3.0
    b = line["batch"]
    assert b["paths"] > 0 and b["batched_ms"] > 0 and b["separate_ms"] > 0
    assert abs(b["batched_over_separate"] - b["separate_ms"] / b["batched_ms"]) < 1e-9
    assert b["small_renders"]["scenes"] > 0 and b["ratio_bound_if_small_renders_were_free"] > 1.0
