"""Benchmark: Mrays/s and ms/frame of the wavefront and megakernel estimators at 1080p, 1 spp, and
the backward/forward time ratio, on the ~1.15M-triangle procedural spheres scene (seeded, synthetic;
it stands in for the paper's glTF benchmark scene, which is not available).

One step = one wavefront frame + one megakernel frame + one path-replay adjoint pass of that frame
(all rows of the hot path), seed = step index.  Inputs are resident in device memory; L2 is flushed
(256 MiB write) between steps outside the timed events.  Rays = extension + shadow rays counted on
the device.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batch      # 64 scenes in one persistent launch vs 64 renders
  python bench.py --workload large      # ~10M-triangle scene, 3840x2160, 4 spp, depth 8
  python bench.py --workload diff       # inverse rendering, 512x512, 64 spp, 256 materials
  python bench.py --workload instanced  # the 1080p scene as a two-level (instanced) scene vs flat
  python bench.py --workload single [--separate-shadow] [--two-level] [--sort M] [--short-stack]
                                        # one untimed frame of each integrator (what ncu captures)
Under torchrun (N > 1) each rank renders its own frames (seed offset by rank, no collective on the
data path: weak scaling); the barrier and max-over-ranks timing are the only communication.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s and ms/frame (1080p, 1 spp) wavefront vs megakernel; bwd/fwd time ratio"
WORKLOAD = ("procedural spheres scene: 200 level-4 icospheres + 256x256-quad ground (1,155,088 tris), "
            "8 emissive quads + constant environment, 1920x1080, 1 spp, max depth 5, roulette from bounce 3; "
            "step = wavefront frame + megakernel frame + adjoint pass")
KERNEL_SOURCES = ["paper_2605_27323_gb300/csrc/pt_k_wave.cu", "paper_2605_27323_gb300/csrc/pt_common.cuh",
                  "paper_2605_27323_gb300/csrc/pt_device.cuh", "paper_2605_27323_gb300/csrc/pt_trace.cuh",
                  "paper_2605_27323_gb300/csrc/pt_k_mega.cu"]
# Unit ceilings of the traversal kernels (per SM per cycle): 4 warp schedulers issue one warp
# instruction each; the L1 data path moves 128 bytes.  A BVH node record is 64 bytes, a triangle
# record 48 bytes.
ISSUE_PER_SM_CLK = 4
L1_BYTES_PER_SM_CLK = 128
NODE_BYTES, TRI_BYTES = 64, 48
# Algorithmic bytes per unit of each stage: the queue and path-state records it must read and write.
BYTES_PER_UNIT = {
    "extend": 40,      # per extension ray: ray o|id + d|flags (32 B) read, hit record (8 B) written
    "shadow": 80,      # per shadow ray: o|tmax + d|id (32 B) + contribution (16 B) read, L rw (32 B)
    "shade": 184,      # per active path: ray+tp (48) + hit (8) + L rw (32) + next ray (48) + shadow (48)
    "megakernel": 12,  # per path: radiance written (scene reads amortise to ~0 per path)
    "raygen": 64,      # per path: ray + throughput (48 B) and radiance (16 B) written
    "reduce": 16,      # per path: radiance read (the image, 12 B per pixel, is added per pixel)
}
ADJ_SHADOW_BYTES = 40  # per shadow walk of the adjoint replay: ray (32 B) read, record flag (8 B) rw


def wavefront_frame_bytes(st: dict, n_paths: int, n_pixels: int) -> float:
    """Algorithmic bytes of one wavefront frame from its device counts: every stage's per-unit
    bytes times the units it processed (extension rays = paths entering each bounce)."""
    ext = float(sum(st["active"]))
    return (ext * (BYTES_PER_UNIT["extend"] + BYTES_PER_UNIT["shade"]) + st["shadow_rays"] * BYTES_PER_UNIT["shadow"]
            + n_paths * (BYTES_PER_UNIT["raygen"] + BYTES_PER_UNIT["reduce"]) + n_pixels * 12)


def traversal_ceilings(units_per_launch: float, avg_launch_ms: float, nodes_per_unit: float, tris_per_unit: float,
                       sms: int, sm_mhz: float, prof) -> dict:
    """Fractions of the traversal kernels' real ceilings for one kernel.  traversal_fetch: the node
    and triangle records its walks fetch (device-counted nodes and triangles per unit x 64 / 48 bytes)
    against the L1 data path.  From the committed ncu counts of the same kernel sources (`prof`, or
    None): issue -- its warp instructions against the issue rate of every scheduler; l2 -- its L2
    bytes against the L2 peak; ncu_utilisation -- the L1 and issue utilisation ncu measured for the
    frame's launches (L1 is limited by the number of divergent requests, not by bytes).  Achieved =
    per-unit work x units per launch / the launch's live duration."""
    t = avg_launch_ms * 1e-3
    clk = sm_mhz * 1e6
    l1_peak = sms * L1_BYTES_PER_SM_CLK * clk / 1e9
    fetch_per_unit = NODE_BYTES * nodes_per_unit + TRI_BYTES * tris_per_unit
    fetch = fetch_per_unit * units_per_launch / t / 1e9
    out = {"traversal_fetch": {"bytes_per_unit": fetch_per_unit, "nodes_per_unit": nodes_per_unit,
                               "tris_per_unit": tris_per_unit, "achieved": fetch, "peak": l1_peak, "unit": "GB/s",
                               "frac": fetch / l1_peak, "peak_basis": f"{L1_BYTES_PER_SM_CLK} B/clk/SM x {sms} SMs x "
                                                                      f"{sm_mhz:.0f} MHz"}}
    if prof:
        issue_peak = sms * ISSUE_PER_SM_CLK * clk / 1e9
        inst = prof["inst_per_unit"] * units_per_launch / t / 1e9
        out["issue"] = {"inst_per_unit": prof["inst_per_unit"], "achieved": inst, "peak": issue_peak,
                        "unit": "G warp-inst/s", "frac": inst / issue_peak,
                        "peak_basis": f"{ISSUE_PER_SM_CLK} warp-inst/clk/SM x {sms} SMs x {sm_mhz:.0f} MHz"}
        l2 = prof["l2_bytes_per_unit"] * units_per_launch / t / 1e9
        out["l2"] = {"bytes_per_unit": prof["l2_bytes_per_unit"], "achieved": l2, "peak": prof["l2_peak_gbs"],
                     "unit": "GB/s", "frac": l2 / prof["l2_peak_gbs"], "peak_basis": "ncu lts__t_bytes peak_sustained"}
        if "utilisation" in prof:
            out["ncu_utilisation"] = prof["utilisation"]
    return out


def rank_seed(step: int, rank: int) -> int:
    """Seed of a step on a rank: every rank renders its own frames (weak scaling, no data exchange)."""
    return step + rank * 1_000_000


def reduce_over_ranks(total_ms: float, total_rays: float, device) -> tuple:
    """Job time = the slowest rank's, job rays = the sum over ranks (the only communication)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor([total_rays], device=device, dtype=torch.float64)
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return float(t.item()), float(r.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic(kernel: str):
    """The committed ncu figures of `kernel` (per-unit DRAM bytes and a few unit utilisations), if
    they were taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(kernel)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, max clock, throttle reasons)."""

    def __init__(self, index: int):
        self.p = None
        self.path = os.path.join(os.environ.get("PT_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx = max(mx, float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def build_workload():
    from paper_2605_27323_gb300 import scenes
    return scenes.spheres_scene(seed=0)


def cpu_baseline(sc, budget_s=12.0, threads=None):
    """The FP64 oracle as it stands, on a bounded sample of the same frame (evenly strided pixels)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    osc = oracle.Scene.from_dict(sc)
    cam = sc["camera"]
    n_pix = cam["width"] * cam["height"]
    probe = np.arange(0, n_pix, max(1, n_pix // 4000), dtype=np.uint32)
    t0 = time.perf_counter()
    _, rays = osc.render_pixels(cam, 1, sc["max_depth"], 0, probe, rr_start=3, n_threads=threads)
    dt = time.perf_counter() - t0
    n = int(min(n_pix, max(len(probe), len(probe) * budget_s / max(dt, 1e-3))))
    pix = np.linspace(0, n_pix - 1, n).astype(np.uint32)
    t0 = time.perf_counter()
    _, rays = osc.render_pixels(cam, 1, sc["max_depth"], 0, pix, rr_start=3, n_threads=threads)
    dt = time.perf_counter() - t0
    total = int(rays[0] + rays[1])
    # the same oracle on one core, on 1/64 of that sample
    pix1 = pix[::64]
    t0 = time.perf_counter()
    _, rays1 = osc.render_pixels(cam, 1, sc["max_depth"], 0, pix1, rr_start=3, n_threads=1)
    dt1 = time.perf_counter() - t0
    # and on the small box workload (128^2 pixels, 16 spp, depth 8), whole frame
    from paper_2605_27323_gb300 import scenes
    box = scenes.box_scene(seed=0, width=128, height=128)
    obox = oracle.Scene.from_dict(box)
    t0 = time.perf_counter()
    _, rays_b = obox.render_pixels(box["camera"], 16, 8, 0, np.arange(128 * 128, dtype=np.uint32), rr_start=3,
                                   n_threads=threads)
    dt_b = time.perf_counter() - t0
    return {"value": total / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} evenly strided pixels of the 1920x1080 frame, 1 spp, depth 5 ({total} rays, "
                      f"{dt:.1f} s, FP64, OpenMP)", "ms_per_frame_extrapolated": dt * 1e3 * n_pix / n,
            "single_core": {"value": float(rays1[0] + rays1[1]) / dt1 / 1e6, "unit": "Mrays/s",
                            "sample": f"{len(pix1)} of those pixels"},
            "box_128x128_16spp": {"value": float(rays_b[0] + rays_b[1]) / dt_b / 1e6, "unit": "Mrays/s",
                                  "ms_per_frame": dt_b * 1e3}}


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, same metric and config."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc = build_workload()
    import oracle
    osc = oracle.Scene.from_dict(sc)
    cam = sc["camera"]
    threads = os.cpu_count() or 1
    n_pix = cam["width"] * cam["height"]
    per_step = 20000
    rays_total, t_total = 0, 0.0
    for step in range(args.warmup + args.steps):
        pix = (np.arange(per_step, dtype=np.uint64) * 7919 + step * 104729) % n_pix
        t0 = time.perf_counter()
        _, rays = osc.render_pixels(cam, 1, sc["max_depth"], step, pix.astype(np.uint32), rr_start=3,
                                    n_threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            rays_total += int(rays[0] + rays[1])
            t_total += dt
    value = rays_total / t_total / 1e6
    line = {"metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{per_step} pixels per step"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} strided pixels of the 1080p frame per step, 1 spp, depth 5"},
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hybrid_sweep(g, cam, spp, depth, thresholds, reps, flush, base_kw):
    """Wavefront frames with the hybrid continuation kernel at each threshold (device-timed, L2
    flushed between frames): {threshold: mean ms per frame}."""
    import torch
    stream = torch.cuda.current_stream()
    res = {}
    for thr in thresholds:
        g.render(cam, spp, depth, 700, hybrid=thr, **base_kw)
        ms = []
        for k in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.render(cam, spp, depth, 800 + k, hybrid=thr, **base_kw)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            flush.fill_(k & 0xFF)
        res[int(thr)] = float(np.mean(ms))
    return res


def run_gpu(args):
    import torch

    import paper_2605_27323_gb300 as pt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc = build_workload()
    g = pt.Scene.from_dict(sc)
    cam, spp, depth = sc["camera"], sc["spp"], sc["max_depth"]
    W, H = cam["width"], cam["height"]
    n_paths = W * H * spp
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(123)
    grad = torch.from_numpy(rng.uniform(-1, 1, size=(H, W, 3)).astype(np.float32)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ss = dict(short_stack=True) if args.short_stack else {}
    sep = dict(separate_shadow=True) if args.separate_shadow else {}
    wf_opts = dict(mode="wavefront", rr_start=3, sort=args.sort, profile=True, **ss, **sep)
    mk_opts = dict(mode="megakernel", rr_start=3, profile=True, **ss)
    mk_static_opts = dict(mode="megakernel", rr_start=3, mk_static=True)

    def step(seed, timing):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        g.render(cam, spp, depth, seed, **wf_opts)
        ev[1].record(stream)
        s_wf = g.stats() if timing else None
        ev_mk = torch.cuda.Event(enable_timing=True)
        ev_mk.record(stream)
        g.render(cam, spp, depth, seed, **mk_opts)
        ev[2].record(stream)
        s_mk = g.stats() if timing else None
        ev_bw = torch.cuda.Event(enable_timing=True)
        ev_bw.record(stream)
        g.backward(cam, spp, depth, seed, grad, rr_start=3, profile=True, **sep)
        ev[3].record(stream)
        s_bw = g.stats() if timing else None
        flush.fill_(seed & 0xFF)                     # L2 flush, outside the timed events
        return ev, ev_mk, ev_bw, s_wf, s_mk, s_bw

    for w in range(args.warmup):
        step(rank_seed(10_000 + w, rank), False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local) if rank == 0 else None
    torch.cuda.synchronize()
    recs = [step(rank_seed(s, rank), True) for s in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    wf_ms = [r[0][0].elapsed_time(r[0][1]) for r in recs]
    mk_ms = [r[1].elapsed_time(r[0][2]) for r in recs]
    bw_ms = [r[2].elapsed_time(r[0][3]) for r in recs]
    wf_rays = [r[3]["extension_rays"] + r[3]["shadow_rays"] for r in recs]
    mk_rays = [r[4]["extension_rays"] + r[4]["shadow_rays"] for r in recs]
    # the adjoint re-traces exactly the forward paths' rays
    step_ms = [a + b + c for a, b, c in zip(wf_ms, mk_ms, bw_ms)]
    total_ms = float(np.sum(step_ms))
    total_rays = float(np.sum(wf_rays) + np.sum(mk_rays) + np.sum(mk_rays))
    if world > 1:
        total_ms, total_rays = reduce_over_ranks(total_ms, total_rays, "cuda")
    value = total_rays / (total_ms * 1e-3) / 1e6

    # stage times from the library's events on the launch stream (timed region); the adjoint's
    # wavefront replay launches the same extend/shadow kernels (and a record-writing shade), so
    # its stages are added to the forward ones
    def tot(key, idx=(3, 5)):
        return sum(r[i][key] for r in recs for i in idx)
    stage = {"extend": tot("ms_extend"), "shade": tot("ms_shade"), "shadow": tot("ms_shadow"),
             "sort": tot("ms_sort"), "raygen": tot("ms_raygen"), "reduce": tot("ms_reduce"),
             "megakernel": sum(r[4]["ms_megakernel"] for r in recs),
             "adjoint_total": sum(r[5]["ms_adjoint"] for r in recs)}
    launches = {"extend": tot("launches_extend"), "shadow": tot("launches_shadow"),
                "megakernel": args.steps, "shade": tot("launches_extend")}
    units = {"extend": 2 * sum(r[3]["extension_rays"] for r in recs),
             "shadow": 2 * sum(r[3]["shadow_rays"] for r in recs),
             "shade": 2 * sum(r[3]["extension_rays"] for r in recs), "megakernel": n_paths * args.steps}
    # The roofline is reported for the wavefront's extend-stage launches (forward + adjoint replay):
    # k_extend at bounce 0 and k_trace after it, which in the default fused order also walks the
    # shadow rays of the previous bounce.  Their algorithmic bytes are the queue records they move:
    # 40 B per extension walk and 80 B per shadow walk; the unit is one walk.  The megakernel, whose
    # total time is similar, keeps each path's state in registers (12 B of radiance written per path),
    # so an HBM roofline does not bound it; every kernel's share of the step is listed beside the
    # roofline, and the traversal ceilings of both kernels next to it.
    dom = "extend"
    fused = launches["shadow"] == 0
    shd_fwd = sum(r[3]["shadow_rays"] for r in recs)
    shd_adj = sum(r[5]["shadow_rays"] for r in recs)
    walks = units["extend"] + ((shd_fwd + shd_adj) if fused else 0)
    # an adjoint shadow walk reads its ray (32 B) and sets the record's visibility flag (8 B)
    alg_bytes = (BYTES_PER_UNIT["extend"] * units["extend"]
                 + ((BYTES_PER_UNIT["shadow"] * shd_fwd + ADJ_SHADOW_BYTES * shd_adj) if fused else 0))
    kernel_ms = {k: stage[k] for k in ("extend", "shadow", "shade", "megakernel", "sort", "raygen", "reduce")}
    kernel_ms["adjoint_other"] = max(0.0, stage["adjoint_total"] - sum(r[5][k] for r in recs for k in
                                                                     ("ms_extend", "ms_shade", "ms_shadow",
                                                                      "ms_raygen", "ms_reduce")))
    shares = {k: v / max(1e-9, sum(kernel_ms.values())) for k, v in kernel_ms.items()}
    peak, peak_src = load_peaks()
    achieved = alg_bytes / (stage[dom] * 1e-3) / 1e9
    tr = load_traffic(dom)
    roofline = {"bound": "hbm", "kernel": "extend" + (" + previous bounce's shadow walks (fused)" if fused else ""),
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "traffic": (float(tr["dram_bytes_per_unit"]) * walks / launches[dom]) if tr else None,
                # what does bound it: ncu's unit utilisations for the same kernel sources
                "ncu_counters": tr.get("counters") if tr else None,
                "walks_per_launch": walks / launches[dom],
                "algorithmic_bytes_per_launch": alg_bytes / launches[dom],
                "avg_launch_ms": stage[dom] / launches[dom],
                "share_of_step_kernel_time": {k: round(v, 4) for k, v in shares.items()}}
    gpu_launches = sum(r[3]["launches_total"] + r[4]["launches_total"] + r[5]["launches_total"] for r in recs)

    wf_frame = float(np.mean(wf_ms))
    mk_frame = float(np.mean(mk_ms))
    wf_bytes = float(np.mean([wavefront_frame_bytes(r[3], n_paths, W * H) for r in recs]))
    wf_bpr = wf_bytes / float(np.mean(wf_rays))
    wf_roof = {"bound": "hbm", "algorithmic_bytes_per_frame": wf_bytes, "bytes_per_ray": wf_bpr,
               "achieved": wf_bytes / (wf_frame * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
               "frac": wf_bytes / (wf_frame * 1e-3) / 1e9 / peak,
               "mrays_s_bound": peak * 1e9 / wf_bpr / 1e6}
    # the paper's megakernel layout (one thread per path over all paths), timed apart from the step
    st_ms = []
    for s_ in range(max(3, args.steps // 2)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.render(cam, spp, depth, 500 + s_, **mk_static_opts)
        e1.record(stream)
        e1.synchronize()
        st_ms.append(e0.elapsed_time(e1))
        flush.fill_(s_ & 0xFF)
    # the hybrid of the paper's future work: the last sparse bounces finished in one kernel
    hyb = hybrid_sweep(g, cam, spp, depth, (1 << 16, 1 << 18, 1 << 20), max(3, args.steps // 2), flush,
                       dict(mode="wavefront", rr_start=3, sort=args.sort))
    hyb_thr = min(hyb, key=hyb.get)
    # estimator variants (not in the step): MIS, and the Halton (2,3) + Cranley-Patterson jitter
    variants = {}
    # (and the two integrators without the per-stage timing events the step records: those cost
    # the wavefront about 2 us per stage boundary)
    for name, kw in (("mis_wavefront", dict(mode="wavefront", mis=True)),
                     ("mis_megakernel", dict(mode="megakernel", mis=True)),
                     ("halton_wavefront", dict(mode="wavefront", sampler="halton")),
                     ("wavefront_no_stage_events", dict(mode="wavefront", sort=args.sort, **ss, **sep)),
                     ("megakernel_no_stage_events", dict(mode="megakernel", **ss))):
        g.render(cam, spp, depth, 900, rr_start=3, **kw)
        ms = []
        for k in range(max(3, args.steps // 2)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.render(cam, spp, depth, 910 + k, rr_start=3, **kw)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            flush.fill_(k & 0xFF)
        st_v = g.stats()
        variants[name] = {"ms_per_frame": float(np.mean(ms)),
                          "mrays_s": (st_v["extension_rays"] + st_v["shadow_rays"]) / (float(np.mean(ms)) * 1e-3) / 1e6}
    variants["wf_over_mk_no_stage_events"] = (variants["megakernel_no_stage_events"]["ms_per_frame"] /
                                              variants["wavefront_no_stage_events"]["ms_per_frame"])
    # the wavefront's advantage against the maximum depth (the paper expects it to grow with depth,
    # as compaction leaves ever fewer active paths per bounce); frames without stage events
    # (and the hybrid, which finishes the sparse late bounces in one kernel)
    depth_sweep = {}
    for dmax in (1, 2, 3, 5, 8, 12, 16):
        row = {}
        for name, kw in (("wavefront", dict(mode="wavefront")), ("megakernel", dict(mode="megakernel")),
                         ("hybrid", dict(mode="wavefront", hybrid=hyb_thr))):
            g.render(cam, spp, dmax, 950, rr_start=3, **kw)
            ms = []
            for k in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.render(cam, spp, dmax, 960 + k, rr_start=3, **kw)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                flush.fill_(k & 0xFF)
            row[name + "_ms"] = float(np.mean(ms))
        row["wf_over_mk"] = row["megakernel_ms"] / row["wavefront_ms"]
        row["hybrid_over_mk"] = row["megakernel_ms"] / row["hybrid_ms"]
        depth_sweep[str(dmax)] = row
    # traversal work per ray (device counters of the counting instantiations; outside the timed region):
    # the wavefront's extend walks per extension ray, the megakernel's walks per path
    g.render(cam, spp, depth, 0, mode="wavefront", rr_start=3, count_traversal=True)
    cw = g.stats()
    g.render(cam, spp, depth, 0, mode="megakernel", rr_start=3, count_traversal=True)
    cm = g.stats()
    trav = {"extension_ray": {"nodes": cw["nodes_closest"] / cw["extension_rays"],
                              "tris": cw["tris_closest"] / cw["extension_rays"]},
            "shadow_ray": {"nodes": cw["nodes_any"] / max(1, cw["shadow_rays"]),
                           "tris": cw["tris_any"] / max(1, cw["shadow_rays"])},
            "megakernel_counts_equal_wavefront": all(cw[k] == cm[k] for k in
                                                     ("nodes_closest", "tris_closest", "nodes_any", "tris_any"))}
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    walk_nodes = (cw["nodes_closest"] + (cw["nodes_any"] if fused else 0)) / (cw["extension_rays"] + (cw["shadow_rays"] if fused else 0))
    walk_tris = (cw["tris_closest"] + (cw["tris_any"] if fused else 0)) / (cw["extension_rays"] + (cw["shadow_rays"] if fused else 0))
    roofline["ceilings"] = {
        "extend": traversal_ceilings(walks / launches["extend"], stage["extend"] / launches["extend"],
                                     walk_nodes, walk_tris, sms, sm_mhz, tr),
        "megakernel": traversal_ceilings(n_paths, stage["megakernel"] / args.steps,
                                         (cm["nodes_closest"] + cm["nodes_any"]) / n_paths,
                                         (cm["tris_closest"] + cm["tris_any"]) / n_paths, sms, sm_mhz,
                                         load_traffic("megakernel"))}
    roofline["traversal_per_ray"] = trav
    # the batched (64 scenes) and inverse-rendering workloads, compact: the batched-over-separate
    # ratio and the backward/forward ratio are measured in every default run
    extra = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extra["inverse_rendering"] = measure_diff(3, 3)
        torch.cuda.empty_cache()
        extra["batch"] = measure_batch(3, 3)
        torch.cuda.empty_cache()
    out = None
    if rank == 0:
        e2e = None
        if world == 1:
            e2e = measure_e2e(g, cam, spp, depth, grad, args, wf_opts, mk_opts,
                              [rank_seed(k, rank) for k in range(args.steps)],
                              [a + 2 * b for a, b in zip(wf_rays, mk_rays)])
        line = {
            "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "resolution": [W, H], "spp": spp, "max_depth": depth,
                       "triangles": int(g.info()["n_tris"]), "sort": args.sort,
                       "traversal_stack": "shared-memory short stack" if args.short_stack else "local memory",
                       "stage_order": "separate" if args.separate_shadow or args.short_stack else "fused",
                       "l2": "flushed between steps (256 MiB write), outside the timed events"},
            "wavefront": {"mrays_s": float(np.sum(wf_rays)) / (np.sum(wf_ms) * 1e-3) / 1e6, "ms_per_frame": wf_frame,
                          "ms_per_frame_median": float(np.median(wf_ms)), "rays_per_frame": float(np.mean(wf_rays)),
                          "mpaths_s": n_paths / (wf_frame * 1e-3) / 1e6},
            "megakernel": {"mrays_s": float(np.sum(mk_rays)) / (np.sum(mk_ms) * 1e-3) / 1e6,
                           "ms_per_frame": mk_frame, "ms_per_frame_median": float(np.median(mk_ms)),
                           "rays_per_frame": float(np.mean(mk_rays)), "mpaths_s": n_paths / (mk_frame * 1e-3) / 1e6},
            # the whole wavefront frame against HBM: every stage's algorithmic bytes (queue and
            # state traffic) over the frame time; its bound in rays/s is peak / (bytes per ray)
            "wavefront_frame_roofline": wf_roof,
            "hybrid": {"ms_per_frame": hyb[hyb_thr], "threshold": hyb_thr, "sweep_ms": hyb,
                       "wavefront_over_hybrid": wf_frame / hyb[hyb_thr],
                       "note": "wavefront frame whose remaining bounces run in one persistent kernel once at "
                               "most `threshold` paths are active; same image; not in the step"},
            "estimator_variants": variants,
            "depth_sweep": depth_sweep,
            "megakernel_static": {"ms_per_frame": float(np.mean(st_ms)),
                                  "mrays_s": float(np.mean(mk_rays)) / (float(np.mean(st_ms)) * 1e-3) / 1e6,
                                  "note": "one thread per path over all paths (the paper's layout); not in the step"},
            "wf_over_mk_speedup": mk_frame / wf_frame,
            "bwd_over_fwd": float(np.mean(bw_ms)) / min(wf_frame, mk_frame),
            "adjoint": {"ms_per_pass": float(np.mean(bw_ms)), "replay": "wavefront stages + per-vertex records"},
            "stage_ms_per_step": {k: v / args.steps for k, v in stage.items()},
            "roofline": roofline,
            "gpu_launches": int(gpu_launches),
            "paper_context": "paper: wavefront 1.16x over megakernel (73.6 vs 64.7 FPS, RTX 3060 Ti, Vulkan RT cores)",
        }
        line.update(extra)
        if e2e:
            line["e2e"] = e2e
        if clk:
            line["clocks"] = clk
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(sc)
        out = line
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def measure_e2e(g, cam, spp, depth, grad, args, wf_opts, mk_opts, seeds, rays_per_step):
    """Same step through the public API with host buffers: the gradient image is copied in from
    pinned memory, both images and the gradients are read back, all inside the timed region.  The
    timed steps render the device-timed steps' seeds, whose ray counts (device-counted there; the
    same seed traces the same rays) give the rays, so nothing but the API calls runs in the timed
    region."""
    import torch
    W, H = cam["width"], cam["height"]
    h_wf = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
    h_mk = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
    h_grad = grad.cpu().pin_memory()
    h_ga = torch.empty((g.n_mats, 3), dtype=torch.float32).pin_memory()
    h_ge = torch.empty((g.n_mats,), dtype=torch.float32).pin_memory()
    wf = {k: v for k, v in wf_opts.items() if k != "profile"}
    mk = {k: v for k, v in mk_opts.items() if k != "profile"}
    stream = torch.cuda.current_stream()
    ms, rays = 0.0, 0.0
    n_timed = min(len(seeds), max(3, args.steps // 2))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k in range(args.warmup + n_timed):
        timed = k >= args.warmup
        seed = seeds[k - args.warmup] if timed else 20_000 + k
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(k & 0xFF)                        # L2 flush, outside the timed events
        torch.cuda.synchronize()
        e0.record(stream)
        g.render(cam, spp, depth, seed, out=h_wf, **wf)
        g.render(cam, spp, depth, seed, out=h_mk, **mk)
        d_grad = h_grad.to("cuda", non_blocking=True)
        ga, ge = g.backward(cam, spp, depth, seed, d_grad, rr_start=3,
                            **({"separate_shadow": True} if args.separate_shadow else {}))
        h_ga.copy_(ga, non_blocking=True)
        h_ge.copy_(ge, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if timed:
            ms += e0.elapsed_time(e1)
            rays += rays_per_step[k - args.warmup]
    return {"value": rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s",
            "h2d_bytes_per_step": int(h_grad.numel() * 4),
            "d2h_bytes_per_step": int(h_wf.numel() * 4 + h_mk.numel() * 4 + h_ga.numel() * 4 + h_ge.numel() * 4)}


def run_large(args):
    """~10M-triangle terrain scene, 3840x2160, 4 spp, depth 8 (33.2M paths; wavefront queues sized to
    all of them): wavefront and megakernel frames, device-timed."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import scenes
    t0 = time.perf_counter()
    sc = scenes.terrain_scene(seed=0)
    g = pt.Scene.from_dict(sc)
    setup_s = time.perf_counter() - t0
    cam, spp, depth = sc["camera"], sc["spp"], sc["max_depth"]
    stream = torch.cuda.current_stream()
    res = {}
    for mode in ("wavefront", "megakernel"):
        for k in range(args.warmup):
            g.render(cam, spp, depth, 100 + k, mode=mode)
        ms, rays = [], []
        for k in range(max(3, min(args.steps, 10))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.render(cam, spp, depth, k, mode=mode)
            e1.record(stream)
            st = g.stats()
            ms.append(e0.elapsed_time(e1))
            rays.append(st["extension_rays"] + st["shadow_rays"])
        res[mode] = {"ms_per_frame": float(np.mean(ms)), "mrays_s": float(np.sum(rays) / (np.sum(ms) * 1e-3) / 1e6),
                     "rays_per_frame": float(np.mean(rays))}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    hyb = hybrid_sweep(g, cam, spp, depth, (1 << 18, 1 << 20, 1 << 22), 3, flush, dict(mode="wavefront"))
    hyb_thr = min(hyb, key=hyb.get)
    res["hybrid"] = {"ms_per_frame": hyb[hyb_thr], "threshold": hyb_thr, "sweep_ms": hyb,
                     "wavefront_over_hybrid": res["wavefront"]["ms_per_frame"] / hyb[hyb_thr]}
    info = g.info()
    # the same recipe as a two-level scene: one icosphere mesh placed 5000 times (TLAS/BLAS), with the
    # heightfield as one mesh or as 8 x 8 tile meshes
    two_level = {}
    for tiles in (1, 8):
        t0 = time.perf_counter()
        isc = scenes.instanced_terrain_scene(seed=0, tiles=tiles)
        gi = pt.Scene.from_dict(isc)
        isetup = time.perf_counter() - t0
        ires = {}
        for mode in ("wavefront", "megakernel"):
            for k in range(args.warmup):
                gi.render(cam, spp, depth, 100 + k, mode=mode)
            ms, rays = [], []
            for k in range(max(3, min(args.steps, 10))):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gi.render(cam, spp, depth, k, mode=mode)
                e1.record(stream)
                st = gi.stats()
                ms.append(e0.elapsed_time(e1))
                rays.append(st["extension_rays"] + st["shadow_rays"])
            ires[mode] = {"ms_per_frame": float(np.mean(ms)),
                          "mrays_s": float(np.sum(rays) / (np.sum(ms) * 1e-3) / 1e6)}
        iinfo = gi.info()
        ires.update({"terrain_meshes": tiles * tiles, "instances": int(len(isc["inst_mesh"])),
                     "triangles_placed": int(iinfo["n_tris"]), "device_bytes": int(iinfo["device_bytes"]),
                     "device_bytes_saved_vs_flat": int(info["device_bytes"]) - int(iinfo["device_bytes"]),
                     "scene_setup_s": isetup})
        two_level[f"terrain_tiles_{tiles}x{tiles}"] = ires
        del gi
    line = {"metric": "Mrays/s and ms/frame, large scene (3840x2160, 4 spp, depth 8)", "value": res["wavefront"]["mrays_s"],
            "unit": "Mrays/s", "n_gpus": 1, "steps": max(3, min(args.steps, 10)), "warmup": args.warmup,
            "ms_per_step": res["wavefront"]["ms_per_frame"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "2048^2 fBm heightfield + 5000 level-2 icospheres, 64 emissive quads",
                       "triangles": int(info["n_tris"]), "bvh_nodes": int(info["n_nodes"]),
                       "device_bytes": int(info["device_bytes"]), "scene_setup_s": setup_s},
            "wavefront": res["wavefront"], "megakernel": res["megakernel"], "hybrid": res["hybrid"],
            "two_level": two_level,
            "wf_over_mk_speedup": res["megakernel"]["ms_per_frame"] / res["wavefront"]["ms_per_frame"]}
    print(json.dumps(line), flush=True)


def measure_diff(steps: int, warmup: int, adam_steps: bool = True) -> dict:
    """Inverse rendering on the 256-material spheres scene (512x512, 64 spp, depth 6, fixed roulette
    0.9): each step renders the image with the current albedos and emissions, takes the L2 loss
    against a target rendered with hidden parameters (another seed), back-propagates through the
    path-replay adjoint and applies an Adam update.  Returns forward and backward device times,
    their ratio, and the loss and parameter error along the way.  Each step renders at a fresh seed,
    so its loss includes both images' Monte Carlo noise, whose size depends on the parameters; the
    loss rendered with the target's own seed (`loss_same_seed`, 0 at the hidden parameters) and the
    albedo error measure progress without that noise."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import scenes
    t0 = time.perf_counter()
    sc = scenes.diff_scene(seed=0)
    g = pt.Scene.from_dict(sc)
    setup_s = time.perf_counter() - t0
    cam, spp, depth = sc["camera"], sc["spp"], sc["max_depth"]
    W, H = cam["width"], cam["height"]
    kw = dict(rr_start=sc["rr_start"], rr_fixed=sc["rr_fixed"])
    alb_t, em_t = (torch.from_numpy(x).cuda() for x in scenes.diff_target(sc, seed=7))
    g.set_materials(alb_t, em_t)
    target = g.render(cam, spp, depth, 999_999, **kw).clone()
    alb = torch.tensor(np.asarray(sc["mat_albedo"], np.float32), device="cuda").reshape(-1, 3).requires_grad_()
    em = torch.tensor(np.asarray(sc["mat_emission"], np.float32), device="cuda").requires_grad_()
    emissive = (em.detach() > 0).float()      # emission is fitted on the materials that emit
    opt = torch.optim.Adam([{"params": [alb], "lr": 0.02}, {"params": [em], "lr": 0.2}])
    stream = torch.cuda.current_stream()
    n_paths = W * H * spp

    def step(seed):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        opt.zero_grad(set_to_none=True)
        ev[0].record(stream)
        g.set_materials(alb, em)
        img = g.render(cam, spp, depth, seed, **kw)
        ev[1].record(stream)
        diff = img - target
        loss = (diff * diff).mean()
        grad_img = (2.0 / diff.numel()) * diff
        ev[2].record(stream)
        ga, ge = g.backward(cam, spp, depth, seed, grad_img, **kw)
        ev[3].record(stream)
        alb.grad, em.grad = ga, ge * emissive
        opt.step()
        with torch.no_grad():
            alb.clamp_(0.0, 1.0)
            em.clamp_(min=0.0)
        ev[4].record(stream)
        return ev, loss.detach()

    def loss_same_seed():
        # the loss with the target's own seed (common random numbers): 0 at the hidden parameters,
        # so unlike the per-step losses it carries no Monte Carlo noise term
        with torch.no_grad():
            g.set_materials(alb, em)
            return float(((g.render(cam, spp, depth, 999_999, **kw) - target) ** 2).mean())

    lam = torch.from_numpy(np.asarray(sc["mat_type"]) == scenes.LAMBERT).cuda()
    alb_err0 = float((alb.detach() - alb_t)[lam].abs().mean())
    loss_ss0 = loss_same_seed()
    for w in range(warmup):
        step(50_000 + w)
    torch.cuda.synchronize()
    recs = [step(s) for s in range(steps)]
    torch.cuda.synchronize()
    fwd = [r[0][0].elapsed_time(r[0][1]) for r in recs]
    bwd = [r[0][2].elapsed_time(r[0][3]) for r in recs]
    tot = [r[0][0].elapsed_time(r[0][4]) for r in recs]
    losses = [float(r[1]) for r in recs]
    g.render(cam, spp, depth, 0, **kw)
    st = g.stats()
    rays_fwd = st["extension_rays"] + st["shadow_rays"]
    alb_err = float((alb.detach() - alb_t)[lam].abs().mean())
    loss_ss1 = loss_same_seed()
    # the adjoint's one-thread-per-path replay (mode="megakernel") on the same gradient, for comparison
    grad_img = torch.ones_like(target) * (1.0 / target.numel())
    g.backward(cam, spp, depth, 1, grad_img, mode="megakernel", **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.backward(cam, spp, depth, 2, grad_img, mode="megakernel", **kw)
    e1.record(stream)
    e1.synchronize()
    bwd_mk = e0.elapsed_time(e1)
    return {"workload": "procedural spheres geometry, 256 shared materials, 512x512, 64 spp, depth 6, roulette "
                        "from bounce 3 with q = 0.9; L2 loss to a target from hidden parameters (seed 7); Adam on "
                        "every albedo and on the emissive material's emission",
            "paths": n_paths, "steps": steps, "warmup": warmup, "scene_setup_s": setup_s,
            "forward_ms": float(np.median(fwd)), "backward_ms": float(np.median(bwd)),
            "bwd_over_fwd": float(np.median(bwd) / np.median(fwd)), "step_ms": float(np.mean(tot)),
            "backward_one_thread_per_path_ms": bwd_mk,
            "forward_mrays_s": rays_fwd / (np.median(fwd) * 1e-3) / 1e6,
            "loss_first": losses[0], "loss_last": losses[-1],
            "loss_same_seed": {"start": loss_ss0, "end": loss_ss1, "steps": warmup + steps},
            "lambert_albedo_mean_abs_error": {"start": alb_err0, "end": alb_err, "steps": warmup + steps}}


def run_diff(args):
    d = measure_diff(args.steps, args.warmup)
    line = {"metric": "inverse-rendering step: backward/forward time ratio (512x512, 64 spp, depth 6, 256 materials)",
            "value": d["bwd_over_fwd"], "unit": "ratio", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": d["step_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": d["workload"], "paths": d["paths"],
                       "l2": "inputs (scene, queues, records) exceed L2; no flush"}}
    line.update({k: v for k, v in d.items() if k not in ("workload", "paths", "steps", "warmup")})
    print(json.dumps(line), flush=True)


def run_instanced(args):
    """The 1080p procedural scene as a two-level scene (one icosphere mesh placed by 200 randomly
    rotated, scaled instances; the ground and the light quads as meshes; 1,155,088 placed
    triangles, 1 spp, depth 5) against the same recipe flattened into one BVH: wavefront and
    megakernel frames, device-timed, L2 flushed between frames."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import scenes
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    for name, sc in (("two_level", scenes.instanced_spheres_scene(seed=0)),
                     ("flat", scenes.spheres_scene(seed=0))):
        g = pt.Scene.from_dict(sc)
        cam, spp, depth = sc["camera"], sc["spp"], sc["max_depth"]
        r = {}
        for mode in ("wavefront", "megakernel"):
            for k in range(args.warmup):
                g.render(cam, spp, depth, 100 + k, mode=mode)
            ms, rays = [], []
            for k in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.render(cam, spp, depth, k, mode=mode)
                e1.record(stream)
                st = g.stats()
                ms.append(e0.elapsed_time(e1))
                rays.append(st["extension_rays"] + st["shadow_rays"])
                flush.fill_(k & 0xFF)
            r[mode] = {"ms_per_frame": float(np.mean(ms)), "mrays_s": float(np.sum(rays) / (np.sum(ms) * 1e-3) / 1e6)}
        info = g.info()
        r["device_bytes"] = int(info["device_bytes"])
        r["triangles"] = int(info["n_tris"])
        res[name] = r
        del g
    line = {"metric": "Mrays/s and ms/frame, 1080p procedural scene as a two-level (instanced) scene",
            "value": res["two_level"]["wavefront"]["mrays_s"], "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["two_level"]["wavefront"]["ms_per_frame"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "200 rotated, scaled instances of one level-4 icosphere mesh + 256x256-quad ground "
                                   "mesh + 8 light-quad instances, 1920x1080, 1 spp, depth 5",
                       "l2": "flushed between frames (256 MiB write)"},
            "two_level": res["two_level"], "flat": res["flat"],
            "two_level_over_flat_time": res["two_level"]["wavefront"]["ms_per_frame"] / res["flat"]["wavefront"]["ms_per_frame"]}
    print(json.dumps(line), flush=True)


def measure_batch(steps: int, warmup: int) -> dict:
    """64 procedural scenes (lognormal triangle counts in [1k, 2M], resolutions from {256^2, 512^2,
    1280x720, 1920x1080}, spp from {1, 4, 16}, depth 5): one persistent batched wavefront (autotuned
    queue capacity, block size and sort granularity; CUDA-graph bounce loop) against 64 separate
    pt_render calls producing the same images.  Also the renders of <= 1M paths (those that leave the
    GPU underfilled on their own) as a batch of their own, and the ratio the whole mix could reach
    if batching made those renders free (the large renders fill the GPU either way)."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import scenes
    t0 = time.perf_counter()
    specs = scenes.batch_scenes(seed=0)
    gs = [pt.Scene.from_dict(sc) for sc in specs]
    setup_s = time.perf_counter() - t0
    cams = [sc["camera"] for sc in specs]
    spps = [int(sc["spp"]) for sc in specs]
    depth = 5
    outs = [torch.empty((c["height"], c["width"], 3), device="cuda") for c in cams]
    tris = [g.n_tris for g in gs]
    paths = sum(c["width"] * c["height"] * s for c, s in zip(cams, spps))
    # rays of one frame of every scene (the same estimator runs in both arms)
    rays = 0
    for g, c, s in zip(gs, cams, spps):
        g.render(c, s, depth, 0, mode="wavefront")
        st = g.stats()
        rays += st["extension_rays"] + st["shadow_rays"]
    t1 = time.perf_counter()
    best = pt.autotune_batch(gs, cams, spps, depth, 0, outs=outs)
    tune_s = time.perf_counter() - t1
    kw = dict(queue_capacity=best["queue_capacity"], block_size=best["block_size"], sort=int(best["sort"]))
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        ms = []
        for k in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    def batched(k):
        pt.render_batch(gs, cams, spps, depth, k, outs=outs, **kw)

    def separate(k):
        for i, (g, c, s) in enumerate(zip(gs, cams, spps)):
            g.render(c, s, depth, k, out=outs[i], mode="wavefront")

    for k in range(warmup):
        batched(100 + k)
        separate(100 + k)
    steps = max(3, min(steps, 10))
    b_ms = timed(batched, steps)
    s_ms = timed(separate, steps)
    small = [i for i, (c, s_) in enumerate(zip(cams, spps)) if c["width"] * c["height"] * s_ <= (1 << 20)]
    sg, sc_, ss, so = [gs[i] for i in small], [cams[i] for i in small], [spps[i] for i in small], [outs[i] for i in small]

    def separate_small(k):
        for i, (g, c, s_) in enumerate(zip(sg, sc_, ss)):
            g.render(c, s_, depth, k, out=so[i], mode="wavefront")

    small_res = None
    if small:
        best_s = pt.autotune_batch(sg, sc_, ss, depth, 0, outs=so)
        kw_s = dict(queue_capacity=best_s["queue_capacity"], block_size=best_s["block_size"], sort=int(best_s["sort"]))

        def batched_small(k):
            pt.render_batch(sg, sc_, ss, depth, k, outs=so, **kw_s)

        batched_small(0)
        separate_small(0)
        bs_ms, ss_ms = timed(batched_small, steps), timed(separate_small, steps)
        small_res = {"scenes": len(small), "paths": int(sum(c["width"] * c["height"] * s_ for c, s_ in zip(sc_, ss))),
                     "batched_ms": bs_ms, "separate_ms": ss_ms, "batched_over_separate": ss_ms / bs_ms,
                     "autotuned": kw_s}
    return {"workload": "64 procedural scenes, lognormal triangle counts in [1k, 2M], resolutions "
                        "{256^2, 512^2, 1280x720, 1920x1080}, spp {1, 4, 16}, depth 5",
            "triangles_total": int(sum(tris)), "triangles_min": int(min(tris)), "triangles_max": int(max(tris)),
            "paths": int(paths), "rays": int(rays), "steps": steps, "autotuned": kw, "autotune_s": tune_s,
            "scene_setup_s": setup_s, "batched_ms": b_ms, "batched_mrays_s": rays / (b_ms * 1e-3) / 1e6,
            "separate_ms": s_ms, "separate_mrays_s": rays / (s_ms * 1e-3) / 1e6, "batched_over_separate": s_ms / b_ms,
            "small_renders": small_res,
            # Amdahl: the large renders fill the GPU on their own, so removing every per-launch and tail
            # cost of the small renders (their whole separate time) bounds what batching can gain
            "ratio_bound_if_small_renders_were_free": (s_ms / (s_ms - small_res["separate_ms"])) if small_res else None}


def run_batch(args):
    b = measure_batch(args.steps, args.warmup)
    line = {"metric": "batched wavefront vs 64 per-scene renders (Mrays/s)", "value": b["batched_mrays_s"],
            "unit": "Mrays/s", "n_gpus": 1, "steps": b["steps"], "warmup": args.warmup, "ms_per_step": b["batched_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {k: b[k] for k in ("workload", "triangles_total", "triangles_min", "triangles_max", "paths",
                                         "rays", "autotuned", "autotune_s", "scene_setup_s")}}
    line.update({k: b[k] for k in ("separate_ms", "separate_mrays_s", "batched_over_separate", "small_renders",
                                   "ratio_bound_if_small_renders_were_free")})
    print(json.dumps(line), flush=True)


def run_single(args):
    """One untimed wavefront frame (1920x1080, 1 spp, depth 5, seed 7) of the ~1.15M-triangle procedural
    scene -- or, with --two-level, of its two-level build -- followed, on the flat scene, by one megakernel
    frame of the same paths: the launches the per-kernel ncu captures select from.  --separate-shadow
    renders the wavefront frame in the separate stage order, --sort with that key sort, --short-stack
    both frames with the shared-memory short stack.  Prints the per-bounce counts."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import scenes
    sc = scenes.instanced_spheres_scene(seed=0) if args.two_level else scenes.spheres_scene(seed=0)
    g = pt.Scene.from_dict(sc)
    cam = sc["camera"]
    g.render(cam, 1, 5, 7, mode="wavefront", separate_shadow=args.separate_shadow, sort=args.sort,
             short_stack=args.short_stack)
    st = g.stats()
    out = {"workload": ("two-level" if args.two_level else "flat") + " 1080p procedural scene, 1 spp, depth 5, seed 7",
           "order": "separate" if args.separate_shadow or args.short_stack else "fused", "sort": args.sort,
           "short_stack": args.short_stack, "status": st["status"],
           "active": st["active"], "shadow_queued": st["shadow_queued"],
           "extension_rays": st["extension_rays"], "shadow_rays": st["shadow_rays"]}
    if not args.two_level:
        g.render(cam, 1, 5, 7, mode="megakernel", short_stack=args.short_stack)
        sm = g.stats()
        out.update(megakernel_extension_rays=sm["extension_rays"], megakernel_shadow_rays=sm["shadow_rays"])
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)
    if st["status"] != 0:
        sys.exit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="frame", choices=["frame", "batch", "large", "diff", "instanced", "single"])
    ap.add_argument("--sort", default="none", choices=["none", "type", "material"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and inverse-rendering summaries")
    ap.add_argument("--separate-shadow", action="store_true", help="separate shadow stage order (frame, single)")
    ap.add_argument("--two-level", action="store_true", help="--workload single: the two-level scene")
    ap.add_argument("--short-stack", action="store_true", help="shared-memory short traversal stack (frame, single)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "large":
        run_large(args)
        return
    if args.workload == "diff":
        run_diff(args)
        return
    if args.workload == "instanced":
        run_instanced(args)
        return
    if args.workload == "single":
        run_single(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
