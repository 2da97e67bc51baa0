"""The batched workload at its full size, in the launch configuration the benchmark times: the 64
procedural scenes (lognormal triangle counts in [1k, 2M], resolutions from {256^2, 512^2, 1280x720,
1920x1080}, spp from {1, 4, 16}, depth 5) rendered in one pt_render_batch call with the autotuner's
queue capacity, block size and sort granularity.  Sampled pixels of eight scenes (the largest render,
the most triangles, and six others) are checked against the FP64 oracle's pixels: a pixel is the
mean of its spp paths, so it must match to 1e-4 relative unless one of its paths left the oracle's
branches (a few in 10^4 paths); >= 99% of the sampled pixels must match, and the median relative
error must stay at FP32 rounding level."""
import numpy as np
import pytest

import oracle
from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_full_batch_mix_sampled_pixels_match_the_oracle():
    import torch

    import paper_2605_27323_gb300 as pt
    assert torch.cuda.is_available()
    specs = scenes.batch_scenes(seed=0)
    gs = [pt.Scene.from_dict(sc) for sc in specs]
    cams = [sc["camera"] for sc in specs]
    spps = [int(sc["spp"]) for sc in specs]
    depth, seed = 5, 17
    outs = [torch.empty((c["height"], c["width"], 3), device="cuda") for c in cams]
    best = pt.autotune_batch(gs, cams, spps, depth, 0, outs=outs)
    pt.render_batch(gs, cams, spps, depth, seed, outs=outs, queue_capacity=best["queue_capacity"],
                    block_size=best["block_size"], sort=int(best["sort"]))
    torch.cuda.synchronize()
    paths = [c["width"] * c["height"] * s for c, s in zip(cams, spps)]
    tris = [len(sc["tris"]) for sc in specs]
    pick = {int(np.argmax(paths)), int(np.argmax(tris))}
    rng = np.random.default_rng(4)
    for i in rng.permutation(len(specs)):
        if len(pick) >= 8:
            break
        pick.add(int(i))
    agree, rel_all = 0, []
    n_checked = 0
    for i in sorted(pick):
        sc, cam, spp = specs[i], cams[i], spps[i]
        img = outs[i].cpu().numpy().reshape(-1, 3).astype(np.float64)
        n_pix = cam["width"] * cam["height"]
        px = np.sort(rng.choice(n_pix, size=min(n_pix, 256), replace=False)).astype(np.uint32)
        ref, _ = oracle.Scene.from_dict(sc).render_pixels(cam, spp, depth, seed, px, rr_start=3)
        g = img[px]
        scale = max(1e-12, float(np.abs(ref).max()))
        ok = np.all(np.abs(g - ref) <= 1e-4 * np.abs(ref) + 1e-6 * scale, axis=1)
        agree += int(ok.sum())
        n_checked += len(px)
        rel_all.append((np.abs(g - ref) / np.maximum(np.abs(ref), 1e-6 * scale)).max(axis=1))
    rel = np.concatenate(rel_all)
    assert agree >= 0.99 * n_checked, (agree, n_checked)
    assert np.median(rel) < 1e-5, float(np.median(rel))
