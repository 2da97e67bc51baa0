"""Progressive accumulation (the running average of the accumulation stage, Sec. 2.3) and the
hybrid wavefront/megakernel render (the hybrid named as future work, Sec. 6.1).

Progressive frames continue each pixel's FP32 sum in sample order, so frames of k1, k2, ... samples
must give the one-call image of k1 + k2 + ... samples bit for bit, in both modes and across waves,
and a render resumed from a saved (sums, count) state must continue identically.  A frame that
starts at a sample offset is also compared with the oracle on those samples.  The hybrid finishes
the last sparse bounces in one kernel with the megakernel's arithmetic, so images, branch
signatures and ray counts must equal the plain wavefront's.
"""
import numpy as np
import pytest

import oracle
from helpers import ATOL_REL, MIN_PIXEL_AGREEMENT, RTOL
from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


@pytest.fixture(scope="module")
def pt(torch):
    import paper_2605_27323_gb300 as P
    return P


@pytest.fixture(scope="module")
def box(pt):
    sc = scenes.box_scene(seed=0, width=72, height=40, lift=2e-3)
    return sc, pt.Scene.from_dict(sc), sc["camera"]


@pytest.fixture(scope="module")
def spheres(pt):
    sc = scenes.spheres_scene(seed=2, n_spheres=40, level=3, ground_quads=64, extent=20.0, width=160, height=90)
    return sc, pt.Scene.from_dict(sc), sc["camera"]


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("mode", ["wavefront", "megakernel"])
@pytest.mark.parametrize("frames", [(16,), (1, 3, 4, 8), (5, 11)])
def test_progressive_frames_equal_one_call(torch, box, mode, frames):
    _, g, cam = box
    depth, seed = 8, 5
    ref = _np(g.render(cam, sum(frames), depth, seed, mode=mode))
    acc = torch.full((cam["height"], cam["width"], 3), 7.0, device="cuda")   # overwritten: offset 0
    off = 0
    for k in frames:
        img = g.render_progressive(cam, k, depth, seed, off, acc, mode=mode)
        off += k
    assert np.array_equal(_np(img), ref)
    assert np.array_equal(_np(acc) * np.float32(1.0 / off), ref)


def test_progressive_first_frame_and_modes(torch, box):
    _, g, cam = box
    acc_w = torch.empty((cam["height"], cam["width"], 3), device="cuda")
    acc_m = torch.empty_like(acc_w)
    first = g.render_progressive(cam, 4, 8, 9, 0, acc_w, mode="wavefront")
    assert np.array_equal(_np(first), _np(g.render(cam, 4, 8, 9, mode="wavefront")))
    g.render_progressive(cam, 4, 8, 9, 0, acc_m, mode="megakernel")
    a = g.render_progressive(cam, 6, 8, 9, 4, acc_w, mode="wavefront", queue_capacity=999)   # several waves
    b = g.render_progressive(cam, 6, 8, 9, 4, acc_m, mode="megakernel")
    assert np.array_equal(_np(a), _np(b))
    assert np.array_equal(_np(a), _np(g.render(cam, 10, 8, 9)))


def test_progressive_resume(torch, pt, box):
    _, g, cam = box
    p = pt.Progressive(g, cam, 8, seed=3)
    p.add(2)
    p.add(5)
    state = p.state()
    q = pt.Progressive.resume(g, cam, 8, state)
    img_q = q.add(9)
    img_p = p.add(9)
    assert p.count == q.count == 16
    assert np.array_equal(_np(img_p), _np(img_q))
    assert np.array_equal(_np(img_p), _np(g.render(cam, 16, 8, 3)))


def test_progressive_offset_frame_matches_oracle(torch, box):
    """Samples o .. o+m-1 alone (sums start at zero with a non-zero offset) against the oracle's
    paths of those samples: pixels whose paths all follow the same branches agree to the parity
    tolerance, and >= 99.9% of pixels agree."""
    sc, g, cam = box
    W, H = cam["width"], cam["height"]
    o_, m, depth, seed = 5, 3, 8, 21
    acc = torch.zeros((H, W, 3), device="cuda")
    sig = torch.empty(W * H * m, device="cuda", dtype=torch.int32)
    img = _np(g.render_progressive(cam, m, depth, seed, o_, acc, sig=sig)).reshape(-1, 3).astype(np.float64)
    gsig = _np(sig).astype(np.uint32).reshape(W * H, m)
    total = o_ + m
    ids = (np.arange(W * H, dtype=np.uint64)[:, None] * total + o_ + np.arange(m, dtype=np.uint64)[None, :]).reshape(-1)
    r = oracle.Scene.from_dict(sc).render_paths(cam, total, depth, seed, ids)
    osig = r["sig"].reshape(W * H, m)
    or_img = r["L"].reshape(W * H, m, 3).sum(1) / total
    scale = max(1e-12, float(np.abs(r["L"]).max()))
    close = np.all(np.abs(img - or_img) <= RTOL * np.abs(or_img) + ATOL_REL * scale, axis=-1)
    same = (gsig == osig).all(1)
    assert (same & ~close).sum() == 0
    assert (same & close).mean() >= MIN_PIXEL_AGREEMENT


def test_progressive_max_depth_zero_and_errors(torch, pt, box):
    from paper_2605_27323_gb300 import capi
    _, g, cam = box
    acc = torch.ones((cam["height"], cam["width"], 3), device="cuda")
    img = g.render_progressive(cam, 4, 0, 1, 4, acc)               # black samples: sums kept, count 8
    assert np.array_equal(_np(img), np.full(img.shape, np.float32(1.0) * np.float32(1.0 / 8), np.float32))
    with pytest.raises(capi.PtError):
        g.render_progressive(cam, 1, 4, 0, 0, torch.zeros((cam["height"], cam["width"], 3)))   # host sums
    with pytest.raises(capi.PtError):
        g.render_progressive(cam, 2, 4, 0, 0xFFFFFFFF, acc)            # sample index overflow


@pytest.mark.parametrize("thr", [1, 700, 3000, 1 << 30])
@pytest.mark.parametrize("kw", [{}, {"queue_capacity": 4001}, {"sort": "material"}])
def test_hybrid_equals_wavefront(torch, spheres, thr, kw):
    _, g, cam = spheres
    depth, spp, seed = 7, 2, 13
    n = cam["width"] * cam["height"] * spp
    ref = g.render(cam, spp, depth, seed, mode="wavefront", sig=True, **kw)
    st_ref = g.stats()
    out = g.render(cam, spp, depth, seed, mode="wavefront", sig=True, hybrid=thr, **kw)
    st = g.stats()
    assert np.array_equal(_np(out["img"]), _np(ref["img"]))
    assert np.array_equal(_np(out["sig"]), _np(ref["sig"]))
    assert st["extension_rays"] == st_ref["extension_rays"] and st["shadow_rays"] == st_ref["shadow_rays"]
    assert st["active"] == st_ref["active"]
    assert st["status"] == 0 and n > 0


def test_hybrid_progressive_and_megakernel_agree(torch, box):
    _, g, cam = box
    acc = torch.empty((cam["height"], cam["width"], 3), device="cuda")
    g.render_progressive(cam, 3, 8, 4, 0, acc, mode="wavefront", hybrid=500)
    img = g.render_progressive(cam, 5, 8, 4, 3, acc, mode="wavefront", hybrid=1 << 20)
    assert np.array_equal(_np(img), _np(g.render(cam, 8, 8, 4, mode="megakernel")))
