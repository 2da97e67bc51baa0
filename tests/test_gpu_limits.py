"""Limits of the path indexing: a render of more than 2^32 paths (64 x 64 pixels x 1,048,577
samples, depth 1, in 128 waves of 2^25 paths).  Path ids, pixel / sample decomposition and the
per-wave accumulation must carry 64-bit ids: the paths' camera-ray hits near and beyond id 2^32
equal the oracle's, and every pixel equals the oracle's count of light hits times Le / spp (with
depth 1 a sample adds exactly 0 or Le = 15; FP32 sums of such terms are exact below 2^24, so the
only differences are samples whose ray lands within FP32 error of the light's edge)."""
import numpy as np
import pytest

import oracle
from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


def test_more_than_2_to_32_paths(torch):
    import paper_2605_27323_gb300 as pt
    sc = scenes.box_scene(seed=0, width=64, height=64)
    cam = sc["camera"]
    spp = (1 << 20) + 1
    n_px = 64 * 64
    assert n_px * spp > (1 << 32)
    g = pt.Scene.from_dict(sc)
    img = g.render(cam, spp, 1, 3, mode="wavefront", queue_capacity=1 << 25).cpu().numpy().reshape(-1, 3)
    st = g.stats()
    assert st["status"] == 0 and st["extension_rays"] == n_px * spp
    # paths around and beyond id 2^32 against the oracle, hit by hit
    ids = np.array([0, 1, (1 << 32) - 2, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, n_px * spp - 1,
                    3000 * spp + 777, 4095 * spp + 12345], np.uint64)
    ev_g, L_g = g.path_events(cam, spp, 1, 3, ids)
    osc = oracle.Scene.from_dict(sc)
    ev_o, L_o = osc.path_events(cam, spp, 1, 3, ids)
    assert len(ev_g) == len(ev_o) == len(ids)
    for a, b in zip(ev_g, ev_o):
        assert [e[:3] for e in a] == [e[:3] for e in b]
    assert np.allclose(L_g, L_o, rtol=1e-6, atol=0)
    # pixels: count of light hits x 15 / spp; the oracle counts them for a few pixels
    le = 15.0
    pix = np.array([0, 4 * 64 + 30, 5 * 64 + 25, 5 * 64 + 32, 5 * 64 + 38], np.uint32)   # black, edges, inside
    o_img, _ = osc.render_pixels(cam, spp, 1, 3, pixels=pix)
    for k, px in enumerate(pix):
        k_o = o_img[k, 0] * spp / le
        k_g = float(img[px, 0]) * spp / le
        assert abs(k_g - k_o) <= 4.0 + 1e-6 * k_o, (int(px), k_g, k_o)
    assert o_img[1, 0] > 0 and o_img[3, 0] == le
    assert np.all(img[:, 0] == img[:, 1]) and np.all(img[:, 0] == img[:, 2])
