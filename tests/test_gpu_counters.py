"""Traversal counters (PT_FLAG_COUNT_TRAVERSAL): the counting instantiations of the extend and
shadow stages and of the regenerating megakernel count the BVH nodes visited and the triangles
tested by every walk.  The walks themselves are unchanged, so images, signatures and ray counts equal
the production kernels'.  The wavefront and the megakernel trace exactly the same rays through the
same walk, in different kernels and orders, so their counts must agree exactly; counts are zero when
the flag is off, and camera rays alone (depth 1) make no any-hit walks."""
import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


KEYS = ("nodes_closest", "tris_closest", "nodes_any", "tris_any")


def test_counts_agree_between_integrators_and_leave_images_unchanged(torch):
    import paper_2605_27323_gb300 as pt
    sc = scenes.spheres_scene(seed=5, n_spheres=40, level=3, ground_quads=32, extent=20.0, width=120, height=80)
    cam = sc["camera"]
    g = pt.Scene.from_dict(sc)
    spp, depth, seed = 4, 6, 13
    out = {}
    for mode in ("wavefront", "megakernel"):
        ref = g.render(cam, spp, depth, seed, mode=mode)
        st0 = g.stats()
        assert all(st0[k] == 0 for k in KEYS), st0
        img = g.render(cam, spp, depth, seed, mode=mode, count_traversal=True)
        st = g.stats()
        assert torch.equal(img, ref), mode
        assert (st["extension_rays"], st["shadow_rays"]) == (st0["extension_rays"], st0["shadow_rays"])
        out[mode] = st
    wf, mk = out["wavefront"], out["megakernel"]
    for k in KEYS:
        assert wf[k] == mk[k] > 0, (k, wf[k], mk[k])
    # every walk starts at the root; a leaf holds at most 8 triangles
    assert wf["nodes_closest"] >= wf["extension_rays"] and wf["nodes_any"] >= wf["shadow_rays"]
    assert wf["tris_closest"] <= 8 * wf["nodes_closest"] and wf["tris_any"] <= 8 * wf["nodes_any"]
    # camera rays only: no shadow walks
    g.render(cam, spp, 1, seed, mode="wavefront", count_traversal=True)
    st1 = g.stats()
    assert st1["nodes_any"] == 0 and st1["tris_any"] == 0 and st1["nodes_closest"] > 0
    g.render(cam, spp, 1, seed, mode="megakernel", count_traversal=True)
    assert g.stats()["nodes_closest"] == st1["nodes_closest"]
