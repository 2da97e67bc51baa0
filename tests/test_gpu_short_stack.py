"""The shared-memory short traversal stack (PT_FLAG_SHORT_STACK): per-warp short stacks of the
scene-intersection stage (Sec. 2.3) and the shadow evaluation (Sec. 3), 8 entries per lane in shared
memory with the deeper entries in local memory.  The walk visits the same nodes in the same order,
so every integrator must give bit-identical images, signatures and ray counts with and without it;
the default render is checked against the FP64 oracle in the same test, so the short-stack renders
are tied to the oracle too.  A dense random soup drives the stacks well past 8 entries, so the
spill to local memory and the pops back out of it are exercised."""
import numpy as np
import pytest

import oracle
from helpers import compare_with_oracle
from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


def _scenes():
    soup = scenes.random_soup(n_tris=6000, seed=9, spread=1.0, size=0.15, n_mats=4)
    soup["mat_emission"] = np.array([0.0, 0.0, 0.0, 4.0], np.float32)
    soup["camera"] = scenes.camera((0.0, 0.3, 3.5), (0.0, 0.0, 0.0), (0, 1, 0), 45.0, 64, 48)
    sph = scenes.spheres_scene(seed=2, n_spheres=40, level=3, ground_quads=32, extent=20.0, width=96, height=64)
    return {"soup": soup, "spheres": sph}


@pytest.mark.parametrize("name", ["soup", "spheres"])
def test_short_stack_renders_bit_identically(torch, name):
    import paper_2605_27323_gb300 as pt
    sc = _scenes()[name]
    cam = sc["camera"]
    spp, depth, seed = 4, 8, 21
    g = pt.Scene.from_dict(sc)
    runs = {}
    for mode, kw in (("wavefront", {}), ("megakernel", {}), ("hybrid", {"hybrid": 1 << 30})):
        m = "wavefront" if mode == "hybrid" else mode
        for ss in (False, True):
            r = g.render(cam, spp, depth, seed, path_L=True, sig=True, mode=m, short_stack=ss, rr_start=3, **kw)
            st = g.stats()
            assert st["status"] == 0, (mode, ss, st["status"])
            runs[(mode, ss)] = (r["img"].cpu().numpy(), r["sig"].cpu().numpy(), r["path_L"].cpu().numpy(),
                                st["extension_rays"], st["shadow_rays"])
    ref = runs[("wavefront", False)]
    for key, v in runs.items():
        assert np.array_equal(v[0], ref[0]) and np.array_equal(v[1], ref[1]), key
        assert v[3:] == ref[3:], (key, v[3:], ref[3:])
    n = cam["width"] * cam["height"] * spp
    o = oracle.Scene.from_dict(sc).render_paths(cam, spp, depth, seed, np.arange(n), rr_start=3)
    compare_with_oracle(ref[2], ref[1], o["L"], o["sig"], spp, label=f"short stack {name}")


def test_short_stack_closest_hits_match_brute_force_on_a_deep_soup(torch):
    """Closest hits through the wavefront's extend stage with the short stack equal the oracle's
    brute-force hits on rays that cross the dense soup (deep stacks)."""
    import paper_2605_27323_gb300 as pt
    sc = _scenes()["soup"]
    cam = dict(sc["camera"], width=40, height=30)
    g = pt.Scene.from_dict(sc)
    a = g.render(cam, 1, 1, 3, sig=True, mode="wavefront", short_stack=True)["sig"].cpu().numpy().astype(np.uint32)
    b = g.render(cam, 1, 1, 3, sig=True, mode="wavefront")["sig"].cpu().numpy().astype(np.uint32)
    assert np.array_equal(a, b)
    o = oracle.Scene.from_dict(sc).render_paths(cam, 1, 1, 3, np.arange(40 * 30), use_bvh=False)
    assert (a == o["sig"]).mean() >= 0.999
