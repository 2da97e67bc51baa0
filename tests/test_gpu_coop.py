"""Cooperative walks in the fused trace stage: when a trace launch has few walks for its grid (the
sparse late bounces), groups of G = 2, 4, ..., 32 lanes share each ray, walking its subtrees side by
side and culling against the group's best distance.  The hit is the smallest (t, original id) over
the group, which is the one-lane walk's hit, so a render must be bit-identical to the separate stage
order (one lane per walk in every launch) and to the megakernel: images, per-path radiance, branch
signatures and ray counts -- on single-level scenes and on a two-level scene, whose group walks carry
each deferred subtree's instance.  The scenes are rendered deep enough that most group sizes run
(`group_walks` counts the walks of each size); the dense soup makes long walks whose deferred
subtrees move between lanes.  Cooperative paths are tied to brute force too: the default render's
paths are compared with the FP64 oracle walking every triangle (no BVH)."""
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


def _soup():
    sc = scenes.random_soup(n_tris=6000, seed=9, spread=1.0, size=0.15, n_mats=4)
    sc["mat_emission"] = np.array([0.0, 0.0, 0.0, 4.0], np.float32)
    sc["camera"] = scenes.camera((0.0, 0.3, 3.5), (0.0, 0.0, 0.0), (0, 1, 0), 45.0, 64, 48)
    return sc


def _cases():
    sph = scenes.spheres_scene(seed=4, n_spheres=40, level=3, ground_quads=32, extent=20.0, width=96, height=64)
    inst = scenes.instanced_spheres_scene(seed=2, n_spheres=20, level=2, ground_quads=16, extent=15.0, width=96,
                                          height=64, n_materials=10)
    return [("soup", _soup(), 4, 14, {}), ("spheres", sph, 8, 16, {}),
            ("spheres_mis_halton", sph, 2, 12, {"mis": True, "sampler": "halton"}),
            ("two_level", inst, 4, 12, {})]


def test_cooperative_walks_are_bit_identical(torch):
    import paper_2605_27323_gb300 as pt
    sizes = np.zeros(5, np.int64)
    for name, sc, spp, depth, kw in _cases():
        g = pt.Scene.from_dict(sc)
        cam = sc["camera"]
        out = {}
        for sep in (False, True):
            r = g.render(cam, spp, depth, 3, mode="wavefront", path_L=True, sig=True, separate_shadow=sep,
                         rr_start=3, **kw)
            st = g.stats()
            assert st["status"] == 0, (name, sep)
            out[sep] = (r, st)
        (a, sa), (b, sb) = out[False], out[True]
        sizes += np.asarray(sa["group_walks"])
        assert sum(sa["group_walks"]) > 0, (name, sa["group_walks"])
        assert sum(sb["group_walks"]) == 0, sb["group_walks"]       # the separate order walks one lane each
        assert sum(sa["group_walks"]) < sa["extension_rays"] + sa["shadow_rays"]
        for key in ("img", "path_L", "sig"):
            assert torch.equal(a[key], b[key]), (name, key)
        assert (sa["extension_rays"], sa["shadow_rays"], sa["active"], sa["shadow_queued"]) == \
            (sb["extension_rays"], sb["shadow_rays"], sb["active"], sb["shadow_queued"]), name
        mk = g.render(cam, spp, depth, 3, mode="megakernel", rr_start=3, **kw)
        assert torch.equal(mk, a["img"]), name
    # groups of 2, 4, 8, 16, 32 lanes: most sizes ran over the four renders
    assert int((sizes > 0).sum()) >= 4, sizes.tolist()


def test_cooperative_walks_match_brute_force_oracle(torch):
    """The soup rendered at depth 4: bounces 2-3 run cooperatively; every path against the oracle's
    brute-force closest and any hits."""
    import paper_2605_27323_gb300 as pt
    sc = _soup()
    cam = dict(sc["camera"], width=40, height=30)
    spp, depth, seed = 2, 4, 11
    g = pt.Scene.from_dict(sc)
    r = g.render(cam, spp, depth, seed, mode="wavefront", path_L=True, sig=True, rr_start=3)
    st = g.stats()
    assert st["status"] == 0 and sum(st["group_walks"]) > 0, st["group_walks"]
    n = cam["width"] * cam["height"] * spp
    o = oracle.Scene.from_dict(sc).render_paths(cam, spp, depth, seed, np.arange(n), rr_start=3, use_bvh=False)
    compare_with_oracle(r["path_L"].cpu().numpy(), r["sig"].cpu().numpy(), o["L"], o["sig"], spp,
                        label="cooperative walks vs brute force")


def test_group_walks_off_in_the_counting_pass(torch):
    """The traversal-counting pass keeps one lane per walk (its counts describe that walk)."""
    import paper_2605_27323_gb300 as pt
    sph = scenes.spheres_scene(seed=4, n_spheres=40, level=3, ground_quads=32, extent=20.0, width=64, height=48)
    g = pt.Scene.from_dict(sph)
    a = g.render(sph["camera"], 4, 12, 1, mode="wavefront", count_traversal=True)
    assert sum(g.stats()["group_walks"]) == 0
    b = g.render(sph["camera"], 4, 12, 1, mode="wavefront")
    assert sum(g.stats()["group_walks"]) > 0
    assert torch.equal(a, b)
