"""The fused stage order of the wavefront (each bounce's extend launch also walks the shadow rays the
previous shading cast; the default) against the paper's separate order (PT_FLAG_SEPARATE_SHADOW,
a shadow stage after each shading): the same walks and the same additions to each path's radiance
in the same order, so images, per-path radiance, signatures and ray counts (per bounce too) are
bit-identical -- on single-level and two-level scenes, with MIS and the Halton jitter, in waves,
with the key sort, and through the adjoint replay.  The default order is the one every oracle-parity test exercises."""
import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


def _cases():
    box = scenes.box_scene(width=48, height=40, lift=2e-3)
    box["mat_type"] = box["mat_type"].copy()
    box["mat_roughness"] = box["mat_roughness"].copy()
    box["mat_type"][5], box["mat_roughness"][5] = 1, 0.25
    box["mat_type"][6] = 2
    sph = scenes.spheres_scene(seed=7, n_spheres=30, level=3, ground_quads=32, extent=20.0, width=120, height=68)
    inst = scenes.instanced_spheres_scene(seed=2, n_spheres=20, level=2, ground_quads=16, extent=15.0, width=96,
                                          height=64, n_materials=10)
    return [("box", box, 8, 8, {}), ("box_mis_halton", box, 4, 12, {"mis": True, "sampler": "halton"}),
            ("spheres_waves_sort", sph, 3, 6, {"queue_capacity": 999, "sort": "material"}),
            ("instanced", inst, 2, 7, {})]


@pytest.mark.parametrize("k", range(4))
def test_fused_and_separate_orders_agree_bitwise(torch, k):
    import paper_2605_27323_gb300 as pt
    name, sc, spp, depth, kw = _cases()[k]
    g = pt.Scene.from_dict(sc)
    cam = sc["camera"]
    out = {}
    for sep in (False, True):
        r = g.render(cam, spp, depth, 5, mode="wavefront", path_L=True, sig=True, separate_shadow=sep, **kw)
        st = g.stats()
        assert st["status"] == 0
        out[sep] = (r["img"].cpu().numpy(), r["path_L"].cpu().numpy(), r["sig"].cpu().numpy(),
                    st["extension_rays"], st["shadow_rays"], st["active"], st["shadow_queued"])
        assert sum(st["shadow_queued"]) == st["shadow_rays"] and sum(st["active"]) == st["extension_rays"]
    a, b = out[False], out[True]
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y), name
    assert a[3:] == b[3:], (name, a[3:5], b[3:5])
    assert a[4] > 0
    mk = g.render(cam, spp, depth, 5, mode="megakernel", **{q: v for q, v in kw.items() if q in ("mis", "sampler")})
    assert np.array_equal(mk.cpu().numpy(), a[0]), name


def test_adjoint_replay_orders_agree(torch):
    import paper_2605_27323_gb300 as pt
    sc = scenes.spheres_scene(seed=7, n_spheres=30, level=3, ground_quads=32, extent=20.0, width=120, height=68,
                              n_materials=24)
    g = pt.Scene.from_dict(sc)
    cam = sc["camera"]
    rng = np.random.default_rng(2)
    delta = torch.from_numpy(rng.uniform(0.0, 1.0, size=(68, 120, 3)).astype(np.float32)).cuda()
    ga, ge = g.backward(cam, 4, 6, 9, delta, rr_start=2, rr_fixed=0.8)
    gb, gE = g.backward(cam, 4, 6, 9, delta, rr_start=2, rr_fixed=0.8, separate_shadow=True)
    # the same records; only the order of the float atomics that add them up may differ
    assert torch.allclose(ga, gb, rtol=1e-5, atol=1e-7 * float(gb.abs().max()))
    assert torch.allclose(ge, gE, rtol=1e-5, atol=1e-7 * float(gE.abs().max()))
    assert float(gb.abs().sum()) > 0
