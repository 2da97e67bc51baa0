"""GPU parity of two-level (instanced) scenes: meshes in object space placed by instances, a
top-level BVH over the instances, rays taken into each instance's object space.

* a flat scene cut into meshes placed by exact transforms (axis sign flips times powers of
  two) must render bit for bit like the flat scene on the GPU: images, branch signatures and ray
  counts in every mode (the transforms and the object-space intersection are exact), and the same
  gradients up to the order of their float-atomic sums;
* randomly rotated and scaled instances against the oracle (which places them in the world in
  FP64): closest hits equal to brute force away from grazing hits and near ties, per-path parity
  under the same contract as single-level scenes, and the adjoint against dual numbers;
* megakernel == wavefront bitwise on instanced scenes; batched rendering rejects them.
"""
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


@pytest.fixture(scope="module")
def pt(torch):
    import paper_2605_27323_gb300 as P
    return P


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def split_pair(pt):
    sc = scenes.spheres_scene(seed=4, n_spheres=30, level=3, ground_quads=32, extent=15.0, width=120, height=72)
    sc["mat_type"] = np.asarray(sc["mat_type"]).copy()
    return sc, pt.Scene.from_dict(sc), pt.Scene.from_dict(scenes.split_as_instances(sc, 9, seed=5))


@pytest.mark.parametrize("kw", [dict(mode="wavefront"), dict(mode="megakernel"), dict(mode="megakernel", mk_static=True),
                                dict(mode="wavefront", hybrid=3000, sort="material", queue_capacity=7001),
                                dict(mode="wavefront", mis=True, sampler="halton")])
def test_exact_instances_render_like_the_flat_scene(torch, split_pair, kw):
    sc, flat, inst = split_pair
    cam = sc["camera"]
    a = flat.render(cam, 3, 6, 7, sig=True, **kw)
    sa = flat.stats()
    b = inst.render(cam, 3, 6, 7, sig=True, **kw)
    sb = inst.stats()
    assert np.array_equal(_np(a["img"]), _np(b["img"])), kw
    assert np.array_equal(_np(a["sig"]), _np(b["sig"]))
    assert sa["extension_rays"] == sb["extension_rays"] and sa["shadow_rays"] == sb["shadow_rays"]
    assert sb["status"] == 0


def test_exact_instances_same_gradients_and_progressive(torch, split_pair):
    sc, flat, inst = split_pair
    cam = sc["camera"]
    rng = np.random.default_rng(3)
    delta = torch.from_numpy(rng.uniform(0, 1, size=(cam["height"], cam["width"], 3)).astype(np.float32)).cuda()
    # the paths are identical; the gradient sums are formed with float atomics, whose order varies
    for mode in ("wavefront", "megakernel"):
        ga, ge = (_np(x) for x in flat.backward(cam, 2, 5, 1, delta, mode=mode))
        gb, geb = (_np(x) for x in inst.backward(cam, 2, 5, 1, delta, mode=mode))
        assert np.allclose(ga, gb, rtol=1e-5, atol=1e-6 * np.abs(ga).max()), mode
        assert np.allclose(ge, geb, rtol=1e-5, atol=1e-6 * np.abs(ge).max()), mode
    acc = torch.empty((cam["height"], cam["width"], 3), device="cuda")
    inst.render_progressive(cam, 2, 6, 5, 0, acc)
    img = inst.render_progressive(cam, 3, 6, 5, 2, acc)
    assert np.array_equal(_np(img), _np(flat.render(cam, 5, 6, 5)))


@pytest.fixture(scope="module")
def rotated(pt):
    sc = scenes.instanced_spheres_scene(seed=2, n_spheres=40, level=3, ground_quads=64, extent=20.0, width=128,
                                        height=128, n_materials=24)
    return sc, pt.Scene.from_dict(sc), oracle.Scene.from_dict(sc)


def _grazing(u, v):
    return np.minimum(np.minimum(u, v), 1.0 - u - v) < 1e-5


def test_instanced_closest_hit_matches_brute_force(torch, rotated):
    sc, g, osc = rotated
    assert g.n_tris == osc.n_tris == scenes.instance_tri_count(sc)
    rng = np.random.default_rng(8)
    o = rng.uniform([-15, 0.5, -15], [15, 8, 15], size=(200000, 3)).astype(np.float32)
    d = rng.normal(size=(200000, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    tg, pg = (x.cpu().numpy() for x in g.trace_closest(o, d))
    to, po, uo, vo = osc.intersect(o.astype(np.float64), d.astype(np.float64), use_bvh=False)
    differ = pg != po
    both = (pg >= 0) & (po >= 0)
    with np.errstate(invalid="ignore"):
        near_tie = both & (np.abs(tg - to) <= 1e-5 * np.maximum(to, 1e-3))
    graz = (po >= 0) & _grazing(uo, vo)
    assert (differ & ~graz & ~near_tie).sum() == 0, np.flatnonzero(differ & ~graz & ~near_tie)[:5]
    assert differ.mean() < 1e-3 and (po >= 0).mean() > 0.3
    same = ~differ & (po >= 0)
    assert np.allclose(tg[same], to[same], rtol=2e-4, atol=1e-5)


@pytest.mark.parametrize("mode", ["wavefront", "megakernel"])
def test_instanced_paths_match_oracle(torch, rotated, mode):
    sc, g, osc = rotated
    cam = sc["camera"]
    spp, depth, seed = 16, 6, 19
    n = cam["width"] * cam["height"] * spp
    r = g.render(cam, spp, depth, seed, mode=mode, path_L=True, sig=True)
    o = osc.render_paths(cam, spp, depth, seed, np.arange(n), rr_start=3)
    res = compare_with_oracle(_np(r["path_L"]), _np(r["sig"]), o["L"], o["sig"], spp, f"instanced {mode}")
    assert res["same_branch"] > 0.999


def test_instanced_megakernel_equals_wavefront(torch, rotated):
    sc, g, _ = rotated
    cam = sc["camera"]
    wf = g.render(cam, 4, 7, 2, mode="wavefront", sig=True, mis=True)
    mk = g.render(cam, 4, 7, 2, mode="megakernel", sig=True, mis=True)
    assert np.array_equal(_np(wf["img"]), _np(mk["img"])) and np.array_equal(_np(wf["sig"]), _np(mk["sig"]))


def test_instanced_adjoint_matches_oracle_dual_numbers(torch, rotated):
    sc, g, osc = rotated
    cam = sc["camera"]
    W, H = 128, 128
    spp, depth, seed = 8, 5, 12
    rng = np.random.default_rng(9)
    delta = rng.uniform(0.0, 1.0, size=(H, W, 3)).astype(np.float32)
    ga, ge = g.backward(cam, spp, depth, seed, torch.from_numpy(delta).cuda(), rr_start=3)
    ga, ge = _np(ga).astype(np.float64), _np(ge).astype(np.float64)
    nm = len(sc["mat_type"])
    da, de = np.zeros((2, nm, 3)), np.zeros((2, nm))
    da[0] = rng.uniform(0.0, 1.0, size=(nm, 3))
    de[1] = rng.uniform(0.0, 1.0, size=nm)
    ids = np.arange(W * H * spp)
    o = osc.render_paths(cam, spp, depth, seed, ids, rr_start=3, dir_albedo=da, dir_emission=de)
    dflat = delta.reshape(-1, 3)[ids // spp].astype(np.float64)
    oracle_dd = np.einsum("nc,nkc->k", dflat, o["dL"]) / spp
    gpu_dd = np.array([(ga * da[k]).sum() + (ge * de[k]).sum() for k in range(2)])
    assert np.all(np.abs(gpu_dd - oracle_dd) <= 1e-3 * np.abs(oracle_dd)), (gpu_dd, oracle_dd)


def test_instanced_scene_errors(torch, pt, rotated):
    from paper_2605_27323_gb300 import capi
    sc, g, _ = rotated
    with pytest.raises(capi.PtError):
        pt.render_batch([g], [sc["camera"]], [1], 3, 0)
    bad = dict(sc)
    bad["inst_xform"] = np.zeros_like(sc["inst_xform"])          # singular transforms
    with pytest.raises(capi.PtError):
        pt.Scene.from_dict(bad)
    bad = dict(sc)
    bad["inst_mesh"] = np.asarray(sc["inst_mesh"]).copy()
    bad["inst_mesh"][0] = 99
    with pytest.raises(capi.PtError):
        pt.Scene.from_dict(bad)
