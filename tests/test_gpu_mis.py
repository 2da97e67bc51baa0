"""GPU parity of multiple importance sampling (PT_FLAG_MIS): next-event estimation and BSDF-sampled
hits on listed lights combined with the power heuristic.

Per-path parity with the oracle's MIS estimator (same contract as the default estimator), the
megakernel == wavefront (also hybrid, batched and progressive) bitwise, the adjoint under MIS
against the oracle's dual numbers, and the MIS image against the NEE-only image within Monte
Carlo error (the weights change the variance, not the expectation).
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


def _glossy_box(width=128, height=128):
    # the tiny box with a GGX box (roughness 0.3), a GGX back wall (roughness 0.15) and a glass box
    sc = scenes.box_scene(seed=1, width=width, height=height, lift=2e-3)
    sc["mat_type"] = np.asarray(sc["mat_type"]).copy()
    sc["mat_roughness"] = np.asarray(sc["mat_roughness"], np.float32).copy()
    sc["mat_type"][2], sc["mat_roughness"][2] = scenes.GGX, 0.15
    sc["mat_type"][5], sc["mat_roughness"][5] = scenes.GGX, 0.3
    sc["mat_type"][6] = scenes.DIELECTRIC
    return sc


@pytest.mark.parametrize("mode", ["wavefront", "megakernel"])
def test_mis_paths_match_oracle(pt, torch, mode):
    sc = _glossy_box()
    cam = sc["camera"]
    spp, depth, seed = 16, 8, 23
    n = 128 * 128 * spp
    g = pt.Scene.from_dict(sc)
    r = g.render(cam, spp, depth, seed, mode=mode, path_L=True, sig=True, mis=True)
    o = oracle.Scene.from_dict(sc).render_paths(cam, spp, depth, seed, np.arange(n), rr_start=3, mis=True)
    res = compare_with_oracle(_np(r["path_L"]), _np(r["sig"]), o["L"], o["sig"], spp, f"mis {mode}")
    assert res["same_branch"] > 0.999
    assert not np.array_equal(_np(r["img"]), _np(g.render(cam, spp, depth, seed, mode=mode)))


def test_mis_megakernel_wavefront_hybrid_batch_progressive(pt, torch):
    sc = scenes.spheres_scene(seed=5, n_spheres=30, level=3, ground_quads=32, extent=15.0, width=120, height=72)
    g = pt.Scene.from_dict(sc)
    cam = sc["camera"]
    kw = dict(mis=True, sampler="halton")
    wf = g.render(cam, 4, 6, 3, mode="wavefront", sig=True, **kw)
    mk = g.render(cam, 4, 6, 3, mode="megakernel", sig=True, **kw)
    assert np.array_equal(_np(wf["img"]), _np(mk["img"])) and np.array_equal(_np(wf["sig"]), _np(mk["sig"]))
    assert np.array_equal(_np(g.render(cam, 4, 6, 3, mode="wavefront", hybrid=4000, **kw)), _np(wf["img"]))
    assert np.array_equal(_np(g.render(cam, 4, 6, 3, mode="wavefront", sort="material", queue_capacity=5000, **kw)),
                          _np(wf["img"]))
    box = _glossy_box(40, 30)
    gb = pt.Scene.from_dict(box)
    outs = pt.render_batch([g, gb], [cam, box["camera"]], [4, 3], 6, 3, **kw)
    assert np.array_equal(_np(outs[0]), _np(wf["img"]))
    assert np.array_equal(_np(outs[1]), _np(gb.render(box["camera"], 3, 6, 3, **kw)))
    p = pt.Progressive(g, cam, 6, seed=3, **kw)
    p.add(1)
    assert np.array_equal(_np(p.add(3)), _np(wf["img"]))


def test_mis_image_matches_nee_image_within_mc_error(pt, torch):
    sc = _glossy_box(48, 32)
    g = pt.Scene.from_dict(sc)
    cam = sc["camera"]
    spp = 2048
    a = _np(g.render(cam, spp, 6, 1, mis=True)).astype(np.float64)
    r = g.render(cam, spp, 6, 2, path_L=True)
    L = _np(r["path_L"]).astype(np.float64).reshape(48 * 32, spp, 3)
    b = L.mean(1).reshape(32, 48, 3)
    se = (L.std(1, ddof=1) / np.sqrt(spp)).reshape(32, 48, 3)
    z = (a - b) / (np.sqrt(2) * se + 1e-9)
    assert np.median(np.abs(z)) < 1.0
    assert abs(a.mean() - b.mean()) < 4 * np.sqrt(np.sum(2 * se ** 2)) / se.size


def test_mis_adjoint_matches_oracle_dual_numbers(pt, torch):
    sc = scenes.spheres_scene(seed=0, n_materials=64, n_spheres=60, level=3, ground_quads=64, extent=20.0,
                              width=96, height=96)
    cam = sc["camera"]
    spp, depth, seed = 16, 5, 8
    W, H = cam["width"], cam["height"]
    g = pt.Scene.from_dict(sc)
    rng = np.random.default_rng(5)
    delta = rng.uniform(0.0, 1.0, size=(H, W, 3)).astype(np.float32)
    ga, ge = g.backward(cam, spp, depth, seed, torch.from_numpy(delta).cuda(), rr_start=3, mis=True)
    ga, ge = _np(ga).astype(np.float64), _np(ge).astype(np.float64)
    nm = len(sc["mat_type"])
    da = np.zeros((3, nm, 3))
    de = np.zeros((3, nm))
    da[0] = rng.uniform(0.0, 1.0, size=(nm, 3))
    de[1] = rng.uniform(0.0, 1.0, size=nm)
    de[2, nm - 1] = 1.0                               # the lights' emission: NEE and BSDF-hit terms
    ids = np.arange(W * H * spp)
    o = oracle.Scene.from_dict(sc).render_paths(cam, spp, depth, seed, ids, rr_start=3, dir_albedo=da,
                                                 dir_emission=de, mis=True)
    dflat = delta.reshape(-1, 3)[ids // spp].astype(np.float64)
    oracle_dd = np.einsum("nc,nkc->k", dflat, o["dL"]) / spp
    gpu_dd = np.array([(ga * da[k]).sum() + (ge * de[k]).sum() for k in range(3)])
    assert np.all(np.abs(gpu_dd - oracle_dd) <= 1e-3 * np.abs(oracle_dd)), (gpu_dd, oracle_dd)
    ga2, ge2 = g.backward(cam, spp, depth, seed, torch.from_numpy(delta).cuda(), rr_start=3, mis=True,
                          mode="megakernel")
    assert np.allclose(_np(ga2), ga, rtol=1e-4, atol=1e-7 * np.abs(ga).max())
    assert np.allclose(_np(ge2), ge, rtol=1e-4, atol=1e-7 * np.abs(ge).max())
