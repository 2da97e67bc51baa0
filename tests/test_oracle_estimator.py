"""Oracle pins: the whole estimator against closed forms (tests/golden/*.txt).

* white furnace (closed Lambert enclosure, all faces emit and are lights): E[L] = sum a^k
  with and without Russian roulette, d/da and d/dLe series;
* direct lighting of a Lambert plane by a parallel one-sided rectangle (form factor);
* glass in a furnace: every escaping path carries exactly Le (refraction in and out scales
  radiance by (1/eta)^2 * eta^2 = 1; reflections carry 1);
* dual-number derivatives == central finite differences of the oracle itself;
* the image function == mean of the per-path function in sample order, and the BVH and
  brute-force paths give identical estimates.
"""
import os

import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([float(x) for x in line.split()])
    return out


def _sphere_rays(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.zeros((n, 3)) + rng.uniform(-0.2, 0.2, size=(n, 3)), d


@pytest.mark.parametrize("a,D,expect", [tuple(r) for r in _rows("furnace.txt")])
def test_furnace_series_golden(oracle_lib, a, D, expect):
    assert abs(sum(a ** k for k in range(int(D))) - expect) < 1e-12   # the table itself
    sc = oracle_lib.Scene.from_dict(scenes.furnace_sphere(albedo=a, emission=1.0, level=4))
    o, d = _sphere_rays(20000, 1)
    L, _ = sc.trace_rays(o, d, np.arange(20000), max_depth=int(D))
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(len(L))
    assert abs(m - expect) < 3 * se + 2e-3 * expect, (m, se, expect)


def test_furnace_with_roulette_converges_to_geometric_limit(oracle_lib):
    a = 0.6
    sc = oracle_lib.Scene.from_dict(scenes.furnace_sphere(albedo=a, emission=1.0, level=4))
    o, d = _sphere_rays(40000, 2)
    L, _ = sc.trace_rays(o, d, np.arange(40000), max_depth=200, rr_start=3)
    m, se = L[:, 1].mean(), L[:, 1].std() / np.sqrt(len(L))
    expect = 1.0 / (1.0 - a)
    assert abs(m - expect) < 3 * se + 3e-3 * expect, (m, se, expect)
    # fixed survival probability is unbiased too
    L2, _ = sc.trace_rays(o, d, np.arange(40000), max_depth=200, rr_start=2, rr_fixed=0.7)
    m2, se2 = L2[:, 2].mean(), L2[:, 2].std() / np.sqrt(len(L2))
    assert abs(m2 - expect) < 3 * se2 + 3e-3 * expect, (m2, se2, expect)


def test_furnace_derivatives(oracle_lib):
    a, D = 0.5, 5
    s = scenes.furnace_sphere(albedo=a, emission=1.0, level=4)
    sc = oracle_lib.Scene.from_dict(s)
    o, d = _sphere_rays(10000, 3)
    da = np.zeros((2, 1, 3))
    de = np.zeros((2, 1))
    da[0, 0] = 1.0       # direction 0: all albedo channels of material 0
    de[1, 0] = 1.0       # direction 1: emission of material 0
    L, dL = sc.trace_rays(o, d, np.arange(10000), max_depth=D, dir_albedo=da, dir_emission=de)
    dA = sum(k * a ** (k - 1) for k in range(1, D))
    dE = sum(a ** k for k in range(D))
    g = dL[:, 0, 0]
    assert abs(g.mean() - dA) < 3 * g.std() / np.sqrt(len(g)) + 2e-3 * dA
    # linear in emission: dL/dLe == L / Le exactly per path
    assert np.allclose(dL[:, 1, :], L, rtol=1e-12, atol=1e-15)
    assert abs(dL[:, 1, 0].mean() - dE) < 3 * dL[:, 1, 0].std() / np.sqrt(len(g)) + 2e-3 * dE


def _corner_ff(X, Y):
    ax, ay = abs(X), abs(Y)
    sx, sy = np.sqrt(1 + ax * ax), np.sqrt(1 + ay * ay)
    return (ax / sx * np.arctan(ay / sx) + ay / sy * np.arctan(ax / sy)) / (2 * np.pi)


def _point_ff(px, pz, hw, hh, c):
    # superposition of the four corner rectangles around the foot point (point under the rect)
    total = 0.0
    for wx in (hw - px, hw + px):
        for wz in (hh - pz, hh + pz):
            total += _corner_ff(wx / c, wz / c)
    return total


@pytest.mark.parametrize("px,pz,hw,hh,c", [tuple(r) for r in _rows("form_factor_parallel_rect.txt")])
def test_direct_light_form_factor(oracle_lib, px, pz, hw, hh, c):
    rho, Le = 0.7, 5.0
    sc = oracle_lib.Scene.from_dict(scenes.rect_over_plane(albedo=rho, emission=Le, half_w=hw, half_h=hh,
                                                           height=c))
    n = 100_000
    o = np.tile([px, 0.5 * c, pz], (n, 1))
    d = np.tile([0.0, -1.0, 0.0], (n, 1))
    L, _ = sc.trace_rays(o, d, np.arange(n), max_depth=2)
    expect = rho * Le * _point_ff(px, pz, hw, hh, c)
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(n)
    assert abs(m - expect) < 4 * se + 1e-4 * expect, (m, se, expect)
    # the textbook value at the unit square corner, as a check of the closed form itself
    assert abs(_corner_ff(1.0, 1.0) - (1 / np.pi) * np.sqrt(0.5) * np.arctan(np.sqrt(0.5))) < 1e-15


def test_glass_in_furnace_carries_exactly_one(oracle_lib):
    sc = oracle_lib.Scene.from_dict(scenes.glass_in_furnace())
    n = 20000
    rng = np.random.default_rng(5)
    o = np.tile([0.0, 0.0, 1.5], (n, 1))
    tgt = rng.uniform(-0.3, 0.3, size=(n, 3)) * np.array([1, 1, 0])
    d = tgt - o
    # total internal reflection can trap a path inside the faceted sphere for a while: give it
    # enough vertices to escape; every escaping path then carries exactly Le = 1
    L, _ = sc.trace_rays(o, d, np.arange(n), max_depth=1024)
    assert np.allclose(L, 1.0, rtol=0, atol=1e-12)
    L64, _ = sc.trace_rays(o, d, np.arange(n), max_depth=64)
    ok = L64[:, 0] > 0
    assert ok.mean() > 0.995 and np.allclose(L64[ok], 1.0, rtol=0, atol=1e-12)


def test_dual_matches_central_differences(oracle_lib):
    s = scenes.box_scene(width=16, height=16)
    # mix in a GGX and a glass material so every BSDF's derivative is exercised
    s["mat_type"] = s["mat_type"].copy()
    s["mat_type"][5] = 1
    s["mat_roughness"] = s["mat_roughness"].copy()
    s["mat_roughness"][5] = 0.3
    s["mat_type"][6] = 2
    s["mat_albedo"][6] = [0.9, 0.95, 1.0]
    sc = oracle_lib.Scene.from_dict(s)
    cam = s["camera"]
    nm = len(s["mat_type"])
    rng = np.random.default_rng(11)
    da = np.zeros((3, nm, 3))
    de = np.zeros((3, nm))
    da[0, 2] = [1.0, 0.0, 0.0]              # one channel of the back wall
    da[1, 5] = [0.0, 1.0, 0.0]              # one channel of the GGX box
    da[1, 6] = [0.0, 0.0, 1.0]              # ...and the glass tint
    de[2, 7] = 1.0                          # the light's emission
    ids = np.arange(16 * 16 * 4)
    # parameters on a 2^-16 grid and a power-of-two step keep theta +- h exact in FP32
    A0 = (np.round(s["mat_albedo"].astype(np.float64) * 2 ** 16) / 2 ** 16).astype(np.float32)
    E0 = s["mat_emission"].astype(np.float32)
    sc.set_materials(A0, E0)
    out = sc.render_paths(cam, 4, 6, 99, ids, rr_start=2, rr_fixed=0.8, dir_albedo=da, dir_emission=de)
    for k in range(3):
        h = 2.0 ** -10
        Ap = (A0 + h * da[k]).astype(np.float32)
        Am = (A0 - h * da[k]).astype(np.float32)
        Ep = (E0 + 32 * h * de[k]).astype(np.float32)
        Em = (E0 - 32 * h * de[k]).astype(np.float32)
        assert np.array_equal(Ap.astype(np.float64) - Am, 2 * h * da[k])
        assert np.array_equal(Ep.astype(np.float64) - Em, 64 * h * de[k])
        step = 2 * h if k < 2 else 64 * h
        sc.set_materials(Ap, Ep)
        Lp = sc.render_paths(cam, 4, 6, 99, ids, rr_start=2, rr_fixed=0.8)["L"]
        sc.set_materials(Am, Em)
        Lm = sc.render_paths(cam, 4, 6, 99, ids, rr_start=2, rr_fixed=0.8)["L"]
        sc.set_materials(A0, E0)
        fd = (Lp - Lm).sum(0) / step
        ad = out["dL"][:, k, :].sum(0)
        assert np.allclose(fd, ad, rtol=1e-5, atol=1e-9 * np.abs(ad).max()), (k, fd, ad)
        assert np.abs(ad).max() > 0


def test_image_is_mean_of_paths_and_bvh_is_exact(oracle_lib):
    s = scenes.box_scene(width=12, height=10)
    sc = oracle_lib.Scene.from_dict(s)
    cam = s["camera"]
    spp = 3
    img, rays = sc.render_pixels(cam, spp, 8, 5, rr_start=3)
    paths = sc.render_paths(cam, spp, 8, 5, np.arange(12 * 10 * spp), rr_start=3)
    acc = np.zeros((120, 3))
    for smp in range(spp):
        acc += paths["L"][smp::spp]
    assert np.array_equal(img, acc / spp)
    assert np.array_equal(rays, paths["rays"])
    brute = sc.render_paths(cam, spp, 8, 5, np.arange(12 * 10 * spp), rr_start=3, use_bvh=False)
    assert np.array_equal(brute["L"], paths["L"]) and np.array_equal(brute["sig"], paths["sig"])
    assert img.max() > 0


def test_degenerate_cases(oracle_lib):
    s = scenes.box_scene(width=4, height=4)
    sc = oracle_lib.Scene.from_dict(s)
    # max_depth 0: nothing traced
    img, rays = sc.render_pixels(s["camera"], 2, 0, 1)
    assert np.all(img == 0) and rays.sum() == 0
    # max_depth 1: emission seen directly only (camera sees the light from below in some pixels)
    img1, rays1 = sc.render_pixels(s["camera"], 2, 1, 1)
    assert rays1[1] == 0
    # empty scene: every camera ray misses and returns the environment
    e = dict(s)
    e.update(verts=np.zeros((0, 3), np.float32), tris=np.zeros((0, 3), np.uint32),
             tri_mat=np.zeros(0, np.uint32), env=np.array([0.25, 0.5, 1.0], np.float32))
    sce = oracle_lib.Scene.from_dict(e)
    img2, rays2 = sce.render_pixels(s["camera"], 2, 5, 1)
    assert np.all(img2 == np.array([0.25, 0.5, 1.0])) and rays2[0] == 32
    assert sce.n_lights == 0
