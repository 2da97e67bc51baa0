"""Pins of the oracle's two-level (instanced) scenes: instances are placed in the world in FP64
(world = R v + t), triangle ids run over the instances in order, and an instance material replaces
its mesh's triangle materials.

* a flat scene cut into meshes placed by exact transforms (axis sign flips times powers of
  two) renders exactly like the flat scene: same images and branch signatures, path by path;
* the white furnace placed by a rotated, scaled instance keeps its closed-form series;
* direct light from a unit-square light mesh scaled non-uniformly into the rectangle keeps the
  point-to-rectangle form factor (the light's world area enters the light pdf);
* an instance material is what the flattened triangles carry.
"""
import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes
from test_oracle_estimator import _point_ff, _rows, _sphere_rays


@pytest.mark.parametrize("which", ["box", "spheres"])
def test_exactly_placed_instances_equal_the_flat_scene(oracle_lib, which):
    if which == "box":
        sc = scenes.box_scene(seed=0, width=24, height=16)
    else:
        sc = scenes.spheres_scene(seed=1, n_spheres=20, level=2, ground_quads=16, extent=10.0, width=32, height=18)
    flat = oracle_lib.Scene.from_dict(sc)
    inst = oracle_lib.Scene.from_dict(scenes.split_as_instances(sc, 7, seed=2))
    assert inst.n_tris == flat.n_tris and inst.n_lights == flat.n_lights
    cam = sc["camera"]
    n = cam["width"] * cam["height"] * 2
    a = flat.render_paths(cam, 2, 6, 9, np.arange(n))
    b = inst.render_paths(cam, 2, 6, 9, np.arange(n))
    assert np.array_equal(a["L"], b["L"]) and np.array_equal(a["sig"], b["sig"])


def _rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _as_single_instance(sc, R, scale, t):
    X = np.zeros((1, 3, 4))
    X[0, :, :3] = R * scale
    X[0, :, 3] = t
    d = {k: sc[k] for k in ("mat_type", "mat_albedo", "mat_emission", "mat_roughness", "mat_ior", "env")}
    d.update(meshes=[{"verts": sc["verts"], "tris": sc["tris"], "tri_mat": sc["tri_mat"]}],
             inst_mesh=np.zeros(1, np.uint32), inst_xform=X.astype(np.float32),
             inst_mat=np.full(1, scenes.NO_MATERIAL, np.uint32))
    return d


@pytest.mark.parametrize("a,D,expect", [tuple(r) for r in _rows("furnace.txt")][:3])
def test_rotated_scaled_furnace_keeps_the_series(oracle_lib, a, D, expect):
    s = scenes.furnace_sphere(albedo=a, emission=1.0, level=4)
    t = np.array([3.0, -1.5, 0.25])
    sc = oracle_lib.Scene.from_dict(_as_single_instance(s, _rotation(3), 2.5, t))
    o, d = _sphere_rays(20000, 6)
    L, _ = sc.trace_rays(o * 2.5 + t, d, np.arange(20000), max_depth=int(D))
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(len(L))
    assert abs(m - expect) < 3 * se + 2e-3 * expect, (m, se, expect)


@pytest.mark.parametrize("px,pz,hw,hh,c", [tuple(r) for r in _rows("form_factor_parallel_rect.txt")][:4])
def test_scaled_light_instance_keeps_the_form_factor(oracle_lib, px, pz, hw, hh, c):
    rho, Le = 0.7, 5.0
    flat = scenes.rect_over_plane(albedo=rho, emission=Le, half_w=hw, half_h=hh, height=c)
    # the plane as one mesh (identity); the light as a unit square (half-size 1, facing -y at y = 0)
    # placed by the non-uniform scale (hw, 1, hh) and the translation (0, c, 0)
    plane_v = flat["verts"][:4]
    unit_v, unit_t = scenes.quad((-1, 0, -1), (1, 0, -1), (1, 0, 1), (-1, 0, 1))
    X = np.zeros((2, 3, 4), np.float32)
    X[0, :, :3] = np.eye(3)
    X[1, :, :3] = np.diag([hw, 1.0, hh])
    X[1, :, 3] = [0.0, c, 0.0]
    d = {k: flat[k] for k in ("mat_type", "mat_albedo", "mat_emission", "mat_roughness", "mat_ior", "env")}
    d.update(meshes=[{"verts": plane_v, "tris": flat["tris"][:2], "tri_mat": flat["tri_mat"][:2]},
                     {"verts": unit_v, "tris": unit_t, "tri_mat": np.ones(2, np.uint32)}],
             inst_mesh=np.array([0, 1], np.uint32), inst_xform=X,
             inst_mat=np.full(2, scenes.NO_MATERIAL, np.uint32))
    sc = oracle_lib.Scene.from_dict(d)
    assert abs(sc.light_area - 4 * hw * hh) < 1e-6 * hw * hh
    n = 100_000
    L, _ = sc.trace_rays(np.tile([px, 0.5 * c, pz], (n, 1)), np.tile([0.0, -1.0, 0.0], (n, 1)), np.arange(n),
                         max_depth=2)
    expect = rho * Le * _point_ff(px, pz, hw, hh, c)
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(n)
    assert abs(m - expect) < 4 * se + 1e-4 * expect, (m, se, expect)


def test_instance_material_replaces_the_mesh_materials(oracle_lib):
    s = scenes.furnace_sphere(albedo=0.5, emission=1.0, level=2)
    d = _as_single_instance(s, np.eye(3), 1.0, np.zeros(3))
    # a second material (albedo 0.25, same emission) assigned by the instance
    for k in ("mat_type", "mat_albedo", "mat_emission", "mat_roughness", "mat_ior"):
        d[k] = np.concatenate([np.asarray(s[k]), np.asarray(s[k])])
    d["mat_albedo"] = np.asarray(d["mat_albedo"], np.float32).copy()
    d["mat_albedo"][1] = 0.25
    d["inst_mat"] = np.array([1], np.uint32)
    sc = oracle_lib.Scene.from_dict(d)
    o, dd = _sphere_rays(20000, 8)
    L, _ = sc.trace_rays(o, dd, np.arange(20000), max_depth=3)
    expect = 1 + 0.25 + 0.25 ** 2
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(len(L))
    assert abs(m - expect) < 3 * se + 2e-3 * expect, (m, se, expect)
