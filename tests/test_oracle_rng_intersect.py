"""Oracle pins: the counter-based random numbers and ray/triangle intersection.

The random-number definition (PCG hash of Jarzynski & Olano, JCGT 2020) has no printed test
vectors, so it is pinned by properties a slip would break: bijectivity (the LCG step and the
RXS-M-XS permutation are both invertible; an even multiplier or a wrong shift breaks that),
avalanche, range/exactness of the 24-bit uniform, uniformity and independence across dims.
Intersection is pinned by closed-form hits and by brute force (exact ids and t).
"""
import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes


def test_pcg_hash_is_bijective_on_a_block(oracle_lib):
    import ctypes
    L = oracle_lib.lib()
    n = 1 << 18
    base = 0x1234567
    out = np.fromiter((L.or_pcg_hash(ctypes.c_uint32(base + i)) for i in range(n)), np.uint32, n)
    assert np.unique(out).size == n


def test_pcg_hash_avalanche(oracle_lib):
    rng = np.random.default_rng(1)
    xs = rng.integers(0, 1 << 32, size=2000, dtype=np.uint64)
    flips = []
    for x in xs:
        h = oracle_lib.pcg_hash(int(x))
        for bit in (0, 7, 16, 31):
            h2 = oracle_lib.pcg_hash(int(x) ^ (1 << bit))
            flips.append(bin(h ^ h2).count("1"))
    assert 14.5 < np.mean(flips) < 17.5


def test_u01_range_exact_and_uniform(oracle_lib):
    n = 200_000
    px = np.arange(n) % 5000
    sm = np.arange(n) // 5000
    u = oracle_lib.u01(7, px, sm, 2, 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    k = u * 2.0 ** 24
    assert np.all(k == np.floor(k))                     # 24-bit grid: exact in FP32 too
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    hist = np.histogram(u, bins=64, range=(0, 1))[0]
    exp = n / 64
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 120                                   # 63 dof: p ~ 1e-5 threshold


def test_u01_dims_bounces_seeds_independent(oracle_lib):
    n = 100_000
    px = np.arange(n)
    base = oracle_lib.u01(0, px, 0, 0, 0)
    for (seed, b, d) in [(0, 0, 1), (0, 1, 0), (1, 0, 0), (0, 3, 8)]:
        other = oracle_lib.u01(seed, px, 0, b, d)
        assert abs(np.corrcoef(base, other)[0, 1]) < 0.015
    # neighbouring pixels and samples decorrelated
    nb = oracle_lib.u01(0, px + 1, 0, 0, 0)
    assert abs(np.corrcoef(base, nb)[0, 1]) < 0.015
    s1 = oracle_lib.u01(0, px, 1, 0, 0)
    assert abs(np.corrcoef(base, s1)[0, 1]) < 0.015


def _one_tri_scene(tris_xyz):
    V = np.asarray(tris_xyz, np.float32).reshape(-1, 3)
    T = np.arange(V.shape[0]).reshape(-1, 3)
    n = T.shape[0]
    return dict(verts=V, tris=T, tri_mat=np.zeros(n), mat_type=[0], mat_albedo=[[0.5] * 3],
                mat_emission=[0.0], mat_roughness=[0.5], mat_ior=[1.5], env=[0, 0, 0])


@pytest.mark.parametrize("use_bvh", [False, True])
def test_intersection_closed_form(oracle_lib, use_bvh):
    sc = oracle_lib.Scene.from_dict(_one_tri_scene([(0, 0, 0), (1, 0, 0), (0, 1, 0)]))
    o = [[0.25, 0.25, 1.0], [0.25, 0.25, -2.0], [0.6, 0.6, 1.0], [0.0, 0.0, 1.0], [0.5, 0.5, 3.0],
         [0.25, 0.25, 0.0]]
    d = [[0, 0, -1], [0, 0, 1], [0, 0, -1], [0, 0, -1], [0, 0, -1], [0, 0, -1]]
    t, prim, u, v = sc.intersect(o, d, use_bvh)
    assert prim[0] == 0 and t[0] == 1.0 and u[0] == 0.25 and v[0] == 0.25
    assert prim[1] == 0 and t[1] == 2.0                 # two-sided: hit from behind
    assert prim[2] == -1                                # u + v = 1.2 > 1
    assert prim[3] == 0 and u[3] == 0.0 and v[3] == 0.0  # vertex: inclusive bounds
    assert prim[4] == 0 and t[4] == 3.0 and u[4] + v[4] == 1.0  # hypotenuse: inclusive
    assert prim[5] == -1                                # t = 0 is not a hit (t > 0)


def test_intersection_tie_goes_to_lower_id(oracle_lib):
    tri = [(0, 0, 0), (1, 0, 0), (0, 1, 0)]
    sc = oracle_lib.Scene.from_dict(_one_tri_scene(tri + tri + [(0, 0, 0.5), (1, 0, 0.5), (0, 1, 0.5)]))
    t, prim, _, _ = sc.intersect([[0.2, 0.2, -1.0], [0.2, 0.2, 1.0]], [[0, 0, 1], [0, 0, -1]])
    assert prim[0] == 0 and t[0] == 1.0     # duplicates 0 and 1 tie at t = 1 -> id 0
    assert prim[1] == 2 and t[1] == 0.5


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bvh_matches_brute_force(oracle_lib, seed):
    sc = oracle_lib.Scene.from_dict(scenes.random_soup(n_tris=3000, seed=seed))
    o, d = scenes.random_rays(20000, seed=seed + 10)
    t0, p0, u0, v0 = sc.intersect(o, d, use_bvh=False)
    t1, p1, u1, v1 = sc.intersect(o, d, use_bvh=True)
    assert np.array_equal(p0, p1)
    assert np.array_equal(t0, t1)
    assert (p0 >= 0).mean() > 0.3
    tmax = np.where(p0 >= 0, t0 * 0.999, 5.0)
    tmax = np.where(np.arange(len(tmax)) % 2 == 0, tmax, 1.7)
    assert np.array_equal(sc.occluded(o, d, tmax, False), sc.occluded(o, d, tmax, True))


def test_bvh_matches_brute_force_on_box_scene(oracle_lib):
    s = scenes.box_scene()
    sc = oracle_lib.Scene.from_dict(s)
    rng = np.random.default_rng(3)
    o = rng.uniform([-0.95, 0.05, -0.95], [0.95, 1.95, 0.95], size=(20000, 3))
    d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t0, p0, _, _ = sc.intersect(o, d, use_bvh=False)
    t1, p1, _, _ = sc.intersect(o, d, use_bvh=True)
    assert np.array_equal(p0, p1) and np.array_equal(t0, t1)


def test_scene_generators_winding_and_counts():
    s = scenes.box_scene()
    assert s["tris"].shape[0] == 36
    V, T = scenes.icosphere(2)
    assert T.shape[0] == 320
    c = V[T].mean(axis=1)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    assert np.all((n * c).sum(1) > 0)                 # outward winding
    # light faces down
    lt = s["tri_mat"] == 7
    V, T = s["verts"], s["tris"][lt]
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    assert np.all(n[:, 1] < 0)
    a = scenes.spheres_scene(seed=0, n_spheres=3, level=1, ground_quads=4)
    b = scenes.spheres_scene(seed=0, n_spheres=3, level=1, ground_quads=4)
    assert np.array_equal(a["verts"], b["verts"])     # seeded and deterministic
