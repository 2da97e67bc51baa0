"""Seeded synthetic scene generators.

This module is the one input source that both the CUDA path and the FP64 oracle consume: it
builds triangle soups, material tables and cameras as plain numpy arrays, and contains none of
the estimator's arithmetic (no sampling, shading or intersection).  Every generator is a pure
function of its seed.

The paper benchmarks a Khronos glTF sample scene that is not available here (Sec. 4); the
procedural scenes below stand in for it:

* ``box_scene``     -- tiny closed-ish box: 5 walls (10 tris), two axis-aligned boxes (24 tris),
                       a 2-triangle ceiling light with emission 15; 128x128, 16 spp, depth 8.
* ``spheres_scene`` -- 200 level-4 icospheres (5,120 tris each, radii lognormal(0, 0.5)) resting
                       on a 256x256-quad ground (the spheres cover its central 56%, the camera looks
                       down so geometry fills most of the frame); 60% Lambert / 30% GGX / 10% glass;
                       8 emissive quads
                       plus a constant environment; 1920x1080, 1 spp, depth 5.
* ``terrain_scene`` -- 2048x2048 fBm heightfield plus 5000 level-2 icospheres, 64 emissive quads;
                       3840x2160, 4 spp, depth 8.
* ``batch_scenes``  -- 64 scenes with lognormal triangle counts in [1k, 2M], resolutions from
                       {256^2, 512^2, 1280x720, 1920x1080} and spp from {1, 4, 16}.
* small fixtures for the closed-form checks (furnace enclosure, rectangle over a plane, glass
  inside a furnace, random triangle soups).

A scene is a dict of arrays: verts (V,3) f32, tris (T,3) u32, tri_mat (T,) u32, mat_type (M,)
u32 (0 Lambert, 1 GGX conductor, 2 smooth dielectric), mat_albedo (M,3) f32, mat_emission (M,)
f32, mat_roughness (M,) f32, mat_ior (M,) f32, env (3,) f32; and a camera dict with eye, target,
up, vfov_deg, width, height.

An instanced scene (two-level: meshes placed by instances) replaces verts/tris/tri_mat with
meshes: a list of {verts, tris, tri_mat} in object space, and inst_mesh (I,) u32, inst_xform
(I,3,4) f32 (object-to-world [R | t]: world = R v + t), inst_mat (I,) u32 (a material for every
triangle of the instance, or NO_MATERIAL to keep the mesh's).  Its triangle ids run over the
instances in order, each mesh's triangles in order.

* ``instanced_spheres_scene`` / ``instanced_terrain_scene`` -- the spheres and terrain recipes with
  one icosphere mesh (and one light quad) placed by instances;
* ``split_as_instances`` -- any flat scene cut into meshes placed by exact transforms (axis sign
  flips times powers of two), so that the instanced scene is the flat one exactly.
"""
from __future__ import annotations

import numpy as np

LAMBERT, GGX, DIELECTRIC = 0, 1, 2
NO_MATERIAL = 0xFFFFFFFF


# ------------------------------------------------------------------ geometry helpers
def quad(p0, p1, p2, p3):
    """Two triangles (p0,p1,p2), (p0,p2,p3); the winding normal is (p1-p0) x (p2-p0)."""
    v = np.array([p0, p1, p2, p3], np.float64)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int64)
    return v, t


def box_mesh(lo, hi, outward=True):
    """Axis-aligned box, 12 triangles, normals outward (or inward)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    faces = [  # each face listed counter-clockwise seen from outside
        [(x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)],  # +z
        [(x1, y0, z0), (x0, y0, z0), (x0, y1, z0), (x1, y1, z0)],  # -z
        [(x1, y0, z1), (x1, y0, z0), (x1, y1, z0), (x1, y1, z1)],  # +x
        [(x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0)],  # -x
        [(x0, y1, z1), (x1, y1, z1), (x1, y1, z0), (x0, y1, z0)],  # +y
        [(x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)],  # -y
    ]
    vs, ts = [], []
    for k, f in enumerate(faces):
        v, t = quad(*f)
        if not outward:
            t = t[:, ::-1]
        vs.append(v)
        ts.append(t + 4 * k)
    return np.concatenate(vs), np.concatenate(ts)


_ICO_CACHE: dict = {}


def icosphere(level: int):
    """Unit icosphere: an icosahedron subdivided `level` times (20 * 4^level triangles), outward
    winding."""
    if level in _ICO_CACHE:
        v, t = _ICO_CACHE[level]
        return v.copy(), t.copy()
    g = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0), (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    t = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    tris = list(t)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nt = []
        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nt += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = nt
    V = np.array(verts, np.float64)
    T = np.array(tris, np.int64)
    _ICO_CACHE[level] = (V, T)
    return V.copy(), T.copy()


def grid_mesh(n, x0, x1, z0, z1, height=None):
    """n x n quads on y = height(x, z) (or 0), 2 n^2 triangles, normals +y."""
    xs = np.linspace(x0, x1, n + 1)
    zs = np.linspace(z0, z1, n + 1)
    X, Z = np.meshgrid(xs, zs, indexing="xy")
    Y = np.zeros_like(X) if height is None else height(X, Z)
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    a = (j * (n + 1) + i).ravel()
    b = a + 1
    c = a + (n + 1) + 1
    d = a + (n + 1)
    # (a, d, c) and (a, c, b): winding normal +y for x to the right, z toward the viewer
    T = np.concatenate([np.stack([a, d, c], 1), np.stack([a, c, b], 1)])
    return V, T


class _Builder:
    def __init__(self):
        self.v, self.t, self.m = [], [], []
        self.nv = 0

    def add(self, V, T, mat):
        self.v.append(np.asarray(V, np.float64))
        self.t.append(np.asarray(T, np.int64) + self.nv)
        self.m.append(np.full(len(T), mat, np.int64))
        self.nv += len(V)

    def arrays(self):
        V = np.concatenate(self.v).astype(np.float32) if self.v else np.zeros((0, 3), np.float32)
        T = np.concatenate(self.t).astype(np.uint32) if self.t else np.zeros((0, 3), np.uint32)
        M = np.concatenate(self.m).astype(np.uint32) if self.m else np.zeros((0,), np.uint32)
        return V, T, M


def _materials(types, albedo, emission, roughness, ior):
    n = len(types)
    return {
        "mat_type": np.asarray(types, np.uint32).reshape(n),
        "mat_albedo": np.asarray(albedo, np.float32).reshape(n, 3),
        "mat_emission": np.asarray(emission, np.float32).reshape(n),
        "mat_roughness": np.asarray(roughness, np.float32).reshape(n),
        "mat_ior": np.asarray(ior, np.float32).reshape(n),
    }


def camera(eye, target, up=(0, 1, 0), vfov_deg=45.0, width=128, height=128):
    return {"eye": np.asarray(eye, np.float32), "target": np.asarray(target, np.float32),
            "up": np.asarray(up, np.float32), "vfov_deg": float(vfov_deg), "width": int(width),
            "height": int(height)}


def _scene(b: _Builder, mats: dict, env, **extra):
    V, T, M = b.arrays()
    sc = {"verts": V, "tris": T, "tri_mat": M, "env": np.asarray(env, np.float32)}
    sc.update(mats)
    sc.update(extra)
    return sc


# ------------------------------------------------------------------ instanced scenes
def _instanced(meshes, inst_mesh, inst_xform, inst_mat, mats, env, **extra):
    sc = {"meshes": [{"verts": np.asarray(m[0], np.float32).reshape(-1, 3),
                      "tris": np.asarray(m[1], np.uint32).reshape(-1, 3),
                      "tri_mat": np.asarray(m[2], np.uint32).reshape(-1)} for m in meshes],
          "inst_mesh": np.asarray(inst_mesh, np.uint32).reshape(-1),
          "inst_xform": np.asarray(inst_xform, np.float32).reshape(-1, 3, 4),
          "inst_mat": np.asarray(inst_mat, np.uint32).reshape(-1),
          "env": np.asarray(env, np.float32)}
    sc.update(mats)
    sc.update(extra)
    return sc


def _xform(scale=1.0, translate=(0.0, 0.0, 0.0), R=None):
    M = np.zeros((3, 4))
    M[:, :3] = (np.eye(3) if R is None else np.asarray(R, np.float64)) * np.asarray(scale, np.float64)
    M[:, 3] = translate
    return M


def instance_tri_count(sc) -> int:
    return int(sum(len(sc["meshes"][m]["tris"]) for m in sc["inst_mesh"]))


def split_as_instances(sc: dict, n_pieces: int = 5, seed: int = 0) -> dict:
    """The flat scene `sc` cut into n_pieces meshes (contiguous triangle ranges), each stored in its
    own object frame and placed back by an exact transform: axis sign flips times a power of two
    (world = 2^k S v, object vertices 2^-k S v, both exact in FP32; no axis permutation, so every
    sum and product is formed in the same order as in world space).  Triangle ids, materials and
    world geometry equal the flat scene's."""
    rng = np.random.default_rng(seed)
    V, T, M = np.asarray(sc["verts"], np.float32), np.asarray(sc["tris"]), np.asarray(sc["tri_mat"])
    cuts = np.linspace(0, len(T), n_pieces + 1).round().astype(int)
    meshes, xf = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        used, inv = np.unique(T[a:b].ravel(), return_inverse=True)
        P = np.diag(rng.choice([-1.0, 1.0], size=3))
        k = int(rng.integers(-3, 4))
        obj = ((V[used].astype(np.float64) @ P) * 2.0 ** (-k)).astype(np.float32)   # P^T v, row form
        meshes.append((obj, inv.reshape(-1, 3), M[a:b]))
        xf.append(_xform(2.0 ** k, (0.0, 0.0, 0.0), P))
    mats = {k: sc[k] for k in ("mat_type", "mat_albedo", "mat_emission", "mat_roughness", "mat_ior")}
    extra = {k: v for k, v in sc.items() if k in ("camera", "spp", "max_depth", "rr_start", "rr_fixed")}
    return _instanced(meshes, np.arange(len(meshes)), xf, np.full(len(meshes), NO_MATERIAL), mats, sc["env"],
                      **extra)


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def instanced_spheres_scene(seed: int = 0, n_spheres=200, level=4, ground_quads=256, n_lights=8, width=1920,
                            height=1080, extent=60.0, rotate=True, n_materials=None):
    """The spheres recipe with one icosphere mesh placed by n_spheres instances (randomly rotated,
    uniformly scaled by lognormal(0, 0.5) radii, resting on the ground, one material each), the
    ground as one mesh and one light quad mesh placed by n_lights translated instances."""
    rng = np.random.default_rng(seed)
    S, ST = icosphere(level)
    radii = rng.lognormal(0.0, 0.5, size=n_spheres)
    cx = rng.uniform(-0.7 * extent, 0.7 * extent, size=n_spheres)
    cz = rng.uniform(-0.7 * extent, 0.7 * extent, size=n_spheres)
    n_sph_mats = n_spheres if n_materials is None else n_materials - 2
    sph_mat = np.arange(n_spheres) if n_materials is None else rng.integers(0, n_sph_mats, size=n_spheres)
    types, albedo, rough = _mix_materials(rng, n_sph_mats)
    ground_mat, light_mat = n_sph_mats, n_sph_mats + 1
    g = 2.5 * extent
    GV, GT = grid_mesh(ground_quads, -g, g, -g, g)
    h = 3.0
    LV, LT = quad((-h, 0.0, -h), (h, 0.0, -h), (h, 0.0, h), (-h, 0.0, h))
    meshes = [(S, ST, np.zeros(len(ST))), (GV, GT, np.full(len(GT), ground_mat)), (LV, LT, np.full(len(LT), light_mat))]
    im, ix, imat = [], [], []
    for k in range(n_spheres):
        im.append(0)
        ix.append(_xform(radii[k], (cx[k], radii[k], cz[k]), _rotation(rng) if rotate else None))
        imat.append(sph_mat[k])
    im.append(1)
    ix.append(_xform())
    imat.append(NO_MATERIAL)
    for k in range(n_lights):
        ang = 2 * np.pi * k / n_lights
        im.append(2)
        ix.append(_xform(1.0, (0.45 * extent * np.cos(ang), 25.0, 0.45 * extent * np.sin(ang))))
        imat.append(NO_MATERIAL)
    types = np.concatenate([types, [LAMBERT, LAMBERT]])
    albedo = np.concatenate([albedo, [[0.5, 0.5, 0.5], [0.8, 0.8, 0.8]]])
    rough = np.concatenate([rough, [0.5, 0.5]])
    emission = np.zeros(len(types))
    emission[light_mat] = 15.0
    mats = _materials(types, albedo, emission, rough, np.full(len(types), 1.5))
    cam = camera((0.0, 0.5 * extent, 0.95 * extent), (0.0, 0.0, -0.1 * extent), (0, 1, 0), 50.0, width, height)
    return _instanced(meshes, im, ix, imat, mats, (0.1, 0.1, 0.1), camera=cam, spp=1, max_depth=5, rr_start=3)


def instanced_terrain_scene(seed: int = 0, grid=2048, n_spheres=5000, level=2, n_lights=64, width=3840,
                            height=2160, extent=200.0, relief=12.0, tiles=1):
    """The terrain recipe with real instancing: the heightfield as one mesh (or tiles x tiles meshes
    of contiguous quads), one level-2 icosphere mesh placed by n_spheres instances (uniform scale,
    translation, one of 253 materials each) and one light quad mesh placed by n_lights instances."""
    rng = np.random.default_rng(seed)
    h = fbm(rng)
    scale = (grid - 1) / (2 * extent)

    def height_fn(X, Z):
        return relief * h(X * scale, Z * scale)

    GV, GT = grid_mesh(grid - 1, -extent, extent, -extent, extent, height_fn)
    n_sph_mats = 253
    types, albedo, rough = _mix_materials(rng, n_sph_mats)
    ground_mat, light_mat = n_sph_mats, n_sph_mats + 1
    S, ST = icosphere(level)
    radii = rng.lognormal(0.0, 0.5, size=n_spheres)
    cx = rng.uniform(-0.9 * extent, 0.9 * extent, size=n_spheres)
    cz = rng.uniform(-0.9 * extent, 0.9 * extent, size=n_spheres)
    cy = height_fn(cx, cz) + radii
    smat = rng.integers(0, n_sph_mats, size=n_spheres)
    hh = 4.0
    LV, LT = quad((-hh, 0.0, -hh), (hh, 0.0, -hh), (hh, 0.0, hh), (-hh, 0.0, hh))
    meshes = [(S, ST, np.zeros(len(ST))), (LV, LT, np.full(len(LT), light_mat))]
    im, ix, imat = [], [], []
    # terrain tiles: quads (i, j) with i, j in a tile's range; both triangles of a quad stay together
    n = grid - 1
    qi = np.concatenate([np.arange(n * n), np.arange(n * n)]) % n          # quad column of each triangle
    qj = np.concatenate([np.arange(n * n), np.arange(n * n)]) // n         # quad row
    edges = np.linspace(0, n, tiles + 1).round().astype(int)
    for tj in range(tiles):
        for ti in range(tiles):
            sel = np.flatnonzero((qi >= edges[ti]) & (qi < edges[ti + 1]) & (qj >= edges[tj]) & (qj < edges[tj + 1]))
            used, inv = np.unique(GT[sel].ravel(), return_inverse=True)
            meshes.append((GV[used], inv.reshape(-1, 3), np.full(len(sel), ground_mat)))
            im.append(len(meshes) - 1)
            ix.append(_xform())
            imat.append(NO_MATERIAL)
    for k in range(n_spheres):
        im.append(0)
        ix.append(_xform(radii[k], (cx[k], cy[k], cz[k])))
        imat.append(smat[k])
    side = int(round(np.sqrt(n_lights)))
    for k in range(n_lights):
        i, j = k % side, k // side
        x = -0.8 * extent + 1.6 * extent * (i + 0.5) / side
        z = -0.8 * extent + 1.6 * extent * (j + 0.5) / side
        im.append(1)
        ix.append(_xform(1.0, (x, 60.0, z)))
        imat.append(NO_MATERIAL)
    types = np.concatenate([types, [LAMBERT, LAMBERT]])
    albedo = np.concatenate([albedo, [[0.45, 0.4, 0.35], [0.8, 0.8, 0.8]]])
    rough = np.concatenate([rough, [0.5, 0.5]])
    emission = np.zeros(len(types))
    emission[light_mat] = 15.0
    matd = _materials(types, albedo, emission, rough, np.full(len(types), 1.5))
    cam = camera((0.0, 0.45 * extent, 1.1 * extent), (0.0, 0.0, 0.0), (0, 1, 0), 55.0, width, height)
    return _instanced(meshes, im, ix, imat, matd, (0.1, 0.1, 0.1), camera=cam, spp=4, max_depth=8, rr_start=3)


# ------------------------------------------------------------------ benchmark scenes
def box_scene(seed: int = 0, width=128, height=128, lift=0.0):
    """Tiny box: 5 walls + two axis-aligned boxes + a 2-triangle ceiling light (36 tris).  `lift`
    raises both boxes off the floor (their bottoms are coplanar with it when 0)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    # walls (inward normals): x in [-1,1], y in [0,2], z in [-1,1], open toward +z
    walls = [
        [(-1, 0, -1), (-1, 0, 1), (1, 0, 1), (1, 0, -1)],      # floor, +y
        [(-1, 2, -1), (1, 2, -1), (1, 2, 1), (-1, 2, 1)],      # ceiling, -y
        [(-1, 0, -1), (1, 0, -1), (1, 2, -1), (-1, 2, -1)],    # back, +z
        [(-1, 0, -1), (-1, 2, -1), (-1, 2, 1), (-1, 0, 1)],    # left, +x
        [(1, 0, -1), (1, 0, 1), (1, 2, 1), (1, 2, -1)],        # right, -x
    ]
    n_surf = 7
    albedo = rng.uniform(0.1, 0.9, size=(n_surf + 1, 3))
    for k, w in enumerate(walls):
        b.add(*quad(*w), k)
    b.add(*box_mesh((-0.7, lift, -0.1), (-0.1, 0.6 + lift, 0.5)), 5)
    b.add(*box_mesh((0.1, lift, -0.7), (0.7, 1.2 + lift, -0.1)), 6)
    # light quad just below the ceiling, facing down
    b.add(*quad((-0.25, 1.98, -0.25), (0.25, 1.98, -0.25), (0.25, 1.98, 0.25), (-0.25, 1.98, 0.25)), 7)
    types = [LAMBERT] * (n_surf + 1)
    emission = [0.0] * n_surf + [15.0]
    mats = _materials(types, albedo, emission, [0.5] * (n_surf + 1), [1.5] * (n_surf + 1))
    cam = camera((0.0, 1.0, 3.4), (0.0, 1.0, 0.0), (0, 1, 0), 40.0, width, height)
    return _scene(b, mats, (0.0, 0.0, 0.0), camera=cam, spp=16, max_depth=8, rr_start=3)


def _mix_materials(rng, n, frac_lambert=0.6, frac_ggx=0.3):
    """Material mix of the procedural scenes: 60% Lambert albedo U[0.1,0.9]^3, 30% GGX conductor
    (F0 U[0.5,1]^3, roughness U[0.05,0.6]), 10% smooth dielectric (IOR 1.5, clear)."""
    u = rng.uniform(size=n)
    types = np.where(u < frac_lambert, LAMBERT, np.where(u < frac_lambert + frac_ggx, GGX, DIELECTRIC))
    albedo = rng.uniform(0.1, 0.9, size=(n, 3))
    f0 = rng.uniform(0.5, 1.0, size=(n, 3))
    albedo = np.where((types == GGX)[:, None], f0, albedo)
    albedo = np.where((types == DIELECTRIC)[:, None], 1.0, albedo)
    rough = rng.uniform(0.05, 0.6, size=n)
    return types, albedo, rough


def spheres_scene(seed: int = 0, n_spheres=200, level=4, ground_quads=256, n_lights=8,
                  width=1920, height=1080, n_materials=None, extent=60.0):
    """~1.15M-triangle procedural scene: icospheres on a ground plane, emissive quads, constant
    environment.  With n_materials = K (>= 3), spheres draw their material from K-2 shared
    materials, the ground uses material K-2 and the lights material K-1."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    S, ST = icosphere(level)
    radii = rng.lognormal(0.0, 0.5, size=n_spheres)
    cx = rng.uniform(-0.7 * extent, 0.7 * extent, size=n_spheres)
    cz = rng.uniform(-0.7 * extent, 0.7 * extent, size=n_spheres)
    if n_materials is None:
        n_sph_mats = n_spheres
        sph_mat = np.arange(n_spheres)
    else:
        n_sph_mats = n_materials - 2
        sph_mat = rng.integers(0, n_sph_mats, size=n_spheres)
    types, albedo, rough = _mix_materials(rng, n_sph_mats)
    ground_mat, light_mat = n_sph_mats, n_sph_mats + 1
    for k in range(n_spheres):
        b.add(S * radii[k] + np.array([cx[k], radii[k], cz[k]]), ST, sph_mat[k])
    g = 2.5 * extent
    GV, GT = grid_mesh(ground_quads, -g, g, -g, g)
    b.add(GV, GT, ground_mat)
    for k in range(n_lights):
        ang = 2 * np.pi * k / n_lights
        x, z = 0.45 * extent * np.cos(ang), 0.45 * extent * np.sin(ang)
        y, h = 25.0, 3.0
        b.add(*quad((x - h, y, z - h), (x + h, y, z - h), (x + h, y, z + h), (x - h, y, z + h)), light_mat)
    types = np.concatenate([types, [LAMBERT, LAMBERT]])
    albedo = np.concatenate([albedo, [[0.5, 0.5, 0.5], [0.8, 0.8, 0.8]]])
    rough = np.concatenate([rough, [0.5, 0.5]])
    emission = np.zeros(len(types))
    emission[light_mat] = 15.0
    mats = _materials(types, albedo, emission, rough, np.full(len(types), 1.5))
    cam = camera((0.0, 0.5 * extent, 0.95 * extent), (0.0, 0.0, -0.1 * extent), (0, 1, 0), 50.0, width, height)
    return _scene(b, mats, (0.1, 0.1, 0.1), camera=cam, spp=1, max_depth=5, rr_start=3)


def diff_scene(seed: int = 0, width=512, height=512):
    """Inverse-rendering workload: the procedural spheres geometry with 256 shared materials (254 on
    the spheres, the ground, the lights), 512x512, 64 spp, depth 6, roulette from bounce 3 with a
    fixed survival probability 0.9 (so that the estimator is smooth in the parameters)."""
    sc = spheres_scene(seed=seed, n_materials=256, width=width, height=height)
    sc.update(spp=64, max_depth=6, rr_start=3, rr_fixed=0.9)
    return sc


def diff_target(sc: dict, seed: int = 7):
    """Hidden target parameters for diff_scene: albedos redrawn per material type (Lambert
    U[0.1,0.9]^3, GGX F0 U[0.5,1]^3, dielectric tint unchanged) and emission scaled by U[0.7,1.3]."""
    rng = np.random.default_rng(seed)
    t = np.asarray(sc["mat_type"])
    n = len(t)
    alb = np.asarray(sc["mat_albedo"], np.float32).reshape(n, 3).copy()
    lam, ggx = t == LAMBERT, t == GGX
    alb[lam] = rng.uniform(0.1, 0.9, size=(int(lam.sum()), 3))
    alb[ggx] = rng.uniform(0.5, 1.0, size=(int(ggx.sum()), 3))
    em = np.asarray(sc["mat_emission"], np.float32).reshape(n) * rng.uniform(0.7, 1.3, size=n)
    return alb.astype(np.float32), em.astype(np.float32)


def _value_noise(rng, res=256):
    table = rng.uniform(-1.0, 1.0, size=(res, res))

    def noise(x, y):
        xi, yi = np.floor(x).astype(np.int64), np.floor(y).astype(np.int64)
        fx, fy = x - xi, y - yi
        sx, sy = fx * fx * (3 - 2 * fx), fy * fy * (3 - 2 * fy)
        a = table[yi % res, xi % res]
        b = table[yi % res, (xi + 1) % res]
        c = table[(yi + 1) % res, xi % res]
        d = table[(yi + 1) % res, (xi + 1) % res]
        return (a * (1 - sx) + b * sx) * (1 - sy) + (c * (1 - sx) + d * sx) * sy

    return noise


def fbm(rng, octaves=6, lacunarity=2.0, gain=0.5, base_freq=1.0 / 16.0):
    noise = _value_noise(rng)

    def f(x, z):
        amp, freq, acc = 1.0, base_freq, np.zeros_like(x)
        for _ in range(octaves):
            acc += amp * noise(x * freq, z * freq)
            amp *= gain
            freq *= lacunarity
        return acc

    return f


def terrain_scene(seed: int = 0, grid=2048, n_spheres=5000, level=2, n_lights=64, width=3840,
                  height=2160, extent=200.0, relief=12.0):
    """~10M-triangle scene: fBm heightfield (grid x grid vertices -> 2 (grid-1)^2 tris) plus
    icospheres flattened into one mesh, 64 emissive quads."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    h = fbm(rng)
    scale = (grid - 1) / (2 * extent)

    def height_fn(X, Z):
        return relief * h(X * scale, Z * scale)

    GV, GT = grid_mesh(grid - 1, -extent, extent, -extent, extent, height_fn)
    n_sph_mats = 253
    types, albedo, rough = _mix_materials(rng, n_sph_mats)
    ground_mat, light_mat = n_sph_mats, n_sph_mats + 1
    b.add(GV, GT, ground_mat)
    S, ST = icosphere(level)
    radii = rng.lognormal(0.0, 0.5, size=n_spheres)
    cx = rng.uniform(-0.9 * extent, 0.9 * extent, size=n_spheres)
    cz = rng.uniform(-0.9 * extent, 0.9 * extent, size=n_spheres)
    cy = height_fn(cx, cz) + radii
    mats = rng.integers(0, n_sph_mats, size=n_spheres)
    # one flattened mesh for all spheres
    SV = (S[None, :, :] * radii[:, None, None] + np.stack([cx, cy, cz], 1)[:, None, :]).reshape(-1, 3)
    STT = (ST[None, :, :] + (np.arange(n_spheres) * len(S))[:, None, None]).reshape(-1, 3)
    b.v.append(SV)
    b.t.append(STT + b.nv)
    b.m.append(np.repeat(mats, len(ST)))
    b.nv += len(SV)
    side = int(round(np.sqrt(n_lights)))
    for k in range(n_lights):
        i, j = k % side, k // side
        x = -0.8 * extent + 1.6 * extent * (i + 0.5) / side
        z = -0.8 * extent + 1.6 * extent * (j + 0.5) / side
        y, hh = 60.0, 4.0
        b.add(*quad((x - hh, y, z - hh), (x + hh, y, z - hh), (x + hh, y, z + hh), (x - hh, y, z + hh)), light_mat)
    types = np.concatenate([types, [LAMBERT, LAMBERT]])
    albedo = np.concatenate([albedo, [[0.45, 0.4, 0.35], [0.8, 0.8, 0.8]]])
    rough = np.concatenate([rough, [0.5, 0.5]])
    emission = np.zeros(len(types))
    emission[light_mat] = 15.0
    matd = _materials(types, albedo, emission, rough, np.full(len(types), 1.5))
    cam = camera((0.0, 0.45 * extent, 1.1 * extent), (0.0, 0.0, 0.0), (0, 1, 0), 55.0, width, height)
    return _scene(b, matd, (0.1, 0.1, 0.1), camera=cam, spp=4, max_depth=8, rr_start=3)


BATCH_RESOLUTIONS = [(256, 256), (512, 512), (1280, 720), (1920, 1080)]
BATCH_SPP = [1, 4, 16]


def batch_scenes(seed: int = 0, n=64, min_tris=1000, max_tris=2_000_000, resolutions=None, spps=None):
    """n independent scenes: triangle counts lognormal clipped to [min_tris, max_tris], each a
    spheres_scene variant sized to its count, with a resolution and spp drawn per scene."""
    rng = np.random.default_rng(seed)
    resolutions = BATCH_RESOLUTIONS if resolutions is None else resolutions
    spps = BATCH_SPP if spps is None else spps
    counts = np.clip(rng.lognormal(np.log(60_000), 1.4, size=n), min_tris, max_tris).astype(np.int64)
    out = []
    for k in range(n):
        target = int(counts[k])
        level = 3 if target >= 20_000 else 1          # 1280 or 80 tris per sphere
        per = 20 * 4 ** level
        gq = int(max(4, min(256, np.sqrt(target / 4))))  # ground gets ~half the budget
        n_sph = max(1, (target - 2 * gq * gq) // per)
        w, h = resolutions[int(rng.integers(0, len(resolutions)))]
        spp = int(spps[int(rng.integers(0, len(spps)))])
        sc = spheres_scene(seed=seed * 1000 + k + 1, n_spheres=int(n_sph), level=level, ground_quads=gq,
                           width=w, height=h, extent=20.0 + 0.02 * np.sqrt(target))
        sc["spp"] = spp
        out.append(sc)
    return out


# ------------------------------------------------------------------ closed-form fixtures
def furnace_sphere(albedo=0.5, emission=1.0, level=3, radius=1.0):
    """Closed icosphere with inward winding: every face is Lambert with the given albedo and
    emits `emission` toward the inside (all faces are lights).  Camera at the centre."""
    V, T = icosphere(level)
    b = _Builder()
    b.add(V * radius, T[:, ::-1], 0)
    mats = _materials([LAMBERT], [[albedo] * 3], [emission], [0.5], [1.5])
    cam = camera((0, 0, 0), (0, 0, -1), (0, 1, 0), 60.0, 16, 16)
    return _scene(b, mats, (0.0, 0.0, 0.0), camera=cam)


def rect_over_plane(albedo=0.7, emission=5.0, half_w=0.5, half_h=0.8, height=1.0, plane_half=10.0, fan=None):
    """Lambert plane y=0 (large) under a parallel emitting rectangle at y=height facing down,
    centred over the origin with half-sizes (half_w along x, half_h along z).

    fan=(fx, fz): the rectangle is cut into six triangles of very unequal area instead of two equal
    ones -- a fan around the interior point (fx * half_w, height, fz * half_h) through the four
    corners and the midpoints of the -z and +x edges.  The emitting region, hence the irradiance of
    the plane, is the same."""
    b = _Builder()
    b.add(*quad((-plane_half, 0, plane_half), (plane_half, 0, plane_half), (plane_half, 0, -plane_half),
                (-plane_half, 0, -plane_half)), 0)
    corners = [(-half_w, height, -half_h), (half_w, height, -half_h), (half_w, height, half_h),
               (-half_w, height, half_h)]
    if fan is None:
        b.add(*quad(*corners), 1)
    else:
        ring = [corners[0], (0.0, height, -half_h), corners[1], (half_w, height, 0.0), corners[2], corners[3]]
        V = np.array([(fan[0] * half_w, height, fan[1] * half_h)] + ring, np.float64)
        T = np.array([[0, 1 + k, 1 + (k + 1) % len(ring)] for k in range(len(ring))], np.int64)
        b.add(V, T, 1)
    mats = _materials([LAMBERT, LAMBERT], [[albedo] * 3, [0.0] * 3], [0.0, emission], [0.5, 0.5], [1.5, 1.5])
    return _scene(b, mats, (0.0, 0.0, 0.0))


def glass_in_furnace(ior=1.5, level_outer=3, level_inner=3, r_inner=0.4):
    """Inward-emitting black enclosure (albedo 0, emission 1) around a clear glass icosphere."""
    b = _Builder()
    V, T = icosphere(level_outer)
    b.add(V * 2.0, T[:, ::-1], 0)
    V2, T2 = icosphere(level_inner)
    b.add(V2 * r_inner, T2, 1)
    mats = _materials([LAMBERT, DIELECTRIC], [[0.0] * 3, [1.0] * 3], [1.0, 0.0], [0.5, 0.5], [1.5, ior])
    cam = camera((0, 0, 1.5), (0, 0, 0), (0, 1, 0), 30.0, 16, 16)
    return _scene(b, mats, (0.0, 0.0, 0.0), camera=cam)


def random_soup(n_tris=200, seed=0, spread=1.0, size=0.3, n_mats=4):
    """Random triangles in a cube, random Lambert materials (intersection tests)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-spread, spread, size=(n_tris, 1, 3))
    V = (c + rng.normal(0.0, size, size=(n_tris, 3, 3))).reshape(-1, 3)
    T = np.arange(3 * n_tris).reshape(-1, 3)
    b = _Builder()
    b.v.append(V)
    b.t.append(T)
    b.m.append(rng.integers(0, n_mats, size=n_tris))
    b.nv = len(V)
    mats = _materials([LAMBERT] * n_mats, rng.uniform(0.1, 0.9, size=(n_mats, 3)), [0.0] * n_mats,
                      [0.5] * n_mats, [1.5] * n_mats)
    return _scene(b, mats, (0.2, 0.3, 0.4))


def random_rays(n, seed=0, spread=1.5):
    """Ray origins in a cube and unit directions (uniform on the sphere), float64."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(-spread, spread, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d
