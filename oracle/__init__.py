"""FP64 CPU oracle for the path-traced light-transport estimator (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this package, and this
package never imports the product package: the two share nothing but the seeded scene
generators' arrays that the caller passes in.

The arithmetic lives in ``oracle.c`` (plain C99, FP64, OpenMP over paths); this module only
compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAT_LAMBERT, MAT_GGX, MAT_DIELECTRIC = 0, 1, 2
BSDF_CODES = {"lambert": 0, "ggx": 1, "ggx_invalid": 2, "reflect": 3, "refract": 4, "tir": 5}


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (portable flags: no -march, no fast-math,
    no FP contraction, so x86 and Arm builds round identically)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _f(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def build_variant(replacements, out_dir: str, name: str = "liboracle_variant.so") -> str:
    """Compile a copy of oracle.c with textual replacements [(old, new), ...] into out_dir (testing
    aid: the pins must fail on an oracle with a planted mistake).  Each `old` must occur exactly once."""
    src = open(_SRC).read()
    for old, new in replacements:
        if src.count(old) != 1:
            raise ValueError(f"planted change does not match exactly once: {old!r}")
        src = src.replace(old, new)
    os.makedirs(out_dir, exist_ok=True)
    c_path = os.path.join(out_dir, name.replace(".so", ".c"))
    with open(c_path, "w") as f:
        f.write(src)
    out = os.path.join(out_dir, name)
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", "-Wall", "-Wno-unused-function", c_path, "-o", out, "-lm"], check=True)
    return out


class use_library:
    """Context manager: route every call of this module to another build of the oracle (a variant
    from build_variant); the default library is restored on exit."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        with _lock:
            self._saved = _lib
            _lib = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _load(_LIB_PATH)
    return _lib


def _load(path: str):
    """Open one build of the oracle and declare its C signatures."""
    L = C.CDLL(path)
    vp, u32, u64, i64, i32, f32, f64 = (C.c_void_p, C.c_uint32, C.c_uint64, C.c_int64,
                                        C.c_int, C.c_float, C.c_double)
    L.or_pcg_hash.restype = u32
    L.or_pcg_hash.argtypes = [u32]
    L.or_path_key.restype = u32
    L.or_path_key.argtypes = [u64, u32, u32]
    L.or_u01.restype = f64
    L.or_u01.argtypes = [u32, u32, u32]
    L.or_u01_batch.argtypes = [u64, vp, vp, vp, vp, i64, vp]
    L.or_radical_inverse24.restype = u32
    L.or_radical_inverse24.argtypes = [u32, u32]
    L.or_pixel_jitter_batch.argtypes = [u32, u64, vp, vp, i64, vp]
    L.or_scene_create.restype = vp
    L.or_scene_create.argtypes = [vp, i64, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp]
    L.or_scene_destroy.argtypes = [vp]
    L.or_scene_create_corners.restype = vp
    L.or_scene_create_corners.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, vp, vp]
    L.or_scene_set_materials.argtypes = [vp, vp, vp]
    L.or_scene_n_lights.restype = i64
    L.or_scene_n_lights.argtypes = [vp]
    L.or_scene_light_area.restype = f64
    L.or_scene_light_area.argtypes = [vp]
    L.or_intersect_batch.argtypes = [vp, vp, vp, i64, i32, vp, vp, vp, vp]
    L.or_occluded_batch.argtypes = [vp, vp, vp, vp, i64, i32, vp]
    L.or_bsdf_eval.argtypes = [u32, vp, f64, vp, vp, vp, vp]
    L.or_bsdf_sample.restype = i32
    L.or_bsdf_sample.argtypes = [u32, vp, f64, f64, vp, vp, vp, f64, f64, f64, vp, vp, vp]
    L.or_onb.argtypes = [vp, vp, vp]
    L.or_bsdf_pdf.restype = f64
    L.or_bsdf_pdf.argtypes = [u32, f64, vp, vp, vp]
    L.or_fresnel_dielectric.restype = f64
    L.or_fresnel_dielectric.argtypes = [f64, f64, f64]
    L.or_ggx_D.restype = f64
    L.or_ggx_D.argtypes = [f64, f64]
    L.or_ggx_G1.restype = f64
    L.or_ggx_G1.argtypes = [f64, f64]
    L.or_render_paths.argtypes = [vp, vp, vp, vp, f32, u32, u32, u32, u32, u64, u32, f64, u32, i32,
                                  vp, i64, i32, vp, vp, i32, vp, vp, vp, vp]
    L.or_render_pixels.argtypes = [vp, vp, vp, vp, f32, u32, u32, u32, u32, u64, u32, f64, u32, i32,
                                   vp, i64, i32, vp, vp]
    L.or_trace_rays.argtypes = [vp, vp, vp, vp, i64, u32, u32, f64, u32, i32, i32, vp, vp, i32, vp, vp]
    L.or_trace_path_events.argtypes = [vp, vp, vp, vp, f32, u32, u32, u32, u32, u64, u32, f64, u32, vp, i64, vp,
                                       vp, vp, vp]
    L.or_max_tangents.restype = i32
    L.or_camera_rays.argtypes = [vp, vp, vp, f32, u32, u32, vp, vp, vp, i64, vp, vp]
    L.or_pick_light_batch.argtypes = [vp, vp, i64, vp]
    L.or_scene_light_tris.argtypes = [vp, vp]
    return L


# ---------------------------------------------------------------- random numbers
def pcg_hash(v: int) -> int:
    return int(lib().or_pcg_hash(v & 0xFFFFFFFF))


def path_key(seed: int, pixel: int, sample: int) -> int:
    return int(lib().or_path_key(seed, pixel, sample))


SAMPLERS = {"pcg": 0, "halton": 1}


def _opts(sampler: str, mis: bool) -> int:
    """Option bits of the render calls: 1 = Halton pixel jitter, 2 = multiple importance sampling."""
    return SAMPLERS[sampler] | (2 if mis else 0)


def radical_inverse24(base: int, s: int) -> int:
    """floor(2^24 * phi_base(s)): the radical inverse of s in 24-bit fixed point."""
    return int(lib().or_radical_inverse24(int(base), int(s)))


def pixel_jitter(sampler: str, seed: int, pixel, sample) -> np.ndarray:
    """Sub-pixel jitter (u0, u1) of camera rays, (n, 2)."""
    px = _f(pixel, np.uint32).reshape(-1)
    sm = _f(sample, np.uint32).reshape(-1)
    out = np.empty((px.size, 2))
    lib().or_pixel_jitter_batch(SAMPLERS[sampler], seed, _p(px), _p(sm), px.size, _p(out))
    return out


def u01(seed, pixel, sample, bounce, dim) -> np.ndarray:
    """Uniforms for arrays of (pixel, sample, bounce, dim) under one seed."""
    px, sm, bo, dm = (_f(np.broadcast_to(a, np.broadcast(pixel, sample, bounce, dim).shape), np.uint32)
                      for a in (pixel, sample, bounce, dim))
    out = np.empty(px.shape, np.float64)
    lib().or_u01_batch(seed, _p(px), _p(sm), _p(bo), _p(dm), px.size, _p(out))
    return out


def camera_rays(cam: dict, pixel, u0, u1):
    """The ray-generation step for explicit pixels and sub-pixel offsets: (origins, unit directions)."""
    px = _f(pixel, np.uint32).reshape(-1)
    a = _f(np.broadcast_to(u0, px.shape), np.float64)
    b = _f(np.broadcast_to(u1, px.shape), np.float64)
    o, d = np.empty((px.size, 3)), np.empty((px.size, 3))
    lib().or_camera_rays(_p(_f(cam["eye"], np.float32)), _p(_f(cam["target"], np.float32)),
                         _p(_f(cam["up"], np.float32)), float(cam["vfov_deg"]), int(cam["width"]),
                         int(cam["height"]), _p(px), _p(a), _p(b), px.size, _p(o), _p(d))
    return o, d


# ---------------------------------------------------------------- BSDFs (pins)
def bsdf_eval(mtype, albedo, roughness, n, wo, wi) -> np.ndarray:
    out = np.empty(3)
    lib().or_bsdf_eval(mtype, _p(_f(albedo, np.float64)), roughness, _p(_f(n, np.float64)),
                       _p(_f(wo, np.float64)), _p(_f(wi, np.float64)), _p(out))
    return out


def bsdf_sample(mtype, albedo, roughness, ior, n, ng, wo, u5, u6, u7):
    wi = np.empty(3)
    w = np.empty(3)
    code = np.zeros(1, np.int32)
    ok = lib().or_bsdf_sample(mtype, _p(_f(albedo, np.float64)), roughness, ior, _p(_f(n, np.float64)),
                              _p(_f(ng, np.float64)), _p(_f(wo, np.float64)), u5, u6, u7, _p(wi), _p(w),
                              _p(code))
    return bool(ok), wi, w, int(code[0])


def bsdf_pdf(mtype, roughness, n, wo, wi) -> float:
    """Solid-angle density with which bsdf_sample draws wi (0 for the smooth dielectric)."""
    return float(lib().or_bsdf_pdf(mtype, roughness, _p(_f(n, np.float64)), _p(_f(wo, np.float64)),
                                   _p(_f(wi, np.float64))))


def onb(n):
    t, b = np.empty(3), np.empty(3)
    lib().or_onb(_p(_f(n, np.float64)), _p(t), _p(b))
    return t, b


def fresnel_dielectric(ci, eta_i, eta_t) -> float:
    return float(lib().or_fresnel_dielectric(ci, eta_i, eta_t))


def ggx_D(roughness, cos_h) -> float:
    return float(lib().or_ggx_D(roughness, cos_h))


def ggx_G1(roughness, cos_v) -> float:
    return float(lib().or_ggx_G1(roughness, cos_v))


# ---------------------------------------------------------------- scenes
class Scene:
    """Oracle scene: triangles (FP32 input, FP64 inside), materials, environment, plain BVH."""

    def __init__(self, verts, tris, tri_mat, mat_type, mat_albedo, mat_emission, mat_roughness,
                 mat_ior, env):
        self._keep = [_f(verts, np.float32).reshape(-1, 3), _f(tris, np.uint32).reshape(-1, 3),
                      _f(tri_mat, np.uint32), _f(mat_type, np.uint32),
                      _f(mat_albedo, np.float32).reshape(-1, 3), _f(mat_emission, np.float32),
                      _f(mat_roughness, np.float32), _f(mat_ior, np.float32), _f(env, np.float32)]
        v, t, tm, mt, ma, me, mr, mi, ev = self._keep
        self.n_tris = t.shape[0]
        self.n_mats = mt.shape[0]
        self.h = lib().or_scene_create(_p(v), v.shape[0], _p(t), t.shape[0], _p(tm), mt.shape[0],
                                       _p(mt), _p(ma), _p(me), _p(mr), _p(mi), _p(ev))

    @classmethod
    def from_dict(cls, sc: dict) -> "Scene":
        if "meshes" in sc:
            return cls.from_instanced(sc)
        return cls(sc["verts"], sc["tris"], sc["tri_mat"], sc["mat_type"], sc["mat_albedo"],
                   sc["mat_emission"], sc["mat_roughness"], sc["mat_ior"], sc["env"])

    @classmethod
    def from_instanced(cls, sc: dict) -> "Scene":
        """A two-level scene placed in the world in FP64: every instance's mesh triangles, in
        instance order, with world = R v + t from the instance's [R | t]; an instance material other
        than 0xFFFFFFFF replaces the mesh's triangle materials."""
        corners, tmat = [], []
        for m, X, im in zip(sc["inst_mesh"], sc["inst_xform"], sc["inst_mat"]):
            mesh = sc["meshes"][int(m)]
            V = np.asarray(mesh["verts"], np.float32).astype(np.float64)
            X = np.asarray(X, np.float32).astype(np.float64)
            W = V @ X[:, :3].T + X[:, 3]
            corners.append(W[np.asarray(mesh["tris"], np.int64)])
            tm = np.asarray(mesh["tri_mat"], np.uint32)
            tmat.append(tm if int(im) == 0xFFFFFFFF else np.full(len(tm), int(im), np.uint32))
        self = cls.__new__(cls)
        c = np.ascontiguousarray(np.concatenate(corners).reshape(-1, 9), np.float64) if corners else np.zeros((0, 9))
        self._keep = [c, _f(np.concatenate(tmat) if tmat else np.zeros(0), np.uint32), _f(sc["mat_type"], np.uint32),
                      _f(sc["mat_albedo"], np.float32).reshape(-1, 3), _f(sc["mat_emission"], np.float32),
                      _f(sc["mat_roughness"], np.float32), _f(sc["mat_ior"], np.float32), _f(sc["env"], np.float32)]
        c, tm, mt, ma, me, mr, mi, ev = self._keep
        self.n_tris = c.shape[0]
        self.n_mats = mt.shape[0]
        self.h = lib().or_scene_create_corners(_p(c), c.shape[0], _p(tm), mt.shape[0], _p(mt), _p(ma), _p(me),
                                               _p(mr), _p(mi), _p(ev))
        return self

    def close(self):
        if getattr(self, "h", None):
            lib().or_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_lights(self) -> int:
        return int(lib().or_scene_n_lights(self.h))

    @property
    def light_area(self) -> float:
        return float(lib().or_scene_light_area(self.h))

    def pick_light(self, u) -> np.ndarray:
        """Light index drawn by each uniform (the NEE light pick on its own)."""
        uu = _f(u, np.float64).reshape(-1)
        out = np.empty(uu.size, np.int64)
        lib().or_pick_light_batch(self.h, _p(uu), uu.size, _p(out))
        return out

    @property
    def light_tris(self) -> np.ndarray:
        """Triangle id of each light, in light-index order."""
        out = np.empty(max(self.n_lights, 0), np.int64)
        if out.size:
            lib().or_scene_light_tris(self.h, _p(out))
        return out

    def set_materials(self, albedo, emission):
        a = _f(albedo, np.float32).reshape(-1, 3)
        e = _f(emission, np.float32)
        self._keep[4], self._keep[5] = a, e
        lib().or_scene_set_materials(self.h, _p(a), _p(e))

    def intersect(self, o, d, use_bvh=True):
        o = _f(o, np.float64).reshape(-1, 3)
        d = _f(d, np.float64).reshape(-1, 3)
        n = o.shape[0]
        t, u, v = np.empty(n), np.empty(n), np.empty(n)
        prim = np.empty(n, np.int64)
        lib().or_intersect_batch(self.h, _p(o), _p(d), n, int(use_bvh), _p(t), _p(prim), _p(u), _p(v))
        return t, prim, u, v

    def occluded(self, o, d, tmax, use_bvh=True):
        o = _f(o, np.float64).reshape(-1, 3)
        d = _f(d, np.float64).reshape(-1, 3)
        tm = _f(tmax, np.float64).reshape(-1)
        out = np.empty(o.shape[0], np.int32)
        lib().or_occluded_batch(self.h, _p(o), _p(d), _p(tm), o.shape[0], int(use_bvh), _p(out))
        return out.astype(bool)

    @staticmethod
    def _cam(cam: dict):
        return (_f(cam["eye"], np.float32), _f(cam["target"], np.float32), _f(cam["up"], np.float32),
                float(cam["vfov_deg"]), int(cam["width"]), int(cam["height"]))

    def render_paths(self, cam, spp, max_depth, seed, path_ids, rr_start=3, rr_fixed=0.0,
                     use_bvh=True, dir_albedo=None, dir_emission=None, n_threads=0, sampler="pcg", mis=False):
        """Per-path radiance, optional directional derivatives, branch signatures, ray counts."""
        eye, tgt, up, fov, W, H = self._cam(cam)
        ids = _f(path_ids, np.uint64).reshape(-1)
        n = ids.size
        L = np.empty((n, 3))
        sig = np.empty(n, np.uint32)
        rays = np.zeros(2, np.uint64)
        nd = 0 if dir_albedo is None else int(np.asarray(dir_albedo).shape[0])
        if nd:
            da = _f(dir_albedo, np.float64).reshape(nd, self.n_mats, 3)
            de = _f(dir_emission, np.float64).reshape(nd, self.n_mats)
            dL = np.empty((n, nd, 3))
            args = (nd, _p(da), _p(de))
        else:
            dL = None
            args = (0, None, None)
        lib().or_render_paths(self.h, _p(eye), _p(tgt), _p(up), fov, W, H, spp, max_depth, seed,
                              rr_start, float(rr_fixed), _opts(sampler, mis), int(use_bvh), _p(ids), n, *args, n_threads,
                              _p(L), _p(dL) if dL is not None else None, _p(sig), _p(rays))
        return {"L": L, "dL": dL, "sig": sig, "rays": rays}

    def render_pixels(self, cam, spp, max_depth, seed, pixels=None, rr_start=3, rr_fixed=0.0,
                      use_bvh=True, n_threads=0, sampler="pcg", mis=False):
        """Mean radiance of the listed pixels (all pixels when None); returns (img (n,3), rays)."""
        eye, tgt, up, fov, W, H = self._cam(cam)
        if pixels is None:
            pixels = np.arange(W * H, dtype=np.uint32)
        px = _f(pixels, np.uint32).reshape(-1)
        img = np.empty((px.size, 3))
        rays = np.zeros(2, np.uint64)
        lib().or_render_pixels(self.h, _p(eye), _p(tgt), _p(up), fov, W, H, spp, max_depth, seed,
                               rr_start, float(rr_fixed), _opts(sampler, mis), int(use_bvh), _p(px), px.size, n_threads,
                               _p(img), _p(rays))
        return img, rays

    def path_events(self, cam, spp, max_depth, seed, path_ids, rr_start=3, rr_fixed=0.0, sampler="pcg", mis=False):
        """Event logs of the listed camera paths: list of [(bounce, kind, value, f0, f1), ...]."""
        eye, tgt, up, fov, W, H = self._cam(cam)
        ids = _f(path_ids, np.uint64).reshape(-1)
        n = ids.size
        ev = np.zeros((n, 64, 2), np.uint32)
        pay = np.zeros((n, 64, 2))
        n_ev = np.zeros(n, np.uint32)
        L = np.zeros((n, 3))
        lib().or_trace_path_events(self.h, _p(eye), _p(tgt), _p(up), fov, W, H, spp, max_depth, seed, rr_start,
                                   float(rr_fixed), _opts(sampler, mis), _p(ids), n, _p(ev), _p(pay), _p(n_ev), _p(L))
        return [[(int(ev[i, k, 0] >> 4), int(ev[i, k, 0] & 15), int(ev[i, k, 1]), float(pay[i, k, 0]),
                  float(pay[i, k, 1])) for k in range(n_ev[i])] for i in range(n)], L

    def trace_rays(self, o, d, keys, max_depth, rr_start=1 << 30, rr_fixed=0.0, use_bvh=True,
                   dir_albedo=None, dir_emission=None, n_threads=0, mis=False):
        o = _f(o, np.float64).reshape(-1, 3)
        d = _f(d, np.float64).reshape(-1, 3)
        k = _f(keys, np.uint32).reshape(-1)
        n = o.shape[0]
        L = np.empty((n, 3))
        nd = 0 if dir_albedo is None else int(np.asarray(dir_albedo).shape[0])
        if nd:
            da = _f(dir_albedo, np.float64).reshape(nd, self.n_mats, 3)
            de = _f(dir_emission, np.float64).reshape(nd, self.n_mats)
            dL = np.empty((n, nd, 3))
            lib().or_trace_rays(self.h, _p(o), _p(d), _p(k), n, max_depth, rr_start, float(rr_fixed),
                                _opts("pcg", mis), int(use_bvh), nd, _p(da), _p(de), n_threads, _p(L), _p(dL))
            return L, dL
        lib().or_trace_rays(self.h, _p(o), _p(d), _p(k), n, max_depth, rr_start, float(rr_fixed),
                            _opts("pcg", mis), int(use_bvh), 0, None, None, n_threads, _p(L), None)
        return L, None
