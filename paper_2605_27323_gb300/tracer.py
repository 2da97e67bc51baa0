"""Python front of the C ABI: scenes, renders, gradients and batches on torch device memory.

torch provides device buffers and the current CUDA stream; every computation runs in libpt.so.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import capi


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (libpt.so has no CPU path)")
    return torch


def _stream(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(None)


def make_camera(cam: dict) -> capi.Camera:
    c = capi.Camera()
    for k in ("eye", "target", "up"):
        getattr(c, k)[:] = [float(x) for x in np.asarray(cam[k], np.float32)]
    c.vfov_deg = float(cam["vfov_deg"])
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def make_opts(mode="wavefront", rr_start=3, rr_fixed=0.0, sort="none", block_size=0, queue_capacity=0,
              profile=False, sig=None, graph=True, mk_static=False, hybrid=0, sampler="pcg",
              mis=False, short_stack=False, count_traversal=False, separate_shadow=False) -> capi.RenderOpts:
    o = capi.RenderOpts()
    o.mode = capi.MODE[mode] if isinstance(mode, str) else int(mode)
    o.rr_start = int(rr_start)
    o.rr_fixed = float(rr_fixed)
    o.sort_mode = capi.SORT[sort] if isinstance(sort, str) else int(sort)
    o.block_size = int(block_size)
    o.flags = ((capi.FLAG_PROFILE if profile else 0) | (0 if graph else capi.FLAG_NO_GRAPH)
               | (capi.FLAG_MK_STATIC if mk_static else 0) | (capi.FLAG_HALTON if sampler == "halton" else 0)
               | (capi.FLAG_MIS if mis else 0) | (capi.FLAG_SHORT_STACK if short_stack else 0)
               | (capi.FLAG_COUNT_TRAVERSAL if count_traversal else 0)
               | (capi.FLAG_SEPARATE_SHADOW if separate_shadow else 0))
    if sampler not in ("pcg", "halton"):
        raise ValueError("sampler must be 'pcg' or 'halton'")
    o.queue_capacity = int(queue_capacity)
    o.d_path_sig = sig.data_ptr() if sig is not None else None
    o.hybrid_threshold = int(hybrid)
    return o


def _materials(sc: dict):
    mt = np.asarray(sc["mat_type"], np.uint32).reshape(-1)
    ma = np.asarray(sc["mat_albedo"], np.float32).reshape(-1, 3)
    me = np.asarray(sc["mat_emission"], np.float32).reshape(-1)
    mr = np.asarray(sc["mat_roughness"], np.float32).reshape(-1)
    mi = np.asarray(sc["mat_ior"], np.float32).reshape(-1)
    n_m = mt.size
    mats = (capi.Material * max(n_m, 1))()
    for k in range(n_m):
        mats[k].type = int(mt[k])
        mats[k].albedo[:] = [float(x) for x in ma[k]]
        mats[k].emission = float(me[k])
        mats[k].roughness = float(mr[k])
        mats[k].ior = float(mi[k])
    return mats


class Scene:
    """A scene uploaded to the current CUDA device (pt_scene_create, pt_scene_create_instanced)."""

    def __init__(self, verts, tris, tri_mat, mat_type, mat_albedo, mat_emission, mat_roughness, mat_ior,
                 env=(0.0, 0.0, 0.0)):
        torch = _torch()
        self._lib = capi.load()
        v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
        t = np.ascontiguousarray(tris, np.uint32).reshape(-1, 3)
        tm = np.ascontiguousarray(tri_mat, np.uint32).reshape(-1)
        n_m = int(np.asarray(mat_type).size)
        mats = _materials({"mat_type": mat_type, "mat_albedo": mat_albedo, "mat_emission": mat_emission,
                           "mat_roughness": mat_roughness, "mat_ior": mat_ior})
        envv = (C.c_float * 3)(*[float(x) for x in np.asarray(env, np.float32).reshape(3)])
        h = C.c_void_p()
        capi.check(self._lib.pt_scene_create(v.ctypes.data_as(C.c_void_p), v.shape[0], t.ctypes.data_as(C.c_void_p),
                                             t.shape[0], tm.ctypes.data_as(C.c_void_p), mats, n_m, envv,
                                             _stream(torch), C.byref(h)))
        self.h = h
        self.n_mats = n_m
        self.n_tris = t.shape[0]

    @classmethod
    def from_dict(cls, sc: dict) -> "Scene":
        if "meshes" in sc:
            return cls.from_instanced(sc)
        return cls(sc["verts"], sc["tris"], sc["tri_mat"], sc["mat_type"], sc["mat_albedo"], sc["mat_emission"],
                   sc["mat_roughness"], sc["mat_ior"], sc["env"])

    @classmethod
    def from_instanced(cls, sc: dict) -> "Scene":
        """A two-level scene (pt_scene_create_instanced): sc["meshes"] = [{verts, tris, tri_mat}] in object
        space; sc["inst_mesh"] (I,), sc["inst_xform"] (I, 3, 4) object-to-world [R | t], sc["inst_mat"] (I,)
        (capi.NO_MATERIAL keeps the mesh's materials)."""
        torch = _torch()
        self = cls.__new__(cls)
        self._lib = capi.load()
        meshes = sc["meshes"]
        nm = len(meshes)
        keep = []
        vp = (C.c_void_p * nm)()
        tp = (C.c_void_p * nm)()
        mp = (C.c_void_p * nm)()
        nv = (C.c_uint32 * nm)()
        nt = (C.c_uint32 * nm)()
        for k, m in enumerate(meshes):
            v = np.ascontiguousarray(m["verts"], np.float32).reshape(-1, 3)
            t = np.ascontiguousarray(m["tris"], np.uint32).reshape(-1, 3)
            tm = np.ascontiguousarray(m["tri_mat"], np.uint32).reshape(-1)
            keep += [v, t, tm]
            vp[k], tp[k], mp[k] = v.ctypes.data, t.ctypes.data, tm.ctypes.data
            nv[k], nt[k] = v.shape[0], t.shape[0]
        im = np.asarray(sc["inst_mesh"], np.uint32).reshape(-1)
        ix = np.asarray(sc["inst_xform"], np.float32).reshape(-1, 12)
        imat = np.asarray(sc["inst_mat"], np.uint32).reshape(-1)
        ni = im.size
        inst = (capi.Instance * ni)()
        for k in range(ni):
            inst[k].xform[:] = [float(x) for x in ix[k]]
            inst[k].mesh = int(im[k])
            inst[k].material = int(imat[k])
        mats = _materials(sc)
        n_m = int(np.asarray(sc["mat_type"]).size)
        envv = (C.c_float * 3)(*[float(x) for x in np.asarray(sc["env"], np.float32).reshape(3)])
        h = C.c_void_p()
        capi.check(self._lib.pt_scene_create_instanced(nm, vp, nv, tp, nt, mp, inst, ni, mats, n_m, envv,
                                                       _stream(torch), C.byref(h)))
        self.h = h
        self.n_mats = n_m
        self.n_tris = int(sum(int(nt[int(m)]) for m in im))
        return self

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.pt_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        a, b, c, e = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        area = C.c_float()
        capi.check(self._lib.pt_scene_info(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(area), C.byref(e)))
        return {"n_tris": a.value, "n_nodes": b.value, "n_lights": c.value, "light_area": area.value,
                "device_bytes": e.value}

    def set_materials(self, albedo=None, emission=None):
        torch = _torch()
        a = albedo.detach().to(device="cuda", dtype=torch.float32).contiguous() if albedo is not None else None
        e = emission.detach().to(device="cuda", dtype=torch.float32).contiguous() if emission is not None else None
        capi.check(self._lib.pt_scene_set_materials(self.h, _ptr(a), _ptr(e), _stream(torch)))
        self._keep = (a, e)

    def render(self, cam: dict, spp: int, max_depth: int, seed: int = 0, out=None, path_L: bool = False,
               sig: bool = False, **opt_kw):
        """Render an H x W x 3 float32 image (torch CUDA tensor, or the given `out`, which may be a
        pinned/pageable CPU tensor: the library then stages the copy).  With path_L / sig the
        per-path radiance (N_p x 3) and branch signatures (N_p) are returned too."""
        torch = _torch()
        c = make_camera(cam)
        W, H = c.width, c.height
        n_paths = W * H * spp
        img = out if out is not None else torch.empty((H, W, 3), device="cuda", dtype=torch.float32)
        pl = torch.empty((n_paths, 3), device="cuda", dtype=torch.float32) if path_L else None
        sg = torch.empty((n_paths,), device="cuda", dtype=torch.int32) if sig else None
        o = make_opts(sig=sg, **opt_kw)
        capi.check(self._lib.pt_render(self.h, C.byref(c), spp, max_depth, seed, C.byref(o), _ptr(img), _ptr(pl),
                                       _stream(torch)))
        if path_L or sig:
            return {"img": img, "path_L": pl, "sig": sg}
        return img

    def render_progressive(self, cam: dict, spp: int, max_depth: int, seed: int, sample_offset: int, accum,
                           out=None, **opt_kw):
        """Add samples sample_offset .. sample_offset + spp - 1 of every pixel to the running sums
        `accum` (H x W x 3 float32 CUDA tensor; zeroed when sample_offset == 0) and return the running
        mean (into `out` if given)."""
        torch = _torch()
        c = make_camera(cam)
        img = out if out is not None else torch.empty((c.height, c.width, 3), device="cuda", dtype=torch.float32)
        o = make_opts(**opt_kw)
        capi.check(self._lib.pt_render_progressive(self.h, C.byref(c), spp, max_depth, seed, int(sample_offset),
                                                   C.byref(o), _ptr(accum), _ptr(img), _stream(torch)))
        return img

    def backward(self, cam: dict, spp: int, max_depth: int, seed: int, grad_img, g_albedo=None, g_emission=None,
                 **opt_kw):
        """Accumulate d(loss)/d(albedo) (n_mats x 3) and d(loss)/d(emission) (n_mats) for the image
        of render(cam, spp, max_depth, seed) given grad_img = d(loss)/d(image)."""
        torch = _torch()
        c = make_camera(cam)
        g = grad_img.detach().to(dtype=torch.float32).contiguous()
        if g_albedo is None:
            g_albedo = torch.zeros((self.n_mats, 3), device="cuda", dtype=torch.float32)
        if g_emission is None:
            g_emission = torch.zeros((self.n_mats,), device="cuda", dtype=torch.float32)
        o = make_opts(**opt_kw)
        capi.check(self._lib.pt_render_backward(self.h, C.byref(c), spp, max_depth, seed, C.byref(o), _ptr(g),
                                                _ptr(g_albedo), _ptr(g_emission), _stream(torch)))
        return g_albedo, g_emission

    def trace_closest(self, o, d):
        """Closest hits of rays (n x 3 origins, n x 3 directions): (t, original triangle id or -1)."""
        torch = _torch()
        o = torch.as_tensor(o, dtype=torch.float32, device="cuda").reshape(-1, 3)
        d = torch.as_tensor(d, dtype=torch.float32, device="cuda").reshape(-1, 3)
        n = o.shape[0]
        rays = torch.zeros((n, 8), device="cuda", dtype=torch.float32)
        rays[:, 0:3] = o
        rays[:, 4:7] = d
        t = torch.empty(n, device="cuda", dtype=torch.float32)
        prim = torch.empty(n, device="cuda", dtype=torch.int32)
        capi.check(self._lib.pt_trace_closest(self.h, _ptr(rays), n, _ptr(t), _ptr(prim), _stream(torch)))
        return t, prim

    def path_events(self, cam: dict, spp: int, max_depth: int, seed: int, path_ids, **opt_kw):
        """Event logs of the listed paths (testing aid): list of [(bounce, kind, value, f0, f1)], and
        the paths' radiance."""
        torch = _torch()
        c = make_camera(cam)
        ids = torch.as_tensor(np.ascontiguousarray(path_ids, np.uint64).astype(np.int64), device="cuda")
        n = ids.numel()
        ev = torch.zeros((n, 64, 2), device="cuda", dtype=torch.int32)
        pay = torch.zeros((n, 64, 2), device="cuda", dtype=torch.float32)
        nev = torch.zeros((n,), device="cuda", dtype=torch.int32)
        L = torch.zeros((n, 3), device="cuda", dtype=torch.float32)
        o = make_opts(**opt_kw)
        capi.check(self._lib.pt_debug_trace_paths(self.h, C.byref(c), spp, max_depth, seed, C.byref(o), _ptr(ids), n,
                                                  _ptr(ev), _ptr(pay), _ptr(nev), _ptr(L), _stream(torch)))
        ev = ev.cpu().numpy().astype(np.uint32)
        pay = pay.cpu().numpy()
        nev = nev.cpu().numpy()
        return [[(int(ev[i, k, 0] >> 4), int(ev[i, k, 0] & 15), int(ev[i, k, 1]), float(pay[i, k, 0]),
                  float(pay[i, k, 1])) for k in range(nev[i])] for i in range(n)], L.cpu().numpy()

    def stats(self) -> dict:
        s = capi.Stats()
        capi.check(self._lib.pt_get_stats(self.h, C.byref(s)))
        d = {k: getattr(s, k) for k, _ in capi.Stats._fields_ if k not in ("active", "shadow_queued", "group_walks")}
        d["group_walks"] = list(s.group_walks)
        d["active"] = list(s.active)[: s.bounces]
        d["shadow_queued"] = list(s.shadow_queued)[: s.bounces]
        return d


class Progressive:
    """Progressive rendering of one view: each add(spp) renders the next spp samples of every pixel
    and returns the running mean; state() / Progressive.resume() save and continue the render from
    (per-pixel sums, sample count)."""

    def __init__(self, scene: Scene, cam: dict, max_depth: int, seed: int = 0, **opt_kw):
        torch = _torch()
        self.scene, self.cam, self.max_depth, self.seed, self.opt_kw = scene, cam, max_depth, seed, opt_kw
        self.sums = torch.zeros((cam["height"], cam["width"], 3), device="cuda", dtype=torch.float32)
        self.count = 0

    def add(self, spp: int, out=None):
        img = self.scene.render_progressive(self.cam, spp, self.max_depth, self.seed, self.count, self.sums, out=out,
                                            **self.opt_kw)
        self.count += int(spp)
        return img

    def state(self) -> dict:
        return {"sums": self.sums.clone(), "count": self.count, "seed": self.seed}

    @classmethod
    def resume(cls, scene: Scene, cam: dict, max_depth: int, state: dict, **opt_kw) -> "Progressive":
        p = cls(scene, cam, max_depth, state["seed"], **opt_kw)
        p.sums.copy_(state["sums"])
        p.count = int(state["count"])
        return p


def debug_rng(seed: int, pixel, sample, bounce, dim):
    torch = _torch()
    lib = capi.load()
    ts = [torch.as_tensor(np.ascontiguousarray(a, np.uint32).astype(np.int32), device="cuda") for a in
          (pixel, sample, bounce, dim)]
    n = ts[0].numel()
    out = torch.empty(n, device="cuda", dtype=torch.float32)
    capi.check(lib.pt_debug_rng(seed, *[_ptr(t) for t in ts], n, _ptr(out), _stream(torch)))
    return out


def render_batch(scenes: Sequence[Scene], cams: Sequence[dict], spps: Sequence[int], max_depth: int, seed: int = 0,
                 outs: Optional[list] = None, **opt_kw):
    """Render several scenes in one persistent wavefront (pt_render_batch)."""
    torch = _torch()
    lib = capi.load()
    n = len(scenes)
    cam_arr = (capi.Camera * n)(*[make_camera(c) for c in cams])
    spp_arr = (C.c_uint32 * n)(*[int(s) for s in spps])
    if outs is None:
        outs = [torch.empty((int(c["height"]), int(c["width"]), 3), device="cuda", dtype=torch.float32) for c in cams]
    sc_arr = (C.c_void_p * n)(*[s.h.value for s in scenes])
    out_arr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    o = make_opts(**opt_kw)
    capi.check(lib.pt_render_batch(sc_arr, cam_arr, spp_arr, n, max_depth, seed, C.byref(o), out_arr,
                                   _stream(torch)))
    return outs


def autotune_batch(scenes: Sequence[Scene], cams: Sequence[dict], spps: Sequence[int], max_depth: int, seed: int = 0,
                   outs: Optional[list] = None, **opt_kw):
    """Pick queue capacity, block size and sort granularity for render_batch by timing candidates."""
    torch = _torch()
    lib = capi.load()
    n = len(scenes)
    cam_arr = (capi.Camera * n)(*[make_camera(c) for c in cams])
    spp_arr = (C.c_uint32 * n)(*[int(s) for s in spps])
    if outs is None:
        outs = [torch.empty((int(c["height"]), int(c["width"]), 3), device="cuda", dtype=torch.float32) for c in cams]
    sc_arr = (C.c_void_p * n)(*[s.h.value for s in scenes])
    out_arr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    base = make_opts(**opt_kw)
    best = capi.RenderOpts()
    ms = C.c_float()
    capi.check(lib.pt_autotune_batch(sc_arr, cam_arr, spp_arr, n, max_depth, seed, C.byref(base), out_arr,
                                     _stream(torch), C.byref(best), C.byref(ms)))
    return {"queue_capacity": best.queue_capacity, "block_size": best.block_size, "sort": best.sort_mode,
            "ms": ms.value}


def _autograd_fn():
    import torch

    class PTRenderFn(torch.autograd.Function):
        """image = render(albedo, emission); backward = path-replay adjoint (pt_render_backward)."""

        @staticmethod
        def forward(ctx, albedo, emission, scene: Scene, cam: dict, spp: int, max_depth: int, seed: int,
                    opt_kw: dict):
            scene.set_materials(albedo, emission)
            img = scene.render(cam, spp, max_depth, seed, **(opt_kw or {}))
            ctx.scene, ctx.cam, ctx.spp, ctx.max_depth, ctx.seed, ctx.opt_kw = scene, cam, spp, max_depth, seed, opt_kw
            return img

        @staticmethod
        def backward(ctx, grad_img):
            kw = dict(ctx.opt_kw or {})
            kw.pop("mode", None)
            ga, ge = ctx.scene.backward(ctx.cam, ctx.spp, ctx.max_depth, ctx.seed, grad_img.contiguous(), **kw)
            return ga, ge, None, None, None, None, None, None

    return PTRenderFn


_PTRenderFn = None


def render_differentiable(albedo, emission, scene: Scene, cam: dict, spp: int, max_depth: int, seed: int = 0,
                          **opt_kw):
    """Differentiable render: gradients flow to albedo (n_mats x 3) and emission (n_mats)."""
    global _PTRenderFn
    if _PTRenderFn is None:
        _PTRenderFn = _autograd_fn()
    return _PTRenderFn.apply(albedo, emission, scene, cam, spp, max_depth, seed, opt_kw)
