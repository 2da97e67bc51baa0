"""pt_render_wavefront_static: the wavefront render for callers that cannot allocate device memory
(an application whose memory manager owns the whole device, or a real-time loop that cannot absorb
cudaMalloc's implicit synchronisation).  Its queues live in a fixed 384 MiB device array inside the
library, so it renders in waves; its images must equal pt_render's (wavefront) bit for bit -- the
tolerance every wavefront variant is held to in these tests -- on two calls in a row, sharing the
array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mixed_box(width, height):
    from paper_2605_27323_gb300 import scenes
    sc = scenes.box_scene(width=width, height=height, lift=2e-3)
    sc["mat_type"] = sc["mat_type"].copy()
    sc["mat_roughness"] = sc["mat_roughness"].copy()
    sc["mat_type"][5], sc["mat_roughness"][5] = 1, 0.25
    sc["mat_type"][6] = 2
    return sc


def test_static_scratch_render_equals_pt_render_on_two_calls():
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import capi, scenes
    from paper_2605_27323_gb300.tracer import make_camera, make_opts

    assert torch.cuda.is_available()
    lib = capi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    box = _mixed_box(96, 72)
    spheres = scenes.spheres_scene(seed=2, n_spheres=30, level=3, ground_quads=64, width=480, height=270,
                                   extent=20.0)
    # call 1: one wave; calls 2 and 3: 4.15 M paths, two waves of the static array, in the default
    # fused stage order and in the separate one
    cases = [(box, box["camera"], 4, 8, 3, "none", False), (spheres, spheres["camera"], 32, 5, 9, "material", False),
             (spheres, spheres["camera"], 32, 5, 9, "material", True)]
    for sc, cam, spp, depth, seed, sort, sep in cases:
        g = pt.Scene.from_dict(sc)
        ref = g.render(cam, spp, depth, seed, mode="wavefront", sort=sort)
        out = torch.full_like(ref, float("nan"))
        c = make_camera(cam)
        o = make_opts(mode="wavefront", sort=sort, separate_shadow=sep)
        st = lib.pt_render_wavefront_static(g.h, C.byref(c), spp, depth, seed, C.byref(o), C.c_void_p(out.data_ptr()),
                                            stream)
        assert st == 0, lib.pt_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert float(out.mean()) > 0


def test_static_scratch_handles_estimator_variants_and_two_level_scenes():
    """The same entry point with MIS and the Halton jitter, on a two-level (instanced) scene."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import capi, scenes
    from paper_2605_27323_gb300.tracer import make_camera, make_opts

    lib = capi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    sc = scenes.instanced_spheres_scene(seed=3, n_spheres=25, level=3, ground_quads=32, extent=15.0, width=200,
                                        height=120, n_materials=12)
    g = pt.Scene.from_dict(sc)
    cam = sc["camera"]
    ref = g.render(cam, 8, 6, 4, mode="wavefront", mis=True, sampler="halton")
    out = torch.full_like(ref, float("nan"))
    c = make_camera(cam)
    o = make_opts(mode="wavefront", mis=True, sampler="halton")
    st = lib.pt_render_wavefront_static(g.h, C.byref(c), 8, 6, 4, C.byref(o), C.c_void_p(out.data_ptr()), stream)
    assert st == 0, lib.pt_last_error()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_static_scratch_rejects_what_it_cannot_hold():
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import capi
    from paper_2605_27323_gb300.tracer import make_camera, make_opts

    lib = capi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    sc = _mixed_box(2, 2)
    g = pt.Scene.from_dict(sc)
    c = make_camera(sc["camera"])
    o = make_opts()
    out = torch.zeros((2, 2, 3), device="cuda")
    # one pixel's samples must fit the array: 3,000,000 x 180 B > 384 MiB
    assert lib.pt_render_wavefront_static(g.h, C.byref(c), 3_000_000, 4, 0, C.byref(o), C.c_void_p(out.data_ptr()),
                                          stream) == 1
    assert b"static scratch" in lib.pt_last_error()
    host = np.zeros((2, 2, 3), np.float32)
    assert lib.pt_render_wavefront_static(g.h, C.byref(c), 1, 4, 0, C.byref(o), host.ctypes.data_as(C.c_void_p),
                                          stream) == 1
    assert b"device memory" in lib.pt_last_error()
    # the megakernel and the hybrid continuation are not part of this entry point
    for kw in ({"mode": "megakernel"}, {"hybrid": 1000}):
        assert lib.pt_render_wavefront_static(g.h, C.byref(c), 1, 4, 0, C.byref(make_opts(**kw)),
                                              C.c_void_p(out.data_ptr()), stream) == 1, kw


def test_static_scratch_depth_zero_clears_image_and_signatures():
    """max_depth 0 renders black and zeroes the per-path signatures, as pt_render does."""
    import torch

    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import capi
    from paper_2605_27323_gb300.tracer import make_camera, make_opts

    lib = capi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    sc = _mixed_box(5, 3)
    g = pt.Scene.from_dict(sc)
    c = make_camera(sc["camera"])
    out = torch.full((3, 5, 3), 7.0, device="cuda")
    sig = torch.full((5 * 3 * 2,), -1, device="cuda", dtype=torch.int32)
    o = make_opts(sig=sig)
    assert lib.pt_render_wavefront_static(g.h, C.byref(c), 2, 0, 0, C.byref(o), C.c_void_p(out.data_ptr()),
                                          stream) == 0, lib.pt_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0 and int(sig.abs().sum()) == 0
