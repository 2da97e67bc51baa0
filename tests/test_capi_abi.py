"""The C-ABI library builds, loads and exports every function include/pt.h declares; argument
validation errors come back as status codes without touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2605_27323_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pt.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_list():
    assert _declared() == sorted(capi.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = capi.load()
    path = capi.lib_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (pt_[a-z_]+)$", out, flags=re.M))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)


def test_status_strings():
    lib = capi.load()
    names = {0: b"ok", 1: b"invalid argument", 2: b"out of memory", 3: b"CUDA error", 4: b"queue overflow",
             5: b"traversal limit exceeded", 6: b"timeout", 7: b"unsupported"}
    for k, v in names.items():
        assert lib.pt_status_string(k) == v
    assert lib.pt_status_string(99) == b"unknown status"


def test_struct_layouts_match_header():
    assert C.sizeof(capi.Material) == 32
    assert C.sizeof(capi.Camera) == 48
    assert C.sizeof(capi.RenderOpts) == 48
    assert capi.RenderOpts.queue_capacity.offset == 24 and capi.RenderOpts.d_path_sig.offset == 32


def test_argument_validation_on_host():
    lib = capi.load()
    # NULL out pointer and NULL scene are rejected before any CUDA call
    assert lib.pt_scene_create(None, 0, None, 0, None, None, 0, None, None, None) == 1
    assert b"out is NULL" in lib.pt_last_error()
    h = C.c_void_p()
    assert lib.pt_scene_create(None, 0, None, 5, None, None, 0, None, None, C.byref(h)) == 1
    assert h.value is None
    cam = capi.Camera()
    assert lib.pt_render(None, C.byref(cam), 1, 1, 0, None, None, None, None) == 1
    assert lib.pt_render_backward(None, C.byref(cam), 1, 1, 0, None, None, None, None, None) == 1
    st = capi.Stats()
    assert lib.pt_get_stats(None, C.byref(st)) == 1
    # out-of-range indices / materials are reported with the offending item
    import numpy as np
    v = np.zeros((3, 3), np.float32)
    t = np.array([[0, 1, 5]], np.uint32)
    m = np.zeros(1, np.uint32)
    mats = (capi.Material * 1)()
    mats[0].ior = 1.5
    assert lib.pt_scene_create(v.ctypes.data, 3, t.ctypes.data, 1, m.ctypes.data, mats, 1, None, None,
                               C.byref(h)) == 1
    assert b"vertex 5" in lib.pt_last_error()
    t = np.array([[0, 1, 2]], np.uint32)
    mats[0].type = 9
    assert lib.pt_scene_create(v.ctypes.data, 3, t.ctypes.data, 1, m.ctypes.data, mats, 1, None, None,
                               C.byref(h)) == 1
    assert b"unknown type" in lib.pt_last_error()
    mats[0].type = 0
    mats[0].emission = -1.0
    assert lib.pt_scene_create(v.ctypes.data, 3, t.ctypes.data, 1, m.ctypes.data, mats, 1, None, None,
                               C.byref(h)) == 1
    v[0, 0] = np.nan
    mats[0].emission = 0.0
    assert lib.pt_scene_create(v.ctypes.data, 3, t.ctypes.data, 1, m.ctypes.data, mats, 1, None, None,
                               C.byref(h)) == 1
    assert b"not finite" in lib.pt_last_error()


def test_no_cpu_fallback_in_product_path():
    # the product package never imports the oracle
    pkg = os.path.join(ROOT, "paper_2605_27323_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_struct_layouts_match_a_compiled_header(tmp_path):
    """sizeof and offsetof of every ABI struct, from a C program compiled against include/pt.h,
    against the ctypes mirrors."""
    fields = {"pt_material": ("Material", ["type", "albedo", "emission", "roughness", "ior", "flags"]),
              "pt_camera": ("Camera", ["eye", "target", "up", "vfov_deg", "width", "height"]),
              "pt_render_opts": ("RenderOpts", ["mode", "rr_start", "rr_fixed", "sort_mode", "block_size", "flags",
                                                "queue_capacity", "d_path_sig", "hybrid_threshold"]),
              "pt_instance": ("Instance", ["xform", "mesh", "material", "reserved"]),
              "pt_stats": ("Stats", ["extension_rays", "shadow_rays", "paths", "bounces", "status", "active",
                                     "ms_raygen", "ms_adjoint", "launches_extend", "launches_total", "ms_total",
                                     "nodes_closest", "tris_any", "shadow_queued", "group_walks"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pt.h"', "int main(void) {"]
    for cname, (_, fs) in fields.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fs:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, (pyname, fs) in fields.items():
        cls = getattr(capi, pyname)
        assert C.sizeof(cls) == got[(cname, "size")], cname
        for f in fs:
            assert getattr(cls, f).offset == got[(cname, f)], (cname, f)


def test_instanced_scene_validation_on_host():
    lib = capi.load()
    h = C.c_void_p()
    # no meshes / no instances are rejected before any CUDA call
    assert lib.pt_scene_create_instanced(0, None, None, None, None, None, None, 0, None, 0, None, None,
                                         C.byref(h)) == 1
    assert b"mesh" in lib.pt_last_error()
    import numpy as np
    v = np.zeros((3, 3), np.float32)
    t = np.array([[0, 1, 2]], np.uint32)
    m = np.zeros(1, np.uint32)
    vp = (C.c_void_p * 1)(v.ctypes.data)
    tp = (C.c_void_p * 1)(t.ctypes.data)
    mp = (C.c_void_p * 1)(m.ctypes.data)
    nv = (C.c_uint32 * 1)(3)
    nt = (C.c_uint32 * 1)(1)
    mats = (capi.Material * 1)()
    mats[0].ior = 1.5
    inst = (capi.Instance * 1)()
    inst[0].mesh = 3                                      # out of range
    assert lib.pt_scene_create_instanced(1, vp, nv, tp, nt, mp, inst, 1, mats, 1, None, None, C.byref(h)) == 1
    assert b"mesh 3" in lib.pt_last_error()
    inst[0].mesh = 0
    inst[0].material = 7                                  # out of range
    assert lib.pt_scene_create_instanced(1, vp, nv, tp, nt, mp, inst, 1, mats, 1, None, None, C.byref(h)) == 1
    assert b"material 7" in lib.pt_last_error()
    inst[0].material = capi.NO_MATERIAL                   # identity not set: the zero transform is singular
    assert lib.pt_scene_create_instanced(1, vp, nv, tp, nt, mp, inst, 1, mats, 1, None, None, C.byref(h)) == 1
    assert b"singular" in lib.pt_last_error()
    assert h.value is None
