"""The per-stage timings the library records when asked (`profile=True`): stages are the intervals
between events on the launch stream, consecutive stages sharing the event between them.

* a wavefront frame's stage times are positive and add up to the frame as timed by events around
  the call (the stages tile the frame; only the work before the first stage lies outside them): in
  the default (fused) order one extend interval per bounce, each holding the previous bounce's shadow
  walks, and no separate shadow interval; in the separate order (PT_FLAG_SEPARATE_SHADOW) one extend
  and one shadow interval per bounce (the bounce loop runs to the maximum depth; counts stay on the
  device);
* a megakernel frame is one megakernel interval; an adjoint pass is one adjoint interval that
  contains its replay's stages;
* profiling does not change the image.
"""
import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


@pytest.fixture(scope="module")
def setup(torch):
    import paper_2605_27323_gb300 as pt
    sc = scenes.spheres_scene(seed=3, n_spheres=40, level=3, ground_quads=64, extent=20.0, width=320, height=240)
    return sc, pt.Scene.from_dict(sc)


def _timed(torch, fn):
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    r = fn()
    b.record(st)
    b.synchronize()
    return r, a.elapsed_time(b)


@pytest.mark.parametrize("separate", [False, True])
def test_wavefront_stages_tile_the_frame(torch, setup, separate):
    sc, g = setup
    cam = sc["camera"]
    plain = g.render(cam, 4, 6, 11, mode="wavefront")
    img, outer = _timed(torch, lambda: g.render(cam, 4, 6, 11, mode="wavefront", profile=True,
                                                separate_shadow=separate))
    s = g.stats()
    assert np.array_equal(plain.cpu().numpy(), img.cpu().numpy())
    for k in ("ms_raygen", "ms_extend", "ms_shade", "ms_reduce") + (("ms_shadow",) if separate else ()):
        assert s[k] > 0.0, k
    assert s["ms_megakernel"] == 0.0 and s["ms_adjoint"] == 0.0
    assert s["launches_extend"] == 6 and s["launches_shadow"] == (6 if separate else 0) and s["bounces"] >= 4
    staged = s["ms_raygen"] + s["ms_extend"] + s["ms_sort"] + s["ms_shade"] + s["ms_shadow"] + s["ms_reduce"]
    assert abs(s["ms_total"] - staged) <= 1e-3 * staged
    assert staged <= outer * 1.001 + 1e-3
    assert staged >= 0.8 * outer, (staged, outer)


def test_megakernel_and_adjoint_intervals(torch, setup):
    sc, g = setup
    cam = sc["camera"]
    _, outer = _timed(torch, lambda: g.render(cam, 4, 6, 11, mode="megakernel", profile=True))
    s = g.stats()
    assert 0.0 < s["ms_megakernel"] <= outer * 1.001 + 1e-3
    assert s["ms_extend"] == 0.0 and s["launches_extend"] == 0
    grad = torch.ones((cam["height"], cam["width"], 3), device="cuda")
    _, outer = _timed(torch, lambda: g.backward(cam, 4, 6, 11, grad, profile=True))
    s = g.stats()
    inner = s["ms_raygen"] + s["ms_extend"] + s["ms_shade"] + s["ms_shadow"] + s["ms_reduce"]
    assert s["launches_extend"] > 0 and inner > 0.0
    assert inner <= s["ms_adjoint"] * 1.001 + 1e-3
    assert s["ms_adjoint"] <= outer * 1.001 + 1e-3
