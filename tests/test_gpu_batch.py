"""Batched rendering: many scenes of uneven triangle counts, resolutions and spp in one persistent
wavefront (pt_render_batch).  Each image must equal its standalone pt_render image bit for bit
(same kernels and random numbers; a pixel whose samples fall in two waves continues its FP32 sum),
with and without the CUDA-graph bounce loop, with key sorting, and with the autotuner's choice; and
in one test the chain batch == standalone == FP64 oracle (per path) is checked end to end."""
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
def specs():
    return [  # (scene, width, height, spp)
        (scenes.box_scene(width=1, height=1), 1, 1, 7),
        (scenes.spheres_scene(seed=3, n_spheres=12, level=2, ground_quads=16, extent=10.0), 61, 37, 3),
        (scenes.box_scene(seed=5), 40, 30, 16),
        (scenes.spheres_scene(seed=4, n_spheres=60, level=3, ground_quads=64, extent=20.0), 200, 113, 1),
        (scenes.spheres_scene(seed=6, n_spheres=5, level=1, ground_quads=4, extent=5.0), 17, 90, 4),
    ]


@pytest.fixture(scope="module")
def batch(torch, specs):
    import paper_2605_27323_gb300 as pt
    out = []
    for sc, w, h, spp in specs:
        cam = dict(sc["camera"], width=w, height=h)
        out.append((pt.Scene.from_dict(sc), cam, spp))
    return out


def _standalone(batch, depth, seed, **kw):
    return [g.render(cam, spp, depth, seed, mode="wavefront", **kw).cpu().numpy() for g, cam, spp in batch]


@pytest.mark.parametrize("kw", [{}, {"graph": False}, {"queue_capacity": 997}, {"queue_capacity": 5000, "sort": "material"},
                                {"sort": "type", "block_size": 128}, {"separate_shadow": True, "queue_capacity": 2000}])
def test_batch_equals_standalone_renders(torch, batch, kw):
    import paper_2605_27323_gb300 as pt
    depth, seed = 6, 11
    ref = _standalone(batch, depth, seed)
    outs = pt.render_batch([g for g, _, _ in batch], [c for _, c, _ in batch], [s for _, _, s in batch], depth, seed,
                           **kw)
    for i, (o, r) in enumerate(zip(outs, ref)):
        assert np.array_equal(o.cpu().numpy(), r), (i, kw)
    # a second call reuses the captured graph with another seed
    ref2 = _standalone(batch, depth, seed + 1)
    outs2 = pt.render_batch([g for g, _, _ in batch], [c for _, c, _ in batch], [s for _, _, s in batch], depth,
                            seed + 1, **kw)
    for o, r in zip(outs2, ref2):
        assert np.array_equal(o.cpu().numpy(), r)


def test_batch_equals_standalone_equals_oracle(torch, batch, specs):
    """One chain in one test: every batch image equals its standalone render bit for bit, and the
    standalone renders of three of the scenes (a box and two sphere scenes, ragged sizes, 1-16 spp)
    match the FP64 oracle path by path (the parity contract of the single-scene tests).  Scene 1 is
    left out of the oracle leg: at its small extent its eight light quads overlap in one plane, so
    about 0.6% of its paths hit two coplanar triangles at the same distance -- a near-tie, decided by
    rounding, that the contract excludes (the event logs of every such path differ only in which of
    the coplanar light triangles was hit)."""
    import oracle
    import paper_2605_27323_gb300 as pt
    from helpers import compare_with_oracle
    depth, seed = 6, 11
    outs = pt.render_batch([g for g, _, _ in batch], [c for _, c, _ in batch], [s for _, _, s in batch], depth, seed)
    for i in (2, 3, 4):
        g, cam, spp = batch[i]
        r = g.render(cam, spp, depth, seed, mode="wavefront", path_L=True, sig=True)
        assert np.array_equal(outs[i].cpu().numpy(), r["img"].cpu().numpy()), i
        n = cam["width"] * cam["height"] * spp
        o = oracle.Scene.from_dict(specs[i][0]).render_paths(cam, spp, depth, seed, np.arange(n), rr_start=3)
        compare_with_oracle(r["path_L"].cpu().numpy(), r["sig"].cpu().numpy(), o["L"], o["sig"], spp,
                            label=f"batch scene {i}")


def test_autotuner_choice_renders_the_same(torch, batch):
    import paper_2605_27323_gb300 as pt
    depth, seed = 5, 2
    gs, cams, spps = [g for g, _, _ in batch], [c for _, c, _ in batch], [s for _, _, s in batch]
    best = pt.autotune_batch(gs, cams, spps, depth, seed)
    assert best["ms"] > 0 and best["block_size"] in (128, 256) and best["sort"] in (0, 1, 2)
    assert best["queue_capacity"] >= 1
    outs = pt.render_batch(gs, cams, spps, depth, seed, queue_capacity=best["queue_capacity"],
                           block_size=best["block_size"], sort=int(best["sort"]))
    for o, r in zip(outs, _standalone(batch, depth, seed)):
        assert np.array_equal(o.cpu().numpy(), r)


def test_batch_argument_errors(torch, batch):
    import paper_2605_27323_gb300 as pt
    from paper_2605_27323_gb300 import capi
    g, cam, spp = batch[0]
    with pytest.raises(capi.PtError):
        pt.render_batch([g], [cam], [0], 4, 0)
    host = [torch.zeros((1, 1, 3))]
    with pytest.raises(capi.PtError):
        pt.render_batch([g], [cam], [1], 4, 0, outs=host)
    with pytest.raises(capi.PtError):
        pt.render_batch([g], [cam], [1], 65, 0)
