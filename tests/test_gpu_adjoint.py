"""GPU parity of the path-replay adjoint (gradients of an image loss with respect to per-material
albedo and emission).

* against the oracle's forward-mode dual numbers on a 64x64 crop of the differentiable-rendering
  workload (the procedural spheres scene at 512x512, 64 spp, depth 6, 256 materials);
* against central finite differences of the GPU renderer itself (common random numbers, fixed
  roulette probability so the estimator is smooth in the parameters, parameter steps exact in FP32);
* through torch.autograd with an L2 loss against a target rendered from hidden parameters.
Relative error <= 1e-3 throughout.
"""
import numpy as np
import pytest

import oracle
from paper_2605_27323_gb300 import scenes

pytestmark = pytest.mark.gpu
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need CUDA"
    return T


@pytest.fixture(scope="module")
def pt(torch):
    import paper_2605_27323_gb300 as P
    return P


def _c5_scene():
    return scenes.spheres_scene(seed=0, n_materials=256, width=512, height=512)


@pytest.mark.parametrize("signs", ["positive", "mixed"])
def test_adjoint_matches_oracle_dual_numbers_on_crop(pt, torch, signs):
    """d(loss)/d(theta) . v for four directions v against the oracle's dual numbers, with
    loss = sum over a 64x64 crop of <delta, image>.  With delta >= 0 the gradient is a sum of
    like-signed terms and must match to 1e-3 of its value.  With mixed signs (as in an L2 loss) it is
    a cancelling sum, and its relative error is measured against the sum of the terms' magnitudes,
    sum_p |delta_p . dL_p/dv| / spp (the few paths whose FP32 and FP64 branches differ each move it by
    a full term)."""
    sc = _c5_scene()
    cam = sc["camera"]
    spp, depth, seed = 64, 6, 3
    W, H = cam["width"], cam["height"]
    g = pt.Scene.from_dict(sc)
    osc = oracle.Scene.from_dict(sc)
    rng = np.random.default_rng(1)
    x0, y0, cw = 224, 200, 64
    lo = 0.0 if signs == "positive" else -1.0
    delta = np.zeros((H, W, 3), np.float32)
    delta[y0:y0 + cw, x0:x0 + cw] = rng.uniform(lo, 1.0, size=(cw, cw, 3)).astype(np.float32)
    ga, ge = g.backward(cam, spp, depth, seed, torch.from_numpy(delta).cuda(), rr_start=3)
    ga, ge = ga.cpu().numpy().astype(np.float64), ge.cpu().numpy().astype(np.float64)
    assert g.stats()["status"] == 0
    nm = len(sc["mat_type"])
    nd = 4
    da = np.zeros((nd, nm, 3))
    de = np.zeros((nd, nm))
    da[0] = rng.uniform(0.0, 1.0, size=(nm, 3))      # an all-positive albedo direction
    de[1] = rng.uniform(0.0, 1.0, size=nm)           # an all-positive emission direction
    m_top = int(np.argmax(np.abs(ga).sum(1)))
    da[2, m_top] = [1.0, 0.0, 0.0]                   # the most influential albedo, one channel
    de[3, nm - 1] = 1.0                              # the lights' emission
    px = np.array([(y0 + j) * W + x0 + i for j in range(cw) for i in range(cw)], np.int64)
    ids = (px[:, None] * spp + np.arange(spp)[None, :]).reshape(-1)
    o = osc.render_paths(cam, spp, depth, seed, ids, rr_start=3, dir_albedo=da, dir_emission=de)
    dflat = delta.reshape(-1, 3)[ids // spp].astype(np.float64)
    terms = np.einsum("nc,nkc->nk", dflat, o["dL"]) / spp
    oracle_dd = terms.sum(0)
    scale = np.abs(oracle_dd) if signs == "positive" else np.abs(terms).sum(0)
    gpu_dd = np.array([(ga * da[k]).sum() + (ge * de[k]).sum() for k in range(nd)])
    for k in range(nd):
        assert abs(gpu_dd[k] - oracle_dd[k]) <= GRAD_RTOL * scale[k] + 1e-9, (k, gpu_dd, oracle_dd, scale)
    assert np.all(np.abs(oracle_dd) > 0)


def _fd_box():
    sc = scenes.box_scene(width=48, height=48, lift=2e-3)
    sc["mat_type"] = sc["mat_type"].copy()
    sc["mat_roughness"] = sc["mat_roughness"].copy()
    sc["mat_type"][5] = 1
    sc["mat_roughness"][5] = 0.3
    sc["mat_type"][6] = 2
    # parameters on a 2^-16 grid so that theta +- 2^-8 is exact in FP32
    sc["mat_albedo"] = (np.round(sc["mat_albedo"].astype(np.float64) * 2 ** 16) / 2 ** 16).astype(np.float32)
    sc["mat_albedo"][6] = [0.875, 0.9375, 1.0]
    return sc


def test_adjoint_matches_central_differences(pt, torch):
    sc = _fd_box()
    cam = sc["camera"]
    spp, depth, seed = 16, 6, 5
    opts = dict(rr_start=2, rr_fixed=0.8)
    g = pt.Scene.from_dict(sc)
    rng = np.random.default_rng(2)
    delta = rng.uniform(0.0, 1.0, size=(48, 48, 3)).astype(np.float32)
    ga, ge = g.backward(cam, spp, depth, seed, torch.from_numpy(delta).cuda(), **opts)
    ga, ge = ga.cpu().numpy().astype(np.float64), ge.cpu().numpy().astype(np.float64)
    A0 = torch.from_numpy(sc["mat_albedo"].copy()).cuda()
    E0 = torch.from_numpy(sc["mat_emission"].copy()).cuda()

    def loss(A, E):
        g.set_materials(A, E)
        img = g.render(cam, spp, depth, seed, mode="wavefront", **opts).cpu().numpy().astype(np.float64)
        return float((img * delta).sum())

    h = 2.0 ** -8
    checks = [("a", 2, 0), ("a", 5, 1), ("a", 6, 2), ("a", 0, 1), ("e", 7, 0), ("e", 3, 0)]
    for kind, m, c in checks:
        A, E = A0.clone(), E0.clone()
        if kind == "a":
            A[m, c] += h
            lp = loss(A, E)
            A[m, c] -= 2 * h
            lm = loss(A, E)
            fd, ad = (lp - lm) / (2 * h), ga[m, c]
        else:
            E[m] += 8 * h
            lp = loss(A, E)
            E[m] -= 16 * h
            lm = loss(A, E)
            fd, ad = (lp - lm) / (16 * h), ge[m]
        assert abs(fd - ad) <= GRAD_RTOL * max(abs(fd), abs(ad)) + 1e-6, (kind, m, c, fd, ad)
    g.set_materials(A0, E0)


def test_autograd_l2_loss_against_hidden_target(pt, torch):
    sc = _c5_scene()
    cam = dict(sc["camera"], width=128, height=128)
    spp, depth = 8, 6
    g = pt.Scene.from_dict(sc)
    nm = len(sc["mat_type"])
    hidden = np.random.default_rng(7)
    A_t = torch.from_numpy(hidden.uniform(0.1, 0.9, size=(nm, 3)).astype(np.float32)).cuda()
    E_t = torch.from_numpy(sc["mat_emission"] * hidden.uniform(0.5, 1.5, size=nm).astype(np.float32)).cuda()
    with torch.no_grad():
        target = pt.render_differentiable(A_t, E_t, g, cam, spp, depth, 1)
    A = torch.from_numpy(sc["mat_albedo"].copy()).cuda().requires_grad_(True)
    E = torch.from_numpy(sc["mat_emission"].copy()).cuda().requires_grad_(True)
    img = pt.render_differentiable(A, E, g, cam, spp, depth, 2)
    loss = ((img - target) ** 2).sum()
    loss.backward()
    ga, ge = g.backward(cam, spp, depth, 2, (2.0 * (img - target)).detach())
    assert torch.allclose(A.grad, ga, rtol=1e-5, atol=1e-7)
    assert torch.allclose(E.grad, ge, rtol=1e-5, atol=1e-7)
    assert float(A.grad.abs().sum()) > 0


@pytest.mark.parametrize("spp,depth,rr", [(4, 6, 0.0), (1, 12, 0.8), (2, 24, 0.9), (3, 32, 0.95)])
def test_wavefront_and_megakernel_replays_agree(pt, torch, spp, depth, rr):
    """The two replays of the adjoint (wavefront stages writing vertex records, and one thread per
    path with thread-local records and path regeneration) compute the same gradients; only the
    order of the FP32 atomic additions differs.  Depths 12, 24 and 32 take the 16- and 32-vertex
    record arrays of the one-thread-per-path replay."""
    sc = _c5_scene()
    cam = dict(sc["camera"], width=160, height=90)
    g = pt.Scene.from_dict(sc)
    rng = np.random.default_rng(3)
    delta = torch.from_numpy(rng.uniform(0.0, 1.0, size=(90, 160, 3)).astype(np.float32)).cuda()
    ga_w, ge_w = g.backward(cam, spp, depth, 4, delta, rr_start=2, rr_fixed=rr, mode="wavefront")
    ga_m, ge_m = g.backward(cam, spp, depth, 4, delta, rr_start=2, rr_fixed=rr, mode="megakernel")
    assert torch.allclose(ga_w, ga_m, rtol=1e-4, atol=1e-6 * float(ga_m.abs().max()))
    assert torch.allclose(ge_w, ge_m, rtol=1e-4, atol=1e-6 * float(ge_m.abs().max()))
    assert float(ga_w.abs().sum()) > 0


def test_backward_argument_errors(pt, torch):
    from paper_2605_27323_gb300 import capi
    sc = scenes.box_scene(width=8, height=8)
    g = pt.Scene.from_dict(sc)
    grad = torch.zeros((8, 8, 3), device="cuda")
    with pytest.raises(capi.PtError) as e:
        g.backward(sc["camera"], 1, 33, 0, grad)
    assert e.value.status == 7
    ga, ge = g.backward(sc["camera"], 1, 0, 0, grad)
    assert float(ga.abs().sum()) == 0 and float(ge.abs().sum()) == 0
