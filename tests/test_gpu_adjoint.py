"""GPU parity of the path-replay adjoint (gradients of an image loss with respect to per-material
albedo and emission).

* every entry against the oracle's forward-mode dual numbers on a 64x64 crop of the
  differentiable-rendering workload (the procedural spheres scene at 512x512, 64 spp, depth 6,
  256 materials);
* against central finite differences of the GPU renderer itself at h = 1e-3 on that crop, and at
  power-of-two steps on a small box (common random numbers, fixed roulette probability so the
  estimator is smooth in the parameters);
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


CROP = (224, 200, 64)          # x0, y0, width of the 64x64 crop of the 512x512 image
C5 = dict(spp=64, depth=6, seed=3)


def _crop_ids(W, spp):
    x0, y0, cw = CROP
    px = np.array([(y0 + j) * W + x0 + i for j in range(cw) for i in range(cw)], np.int64)
    return px, (px[:, None] * spp + np.arange(spp)[None, :]).reshape(-1)


def _oracle_gradients(osc, cam, ids, deltas, spp, depth, seed, nm, **kw):
    """Every entry of d(loss)/d(albedo) (nm x 3) and d(loss)/d(emission) (nm) from the oracle's
    forward-mode dual numbers, for loss = sum_p <delta, image_p> and each delta in `deltas`
    (per-path rows), 8 tangents (unit parameter directions) per pass.  Also returns, per entry, the
    sum of the magnitudes of its per-path terms."""
    nk = 8
    n_par = 4 * nm
    g = np.zeros((len(deltas), n_par))
    gabs = np.zeros((len(deltas), n_par))
    sig = None
    for k0 in range(0, n_par, nk):
        da = np.zeros((nk, nm, 3))
        de = np.zeros((nk, nm))
        for t in range(nk):
            q = k0 + t
            if q < 3 * nm:
                da[t, q // 3, q % 3] = 1.0
            else:
                de[t, q - 3 * nm] = 1.0
        o = osc.render_paths(cam, spp, depth, seed, ids, dir_albedo=da, dir_emission=de, **kw)
        sig = o["sig"] if sig is None else sig
        assert np.array_equal(sig, o["sig"])
        for i, dl in enumerate(deltas):
            terms = np.einsum("nc,nkc->nk", dl, o["dL"]) / spp
            g[i, k0:k0 + nk] = terms.sum(0)
            gabs[i, k0:k0 + nk] = np.abs(terms).sum(0)
    split = lambda a: (a[..., :3 * nm].reshape(a.shape[:-1] + (nm, 3)), a[..., 3 * nm:])
    return split(g), split(gabs), sig


def test_adjoint_matches_oracle_dual_numbers_elementwise(pt, torch):
    """All 256 x 3 albedo and 256 emission gradient entries of loss = sum over a 64x64 crop of
    <delta, image> (the inverse-rendering workload: 512x512, 64 spp, depth 6, 256 materials) against
    the oracle's dual numbers, entry by entry.  Pixels holding a path whose FP32 branches differ
    from the oracle's FP64 branches (branch signatures) get delta = 0, so both sides sum the same
    paths.  delta >= 0: every per-path term is >= 0 (each BSDF weight, Schlick's F and the emitted
    radiance grow with their parameter), so every entry above the floor must match to 1e-3 of its
    value.  Mixed-sign delta (an L2 loss's shape): entries whose terms do not cancel by more than
    10x must match to 1e-3 of their value, the others to 1e-3 of the sum of their terms' magnitudes."""
    sc = _c5_scene()
    cam = sc["camera"]
    spp, depth, seed = C5["spp"], C5["depth"], C5["seed"]
    W, H = cam["width"], cam["height"]
    nm = len(sc["mat_type"])
    g = pt.Scene.from_dict(sc)
    osc = oracle.Scene.from_dict(sc)
    px, ids = _crop_ids(W, spp)
    r = g.render(cam, spp, depth, seed, sig=True, mode="wavefront", rr_start=3)
    gsig = r["sig"].cpu().numpy().astype(np.uint32)[ids]
    o0 = osc.render_paths(cam, spp, depth, seed, ids, rr_start=3)
    same = gsig == o0["sig"]
    same_pix = same.reshape(-1, spp).all(1)
    # a few camera rays land within FP32 error of an edge: >= 99.9% of the paths take the oracle's
    # branches (with 64 samples per pixel that leaves about half a percent of the pixels masked)
    assert same.mean() >= 0.999 and same_pix.mean() >= 0.98, (same.mean(), same_pix.mean())
    rng = np.random.default_rng(1)
    deltas_img = []
    for lo in (0.1, -1.0):
        d = np.zeros((H, W, 3), np.float32)
        vals = rng.uniform(lo, 1.0, size=(px.size, 3)).astype(np.float32)
        vals[~same_pix] = 0.0
        d.reshape(-1, 3)[px] = vals
        deltas_img.append(d)
    gpu = []
    for d in deltas_img:
        ga, ge = g.backward(cam, spp, depth, seed, torch.from_numpy(d).cuda(), rr_start=3)
        assert g.stats()["status"] == 0
        gpu.append((ga.cpu().numpy().astype(np.float64), ge.cpu().numpy().astype(np.float64)))
    per_path = [d.reshape(-1, 3)[ids // spp].astype(np.float64) for d in deltas_img]
    (oa, oe), (aa, ae), osig = _oracle_gradients(osc, cam, ids, per_path, spp, depth, seed, nm, rr_start=3)
    assert np.array_equal(osig, o0["sig"])
    report = []
    for i, kind in enumerate(("positive", "mixed")):
        for name, gv, ov, av in (("albedo", gpu[i][0], oa[i], aa[i]), ("emission", gpu[i][1], oe[i], ae[i])):
            floor = 1e-6 * np.abs(ov).max()
            big = np.abs(ov) > floor
            if kind == "positive":
                assert np.all(ov >= 0) and np.all(gv >= -floor), (name, ov.min(), gv.min())
                scale = np.abs(ov)
            else:
                scale = np.where(np.abs(ov) >= 0.1 * av, np.abs(ov), av)
            err = np.abs(gv - ov)
            rel = np.where(big, err / np.maximum(scale, 1e-300), 0.0)
            report.append((kind, name, int(big.sum()), float(rel.max())))
            assert np.all(err[big] <= GRAD_RTOL * scale[big]), (kind, name, float(rel.max()), report)
            assert np.all(np.abs(gv[~big]) <= 2 * floor + GRAD_RTOL * av[~big]), (kind, name)
    # the check covers many entries, not just a few large ones
    assert report[0][2] >= 100 and report[1][2] >= 10, report


def test_adjoint_matches_central_differences_on_crop(pt, torch):
    """Central differences at h = 1e-3 on the same crop, with common random numbers: the image is
    rendered again with one parameter moved by +-h (the step is taken as the difference of the two
    FP32 parameter values).  A fixed roulette probability keeps every branch independent of the
    parameters, so the image is a polynomial in the albedos and linear in the emissions."""
    sc = _c5_scene()
    cam = sc["camera"]
    spp, depth, seed = C5["spp"], C5["depth"], C5["seed"]
    W, H = cam["width"], cam["height"]
    opts = dict(rr_start=3, rr_fixed=0.8)
    g = pt.Scene.from_dict(sc)
    px, _ = _crop_ids(W, spp)
    rng = np.random.default_rng(5)
    delta = np.zeros((H, W, 3), np.float32)
    delta.reshape(-1, 3)[px] = rng.uniform(0.1, 1.0, size=(px.size, 3)).astype(np.float32)
    ga, ge = g.backward(cam, spp, depth, seed, torch.from_numpy(delta).cuda(), **opts)
    ga, ge = ga.cpu().numpy().astype(np.float64), ge.cpu().numpy().astype(np.float64)
    A0 = sc["mat_albedo"].astype(np.float32).copy()
    E0 = sc["mat_emission"].astype(np.float32).copy()
    d64 = delta.astype(np.float64)

    def loss(A, E):
        g.set_materials(torch.from_numpy(A).cuda(), torch.from_numpy(E).cuda())
        img = g.render(cam, spp, depth, seed, mode="wavefront", **opts).cpu().numpy().astype(np.float64)
        return float((img * d64).sum())

    h = 1e-3
    top_a = np.argsort(-np.abs(ga).reshape(-1))[:4]
    checks = [("a", int(q // 3), int(q % 3)) for q in top_a]
    checks += [("e", int(m), 0) for m in np.argsort(-np.abs(ge))[:3]]
    try:
        for kind, m, c in checks:
            A, E = A0.copy(), E0.copy()
            arr, idx = (A, (m, c)) if kind == "a" else (E, (m,))
            base = float(arr[idx])
            arr[idx] = np.float32(base + h)
            hi = float(arr[idx])
            lp = loss(A, E)
            arr[idx] = np.float32(base - h)
            lo = float(arr[idx])
            lm = loss(A, E)
            fd = (lp - lm) / (hi - lo)
            ad = ga[m, c] if kind == "a" else ge[m]
            assert abs(fd - ad) <= GRAD_RTOL * max(abs(fd), abs(ad)), (kind, m, c, fd, ad)
            assert ad > 0
    finally:
        g.set_materials(torch.from_numpy(A0).cuda(), torch.from_numpy(E0).cuda())


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
