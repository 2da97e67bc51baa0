"""Pins of the oracle's multiple importance sampling (power heuristic, Veach 1997) between
next-event estimation and BSDF-sampled light hits.

* the BSDF sampling density used in the weights is the density bsdf_sample actually draws from:
  it integrates to the probability of a valid sample, and binned sample counts match its integral
  over each bin (Lambert and GGX);
* the MIS estimator keeps the closed forms: the point-to-rectangle form factor of direct lighting
  (tests/golden) and the white-furnace series;
* MIS and NEE alone have the same expectation on a glossy plane under a large light, and MIS has
  the much lower variance that motivates it there.
"""
import os

import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes
from test_oracle_estimator import _point_ff, _rows, _sphere_rays

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _hemisphere_grid(n_t=96, n_p=192):
    # midpoint grid in (cos theta, phi): equal solid angle 2 pi / (n_t n_p) per cell
    ct = (np.arange(n_t) + 0.5) / n_t
    ph = (np.arange(n_p) + 0.5) / n_p * 2 * np.pi
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C * C)
    return np.stack([S * np.cos(P), S * np.sin(P), C], -1), 2 * np.pi / (n_t * n_p)


# (the midpoint grid resolves lobes down to roughness ~0.3; the formula is the same for every roughness)
@pytest.mark.parametrize("mtype,rough,wo", [(0, 0.5, (0.3, 0.1, 0.95)), (1, 0.3, (0.5, 0.2, 0.84)),
                                            (1, 0.6, (0.9, 0.0, 0.3)), (1, 0.35, (0.8, -0.3, 0.52))])
def test_bsdf_pdf_is_the_sampling_density(oracle_lib, mtype, rough, wo):
    n = np.array([0.0, 0.0, 1.0])
    wo = np.asarray(wo, np.float64)
    wo /= np.linalg.norm(wo)
    grid, dw = _hemisphere_grid()
    pdf = np.array([[oracle_lib.bsdf_pdf(mtype, rough, n, wo, w) for w in row] for row in grid])
    rng = np.random.default_rng(7)
    m = 60000
    dirs, valid = [], 0
    for u in rng.uniform(size=(m, 3)):
        ok, wi, _, _ = oracle_lib.bsdf_sample(mtype, [0.5, 0.5, 0.5], rough, 1.5, n, n, wo, *u)
        if ok:
            valid += 1
            dirs.append(wi)
    dirs = np.array(dirs)
    # total probability of a valid sample
    assert abs(pdf.sum() * dw - valid / m) < 4 * np.sqrt(valid / m * (1 - valid / m) / m) + 3e-3
    # coarse bins: 8 in cos theta x 8 in phi; expected mass from the fine grid
    bt = np.minimum((dirs[:, 2] * 8).astype(int), 7)
    bp = np.minimum(((np.arctan2(dirs[:, 1], dirs[:, 0]) % (2 * np.pi)) / (2 * np.pi) * 8).astype(int), 7)
    counts = np.zeros((8, 8))
    np.add.at(counts, (bt, bp), 1)
    mass = pdf.reshape(8, 12, 8, 24).sum((1, 3)) * dw * m
    big = mass > 50
    z = (counts[big] - mass[big]) / np.sqrt(mass[big])
    assert np.max(np.abs(z)) < 5.0, np.max(np.abs(z))
    assert np.mean(z ** 2) < 2.0


@pytest.mark.parametrize("px,pz,hw,hh,c", [tuple(r) for r in _rows("form_factor_parallel_rect.txt")][:4])
def test_mis_keeps_the_form_factor(oracle_lib, px, pz, hw, hh, c):
    rho, Le = 0.7, 5.0
    sc = oracle_lib.Scene.from_dict(scenes.rect_over_plane(albedo=rho, emission=Le, half_w=hw, half_h=hh,
                                                           height=c))
    n = 100_000
    o = np.tile([px, 0.5 * c, pz], (n, 1))
    d = np.tile([0.0, -1.0, 0.0], (n, 1))
    L, _ = sc.trace_rays(o, d, np.arange(n), max_depth=2, mis=True)
    expect = rho * Le * _point_ff(px, pz, hw, hh, c)
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(n)
    assert abs(m - expect) < 4 * se + 1e-4 * expect, (m, se, expect)


@pytest.mark.parametrize("a,D,expect", [tuple(r) for r in _rows("furnace.txt")][:3])
def test_mis_keeps_the_furnace_series(oracle_lib, a, D, expect):
    sc = oracle_lib.Scene.from_dict(scenes.furnace_sphere(albedo=a, emission=1.0, level=4))
    o, d = _sphere_rays(20000, 4)
    L, _ = sc.trace_rays(o, d, np.arange(20000), max_depth=int(D), mis=True)
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(len(L))
    assert abs(m - expect) < 3 * se + 2e-3 * expect, (m, se, expect)


def test_mis_on_glossy_plane_same_mean_lower_variance(oracle_lib):
    s = scenes.rect_over_plane(albedo=0.9, emission=5.0, half_w=2.0, half_h=2.0, height=1.0)
    s["mat_type"] = np.asarray(s["mat_type"]).copy()
    s["mat_roughness"] = np.asarray(s["mat_roughness"], np.float32).copy()
    s["mat_type"][0] = scenes.GGX
    s["mat_roughness"][0] = 0.2
    sc = oracle_lib.Scene.from_dict(s)
    n = 100_000
    o = np.tile([-0.6, 0.6, 0.0], (n, 1))
    d = np.tile(np.array([0.6, -0.6, 0.0]) / np.sqrt(0.72), (n, 1))     # mirror direction enters the light
    L_nee, _ = sc.trace_rays(o, d, np.arange(n), max_depth=2)
    L_mis, _ = sc.trace_rays(o, d, np.arange(n), max_depth=2, mis=True)
    m1, s1 = L_nee[:, 0].mean(), L_nee[:, 0].std()
    m2, s2 = L_mis[:, 0].mean(), L_mis[:, 0].std()
    assert abs(m1 - m2) < 4 * np.sqrt((s1 ** 2 + s2 ** 2) / n), (m1, m2, s1, s2)
    assert s2 < 0.5 * s1, (s1, s2)
