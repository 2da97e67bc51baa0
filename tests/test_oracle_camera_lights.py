"""Oracle pins of the ray-generation step (Sec. 2.3, Sec. 2.2 step 1) and of the light pick of the
shadow-evaluation stage (Sec. 3), against pinhole geometry and the area-proportional light pmf.

Camera: the pinhole camera is fixed by eye, target, up, the full vertical field of view and the
image size, with row 0 at the top and +x to the right.  Its facts, checked without the oracle's own
formula: the ray through the image centre points at the target; the rays through the middle of the
top and left image edges make the vertical half-angle vfov/2 and the horizontal half-angle
atan(tan(vfov/2) W/H) with the view axis, above and to the left of it; pixels are square on the
image plane (one pitch, 2 tan(vfov/2) / H, in both directions); rows go down and columns go right;
every ray starts at the eye and has unit length.

Light pick: light j (the j-th emissive triangle in ascending id) is drawn with probability
area_j / total area.  Checked by counting picks over 10^6 uniforms on the 2^-24 grid (chi-square),
and through the estimator: a rectangle light cut into six triangles of very unequal area must still
give the closed-form irradiance of the rectangle (a count-uniform pick, or a pick off by one index,
does not).

Each pin must fail on a copy of the oracle with a planted mistake (test_planted_*).
"""
import math
import os

import numpy as np
import pytest

from paper_2605_27323_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")

CAMERAS = [  # eye, target, up (not orthogonal to the view), vfov, W, H
    dict(eye=(1.5, 2.0, -3.0), target=(-0.5, 0.25, 1.0), up=(0.2, 1.0, 0.3), vfov_deg=50.0, width=64, height=36),
    dict(eye=(0.0, 0.0, 5.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), vfov_deg=30.0, width=33, height=51),
    dict(eye=(-2.0, 7.0, 1.0), target=(3.0, -1.0, 2.0), up=(0.0, 0.0, 1.0), vfov_deg=110.0, width=20, height=10),
]


def _frame(cam):
    e = np.asarray(cam["eye"], np.float32).astype(np.float64)
    t = np.asarray(cam["target"], np.float32).astype(np.float64)
    up = np.asarray(cam["up"], np.float32).astype(np.float64)
    f = (t - e) / np.linalg.norm(t - e)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    return e, f, r, np.cross(r, f)


def _angle(a, b):
    return math.atan2(np.linalg.norm(np.cross(a, b)), float(np.dot(a, b)))


def camera_failures(oracle, cam):
    """Every pinhole fact the oracle's camera violates (empty list: all hold)."""
    fails = []
    W, H = cam["width"], cam["height"]
    e, f, r, u = _frame(cam)
    half_v = math.radians(cam["vfov_deg"]) / 2
    half_h = math.atan(math.tan(half_v) * W / H)
    tol = 1e-12

    def ray(x, y, u0, u1):
        o, d = oracle.camera_rays(cam, [y * W + x], [u0], [u1])
        return o[0], d[0]

    # image centre: a pixel corner for even sizes, a pixel centre for odd sizes
    cx, cu = (W // 2, 0.0) if W % 2 == 0 else ((W - 1) // 2, 0.5)
    cy, cv = (H // 2, 0.0) if H % 2 == 0 else ((H - 1) // 2, 0.5)
    o, d = ray(cx, cy, cu, cv)
    if np.abs(o - e).max() > 0:
        fails.append("origin is not the eye")
    if abs(np.linalg.norm(d) - 1) > tol:
        fails.append("direction is not unit length")
    if _angle(d, f) > 1e-9:
        fails.append("centre ray does not point at the target")
    # middle of the top edge: vfov/2 above the axis, in the plane of the view axis and up
    _, d = ray(cx, 0, cu, 0.0)
    if abs(_angle(d, f) - half_v) > 1e-9:
        fails.append("top-edge angle is not vfov/2")
    if not np.dot(d, u) > 0:
        fails.append("row 0 is not at the top")
    if abs(np.dot(d, r)) > 1e-9:
        fails.append("top-edge ray leaves the vertical plane")
    # middle of the left edge: the horizontal half-angle, to the left
    _, d = ray(0, cy, 0.0, cv)
    if abs(_angle(d, f) - half_h) > 1e-9:
        fails.append("left-edge angle is not atan(tan(vfov/2) W/H)")
    if not np.dot(d, r) < 0:
        fails.append("column 0 is not on the left")
    # square pixels on the image plane at unit distance along the axis; rows down, columns right
    xs, ys = np.meshgrid(np.arange(W), np.arange(H))
    px = (ys * W + xs).reshape(-1)
    _, d = oracle.camera_rays(cam, px, 0.5, 0.5)
    p = d / (d @ f)[:, None]
    P = np.stack([p @ r, p @ u], axis=-1).reshape(H, W, 2)
    pitch = 2 * math.tan(half_v) / H
    if W > 1 and not np.allclose(P[:, 1:, 0] - P[:, :-1, 0], pitch, rtol=1e-9, atol=0):
        fails.append("horizontal pixel pitch is not 2 tan(vfov/2)/H (columns left to right)")
    if H > 1 and not np.allclose(P[:-1, :, 1] - P[1:, :, 1], pitch, rtol=1e-9, atol=0):
        fails.append("vertical pixel pitch is not 2 tan(vfov/2)/H (rows top to bottom)")
    if not np.allclose(P[:, :, 0], P[:1, :, 0], rtol=0, atol=1e-12):
        fails.append("columns are not vertical")
    if not np.allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=tol):
        fails.append("directions are not unit length")
    # sub-pixel offsets move across the pixel: (u0, u1) = (1, 1) of pixel (x, y) is (0, 0) of (x+1, y+1)
    _, d0 = ray(1, 1, 0.0, 0.0)
    _, d1 = ray(0, 0, 1.0, 1.0)
    if _angle(d0, d1) > 1e-12:
        fails.append("sub-pixel offset does not span the pixel")
    return fails


@pytest.mark.parametrize("k", range(len(CAMERAS)))
def test_camera_is_the_pinhole(oracle_lib, k):
    assert camera_failures(oracle_lib, CAMERAS[k]) == []


# ------------------------------------------------------------------ light pick
def _light_scene(kind):
    if kind == "fan":
        return scenes.rect_over_plane(half_w=0.9, half_h=0.6, height=1.0, fan=(0.8, 0.7))
    sc = scenes.random_soup(n_tris=300, seed=4, size=0.4, n_mats=5)
    sc["mat_emission"] = np.array([0.0, 2.0, 0.0, 7.0, 0.0], np.float32)
    return sc


def _areas(sc):
    V = np.asarray(sc["verts"], np.float32).astype(np.float64)
    T = np.asarray(sc["tris"], np.int64)
    a = V[T[:, 1]] - V[T[:, 0]]
    b = V[T[:, 2]] - V[T[:, 0]]
    return 0.5 * np.linalg.norm(np.cross(a, b), axis=1)


def light_pick_failures(oracle, sc, n=1_000_000, seed=3):
    fails = []
    osc = oracle.Scene.from_dict(sc)
    emissive = np.asarray(sc["mat_emission"])[np.asarray(sc["tri_mat"], np.int64)] > 0
    lights = np.flatnonzero(emissive)
    if not np.array_equal(osc.light_tris, lights):
        fails.append("light list is not the emissive triangles in ascending id")
        return fails
    area = _areas(sc)[lights]
    if abs(osc.light_area - area.sum()) > 1e-12 * area.sum():
        fails.append("total light area")
    # uniforms exactly as the renderer draws them: 24-bit fractions
    u = np.random.default_rng(seed).integers(0, 1 << 24, size=n) / float(1 << 24)
    j = osc.pick_light(u)
    if j.min() < 0 or j.max() >= len(lights):
        fails.append("light index out of range")
        return fails
    obs = np.bincount(j, minlength=len(lights)).astype(np.float64)
    exp = n * area / area.sum()
    stat = float(((obs - exp) ** 2 / exp).sum())
    from scipy.stats import chi2
    if chi2.sf(stat, len(lights) - 1) < 1e-6:
        fails.append(f"pick counts are not area-proportional (chi2 {stat:.1f}, {len(lights) - 1} dof)")
    # the inverse cdf is monotone in u (the boundaries are the inclusive prefix sums)
    order = np.argsort(u, kind="stable")
    if np.any(np.diff(j[order]) < 0):
        fails.append("pick is not monotone in u")
    return fails


@pytest.mark.parametrize("kind", ["fan", "soup"])
def test_light_pick_is_area_proportional(oracle_lib, kind):
    pytest.importorskip("scipy")
    sc = _light_scene(kind)
    areas = _areas(sc)[np.asarray(sc["mat_emission"])[np.asarray(sc["tri_mat"], np.int64)] > 0]
    assert areas.max() > 4 * areas.min()        # the pin needs lights of very unequal area
    assert light_pick_failures(oracle_lib, sc) == []


def _rows(name):
    return [[float(x) for x in ln.split()] for ln in open(os.path.join(GOLD, name))
            if ln.strip() and not ln.startswith("#")]


def _corner_ff(X, Y):
    ax, ay = abs(X), abs(Y)
    sx, sy = np.sqrt(1 + ax * ax), np.sqrt(1 + ay * ay)
    return (ax / sx * np.arctan(ay / sx) + ay / sy * np.arctan(ax / sy)) / (2 * np.pi)


def _point_ff(px, pz, hw, hh, c):
    return sum(_corner_ff(wx / c, wz / c) for wx in (hw - px, hw + px) for wz in (hh - pz, hh + pz))


def fan_form_factor_failures(oracle, row, n=200_000):
    """Irradiance of a Lambert point under a parallel rectangle light cut into unequal triangles."""
    px, pz, hw, hh, c = row
    rho, Le = 0.7, 5.0
    sc = oracle.Scene.from_dict(scenes.rect_over_plane(albedo=rho, emission=Le, half_w=hw, half_h=hh, height=c,
                                                       fan=(0.8, 0.7)))
    o = np.tile([px, 0.5 * c, pz], (n, 1))
    d = np.tile([0.0, -1.0, 0.0], (n, 1))
    L, _ = sc.trace_rays(o, d, np.arange(n), max_depth=2)
    expect = rho * Le * _point_ff(px, pz, hw, hh, c)
    m, se = L[:, 0].mean(), L[:, 0].std() / np.sqrt(n)
    if not abs(m - expect) < 4 * se + 1e-4 * expect:
        return [f"fan light irradiance {m:.6g} +- {se:.2g}, closed form {expect:.6g}"]
    return []


@pytest.mark.parametrize("row", _rows("form_factor_parallel_rect.txt"))
def test_fan_light_form_factor(oracle_lib, row):
    assert fan_form_factor_failures(oracle_lib, row) == []


# ------------------------------------------------------------------ planted mistakes
PLANTED_CAMERA = {
    "rows flipped": [("(1.0 - 2.0 * sy) * c->th", "(2.0 * sy - 1.0) * c->th")],
    "half the field of view": [("c.th = tan((double)vfov_deg * OR_PI / 360.0);",
                                "c.th = tan((double)vfov_deg * OR_PI / 720.0);")],
    "mirrored right axis": [("c.u = nrm(cross(mk(up[0], up[1], up[2]), c.w));",
                             "c.u = nrm(cross(c.w, mk(up[0], up[1], up[2])));")],
    "aspect on the vertical": [("c.tw = c.th * (double)W / (double)H;",
                                "c.tw = c.th; c.th = c.th * (double)H / (double)W;")],
}

PLANTED_LIGHT = {
    "count-uniform pick": [("static int64_t pick_light(const or_scene* s, double u) {",
                            "static int64_t pick_light(const or_scene* s, double u) {\n"
                            "    if (s->n_lights > 0) return (int64_t)(u * (double)s->n_lights);")],
    "pick one index low": [("        else lo = mid + 1;\n    }\n    return lo;",
                            "        else lo = mid + 1;\n    }\n    return lo > 0 ? lo - 1 : 0;")],
}


@pytest.fixture(scope="module")
def variants(oracle_lib, tmp_path_factory):
    out = tmp_path_factory.mktemp("oracle_variants")
    libs = {}
    for i, (name, rep) in enumerate(list(PLANTED_CAMERA.items()) + list(PLANTED_LIGHT.items())):
        libs[name] = oracle_lib.build_variant(rep, str(out), f"liboracle_v{i}.so")
    return libs


@pytest.mark.parametrize("name", list(PLANTED_CAMERA))
def test_planted_camera_mistake_fails_the_pin(oracle_lib, variants, name):
    with oracle_lib.use_library(variants[name]):
        caught = [camera_failures(oracle_lib, cam) for cam in CAMERAS]
    assert all(caught), (name, caught)


@pytest.mark.parametrize("name", list(PLANTED_LIGHT))
def test_planted_light_pick_mistake_fails_the_pins(oracle_lib, variants, name):
    pytest.importorskip("scipy")
    rows = _rows("form_factor_parallel_rect.txt")
    with oracle_lib.use_library(variants[name]):
        pick = [light_pick_failures(oracle_lib, _light_scene(k)) for k in ("fan", "soup")]
        ff = [fan_form_factor_failures(oracle_lib, r) for r in rows]
    # the counting pin catches it on both scenes, and the estimator pin on some geometry
    assert all(pick), (name, pick)
    assert any(ff), (name, ff)
