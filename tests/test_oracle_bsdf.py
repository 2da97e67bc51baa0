"""Oracle pins: BSDF identities.

Each check is something the mathematics fixes independently of how the oracle wrote it:
Lambert value a/pi and cosine-distributed samples; GGX normalisation of D, G1 limits,
reciprocity, and the visible-normal sampler's distribution (the mean sample weight equals the
directional albedo computed by quadrature of f cos over the hemisphere, for several test
functions); Fresnel limits (normal incidence ((n-1)/(n+1))^2, grazing -> 1, total internal
reflection past the critical angle, and the reciprocity F(i, n1->n2) = F(t, n2->n1)); Snell's
law and unit length of sampled directions; Schlick endpoints.
"""
import numpy as np
import pytest

N = np.array([0.0, 0.0, 1.0])


def _dir(theta, phi=0.3):
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


def test_lambert_value(oracle_lib):
    a = np.array([0.2, 0.5, 0.9])
    f = oracle_lib.bsdf_eval(0, a, 0.5, N, _dir(0.3), _dir(1.1, 2.0))
    assert np.allclose(f, a / np.pi, rtol=0, atol=1e-15)
    assert np.all(oracle_lib.bsdf_eval(0, a, 0.5, N, _dir(0.3), -_dir(1.1)) == 0)


def test_lambert_samples_cosine_distributed(oracle_lib):
    rng = np.random.default_rng(0)
    cos2 = []
    for _ in range(20000):
        ok, wi, w, code = oracle_lib.bsdf_sample(0, [0.3, 0.4, 0.5], 0.5, 1.5, N, N, _dir(0.4), 0.0,
                                                 rng.uniform(), rng.uniform())
        assert ok and code == 0 and np.allclose(w, [0.3, 0.4, 0.5])
        assert abs(np.linalg.norm(wi) - 1) < 1e-12
        cos2.append(wi[2] ** 2)
    hist = np.histogram(cos2, bins=20, range=(0, 1))[0]   # cos^2 ~ U(0,1) for p = cos/pi
    exp = len(cos2) / 20
    assert ((hist - exp) ** 2 / exp).sum() < 50


@pytest.mark.parametrize("r", [0.05, 0.2, 0.6, 1.0])
def test_ggx_D_normalised(oracle_lib, r):
    # integral of D(h) cos(theta_h) d(omega_h) over the hemisphere = 1.  With mu = cos^2 the
    # measure cos d(omega) = pi d(mu); a geometric grid in s = 1 - mu resolves sharp lobes.
    s = np.concatenate([[0.0], np.geomspace(1e-13, 1.0, 60001)])
    D = np.array([oracle_lib.ggx_D(r, np.sqrt(1.0 - x)) for x in s])
    val = np.trapezoid(D * np.pi, s)
    assert abs(val - 1.0) < 1e-4


def test_ggx_G1_limits(oracle_lib):
    assert abs(oracle_lib.ggx_G1(0.5, 1.0) - 1.0) < 1e-15
    g = [oracle_lib.ggx_G1(0.5, c) for c in np.linspace(0.05, 1.0, 20)]
    assert np.all(np.diff(g) > 0) and max(g) <= 1.0


def test_ggx_reciprocity(oracle_lib):
    rng = np.random.default_rng(1)
    for _ in range(200):
        wo = _dir(rng.uniform(0, 1.5), rng.uniform(0, 6.28))
        wi = _dir(rng.uniform(0, 1.5), rng.uniform(0, 6.28))
        a = rng.uniform(0.1, 1, 3)
        r = rng.uniform(0.05, 1)
        f1 = oracle_lib.bsdf_eval(1, a, r, N, wo, wi)
        f2 = oracle_lib.bsdf_eval(1, a, r, N, wi, wo)
        assert np.allclose(f1, f2, rtol=1e-12, atol=0)


def _hemi_quadrature(oracle_lib, a, r, wo, g, n_th=300, n_ph=300):
    # integral of g(wi) f(wo, wi) cos(theta_i) d(omega_i) by midpoint rule in (mu = cos^2, phi)
    mu = (np.arange(n_th) + 0.5) / n_th
    ph = (np.arange(n_ph) + 0.5) / n_ph * 2 * np.pi
    acc = np.zeros(3)
    for m in mu:
        c = np.sqrt(m)
        s = np.sqrt(1 - m)
        for p in ph:
            wi = np.array([s * np.cos(p), s * np.sin(p), c])
            acc += g(wi) * oracle_lib.bsdf_eval(1, a, r, N, wo, wi)
    # d(omega) cos = sin cos dtheta dphi = 0.5 d(mu) dphi
    return acc * 0.5 * (1.0 / n_th) * (2 * np.pi / n_ph)


@pytest.mark.parametrize("r,theta_o", [(0.6, 0.5), (0.35, 1.2)])
def test_ggx_vndf_sampler_matches_quadrature(oracle_lib, r, theta_o):
    a = np.array([0.9, 0.6, 0.3])
    wo = _dir(theta_o, 0.7)
    n = 128
    tests = {"albedo": lambda w: 1.0, "x": lambda w: w[0], "z2": lambda w: w[2] ** 2}
    est = {k: np.zeros(3) for k in tests}
    for i in range(n):
        for j in range(n):
            ok, wi, w, code = oracle_lib.bsdf_sample(1, a, r, 1.5, N, N, wo, 0.0, (i + 0.5) / n, (j + 0.5) / n)
            if not ok:
                assert code == 2
                continue
            assert abs(np.linalg.norm(wi) - 1) < 1e-12
            for k, g in tests.items():
                est[k] += g(wi) * w
    for k, g in tests.items():
        ref = _hemi_quadrature(oracle_lib, a, r, wo, g, 160, 160)
        assert np.allclose(est[k] / n ** 2, ref, rtol=2e-2, atol=2e-3), (k, est[k] / n ** 2, ref)


def test_ggx_energy_bounded(oracle_lib):
    for r in (0.05, 0.3, 0.8):
        for th in (0.1, 0.8, 1.4):
            ref = _hemi_quadrature(oracle_lib, np.ones(3), r, _dir(th), lambda w: 1.0, 120, 120)
            assert np.all(ref <= 1.0 + 1e-2)


def test_fresnel_limits_and_reciprocity(oracle_lib):
    assert abs(oracle_lib.fresnel_dielectric(1.0, 1.0, 1.5) - 0.04) < 1e-15
    assert abs(oracle_lib.fresnel_dielectric(1.0, 1.5, 1.0) - 0.04) < 1e-15
    assert oracle_lib.fresnel_dielectric(1e-9, 1.0, 1.5) > 0.9999
    crit = np.sqrt(1 - (1 / 1.5) ** 2)            # cos of the critical angle inside glass
    assert oracle_lib.fresnel_dielectric(crit * 0.999, 1.5, 1.0) == 1.0
    assert oracle_lib.fresnel_dielectric(crit * 1.001, 1.5, 1.0) < 1.0
    for ci in np.linspace(0.05, 1.0, 20):
        st = np.sqrt(1 - ci * ci) / 1.5
        ct = np.sqrt(1 - st * st)
        assert abs(oracle_lib.fresnel_dielectric(ci, 1.0, 1.5) - oracle_lib.fresnel_dielectric(ct, 1.5, 1.0)) < 1e-12


def test_dielectric_sampling_snell_and_weights(oracle_lib):
    ng = N
    for th in np.linspace(0.05, 1.5, 15):
        wo = _dir(th, 0.4)
        F = oracle_lib.fresnel_dielectric(np.cos(th), 1.0, 1.5)
        ok, wr, w, code = oracle_lib.bsdf_sample(2, [1, 1, 1], 0.5, 1.5, N, ng, wo, F * 0.5, 0.3, 0.3)
        assert ok and code == 3 and np.allclose(w, 1)
        assert np.allclose(wr, [-wo[0], -wo[1], wo[2]], atol=1e-14)       # mirror
        ok, wt, w, code = oracle_lib.bsdf_sample(2, [1, 1, 1], 0.5, 1.5, N, ng, wo, F + (1 - F) * 0.5, 0.3, 0.3)
        assert ok and code == 4
        assert abs(np.linalg.norm(wt) - 1) < 1e-12 and wt[2] < 0
        sin_i = np.sin(th)
        sin_t = np.hypot(wt[0], wt[1])
        assert abs(sin_i - 1.5 * sin_t) < 1e-12                               # Snell
        assert np.allclose(w, (1 / 1.5) ** 2)                                  # radiance scale
    # from inside: total internal reflection past the critical angle
    wo = _dir(1.2, 0.0) * np.array([1, 1, -1])     # wo below the winding normal -> inside
    ok, wi, w, code = oracle_lib.bsdf_sample(2, [1, 1, 1], 0.5, 1.5, -N, ng, wo, 0.999999, 0.3, 0.3)
    assert ok and code == 5 and np.allclose(w, 1)


def test_schlick_endpoints(oracle_lib):
    a = np.array([0.3, 0.6, 0.9])
    wo = _dir(0.0)
    f = oracle_lib.bsdf_eval(1, a, 0.5, N, wo, wo)   # h = n, cos = 1 -> F = F0
    D = oracle_lib.ggx_D(0.5, 1.0)
    # G2 = 1 at normal incidence for both directions, so f = F0 D / 4 exactly
    assert np.allclose(f, a * D / 4.0, rtol=1e-14)
    # grazing half-vector: Schlick -> 1 regardless of F0
    wo = _dir(1.5707, 0.0)
    wi = _dir(1.5707, np.pi)
    f2 = oracle_lib.bsdf_eval(1, a, 0.5, N, wo, wi)   # h ~ n, cos(wi, h) ~ 0 -> F ~ 1
    assert np.allclose(f2 / f2.max(), 1.0, atol=1e-3)


def test_onb_orthonormal_and_continuous_on_axis_planes(oracle_lib):
    rng = np.random.default_rng(4)
    ns = rng.normal(size=(500, 3))
    ns = np.concatenate([ns, np.eye(3), -np.eye(3), [[0.6, 0.8, 0.0], [0.0, -0.6, 0.8]]])
    for n in ns:
        n = n / np.linalg.norm(n)
        t, b = oracle_lib.onb(n)
        M = np.stack([t, b, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(t, b), n, atol=1e-12)          # right-handed
    # the basis does not jump for normals on the coordinate planes (floors, walls): a tilt of
    # 1e-9 across z = 0, y = 0 or x = 0 moves it by about the tilt
    for n in (np.array([0.0, 1.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.6, 0.0, 0.8])):
        for axis in range(3):
            e = np.zeros(3)
            e[axis] = 1e-9
            t1, b1 = oracle_lib.onb((n + e) / np.linalg.norm(n + e))
            t2, b2 = oracle_lib.onb((n - e) / np.linalg.norm(n - e))
            assert np.abs(t1 - t2).max() < 1e-7 and np.abs(b1 - b2).max() < 1e-7
