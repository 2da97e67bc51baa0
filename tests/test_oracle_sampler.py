"""Pins of the oracle's pixel samplers (ray generation, Sec. 2.3): the Halton (2,3) sequence with a
per-pixel Cranley-Patterson rotation, in 24-bit fixed point.

The radical inverses are pinned to the published first terms of the van der Corput sequences in
bases 2 and 3 and to their stratification property (the first b^k terms are exactly the fractions
j / b^k, one per interval [j / b^k, (j + 1) / b^k)); the rotation must keep that stratification (a shift modulo
1 moves every point by the same amount), differ between pixels and leave the PCG sampler's jitter
untouched.  The estimator with the Halton jitter must agree with the PCG jitter's image within
Monte Carlo error.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_27323_gb300 import scenes

# van der Corput sequences (the first Halton coordinates): phi_2(1..8) and phi_3(1..9)
VDC2 = [Fraction(1, 2), Fraction(1, 4), Fraction(3, 4), Fraction(1, 8), Fraction(5, 8), Fraction(3, 8),
        Fraction(7, 8), Fraction(1, 16)]
VDC3 = [Fraction(1, 3), Fraction(2, 3), Fraction(1, 9), Fraction(4, 9), Fraction(7, 9), Fraction(2, 9),
        Fraction(5, 9), Fraction(8, 9), Fraction(1, 27)]


def _fix24(x: Fraction) -> int:
    return (x.numerator << 24) // x.denominator


def test_radical_inverse_first_terms():
    assert oracle.radical_inverse24(2, 0) == 0 and oracle.radical_inverse24(3, 0) == 0
    for s, v in enumerate(VDC2, start=1):
        assert oracle.radical_inverse24(2, s) == _fix24(v), s
    for s, v in enumerate(VDC3, start=1):
        assert oracle.radical_inverse24(3, s) == _fix24(v), s


@pytest.mark.parametrize("base,k", [(2, 10), (2, 16), (3, 6), (3, 9)])
def test_radical_inverse_stratifies(base, k):
    # the first b^k terms are exactly the fractions j / b^k (each stratum holds one, on its left edge)
    n = base ** k
    v = np.array([oracle.radical_inverse24(base, s) for s in range(n)], np.int64)
    assert np.array_equal(np.sort(v), (np.arange(n, dtype=np.int64) << 24) // n)


def test_radical_inverse_large_indices():
    # digit reversal of large indices: 2^31 -> 1/2^32 (below the 24-bit resolution), 2^32 - 1 -> 1 - 2^-32
    assert oracle.radical_inverse24(2, 1 << 31) == 0
    assert oracle.radical_inverse24(2, (1 << 32) - 1) == (1 << 24) - 1
    assert oracle.radical_inverse24(2, 3 << 30) == 0
    assert oracle.radical_inverse24(2, 1 << 8) == 1 << 15
    # 3^20 has the single digit 1 at position 20: phi = 3^-21 -> floor(2^24 / 3^21) = 0; 2 * 3^19 -> 2 / 3^20
    assert oracle.radical_inverse24(3, 3 ** 20) == 0
    assert oracle.radical_inverse24(3, 2 * 3 ** 10) == _fix24(Fraction(2, 3 ** 11))


def test_rotation_keeps_stratification_and_differs_per_pixel():
    n = 256
    pix = np.array([0, 1, 5, 77, 12345], np.uint32)
    rots = []
    for p in pix:
        j = oracle.pixel_jitter("halton", 42, np.full(n, p, np.uint32), np.arange(n, dtype=np.uint32))
        x = np.round(j[:, 0] * (1 << 24)).astype(np.int64)
        # a cyclic shift of {m * 2^16}: sorted gaps all 2^16 (including the wrap-around)
        xs = np.sort(x)
        gaps = np.diff(np.concatenate([xs, [xs[0] + (1 << 24)]]))
        assert np.all(gaps == (1 << 16)), p
        # base-3 coordinate of the first 243 samples: one point per stratum of width 1/243 after the shift
        y = np.round(j[:243, 1] * (1 << 24)).astype(np.int64)
        shift = (y[0] - oracle.radical_inverse24(3, 0)) % (1 << 24)
        unshifted = (y - shift) % (1 << 24)
        assert np.array_equal(np.sort(unshifted), (np.arange(243, dtype=np.int64) << 24) // 243)
        rots.append(shift)
    assert len(set(rots)) == len(rots)
    assert np.all((j >= 0) & (j < 1))


def test_pcg_jitter_is_the_path_uniforms():
    rng = np.random.default_rng(1)
    px = rng.integers(0, 1 << 20, 1000).astype(np.uint32)
    sm = rng.integers(0, 1 << 10, 1000).astype(np.uint32)
    j = oracle.pixel_jitter("pcg", 9, px, sm)
    assert np.array_equal(j[:, 0], oracle.u01(9, px, sm, np.zeros(1000, np.uint32), np.zeros(1000, np.uint32)))
    assert np.array_equal(j[:, 1], oracle.u01(9, px, sm, np.zeros(1000, np.uint32), np.ones(1000, np.uint32)))


def test_halton_image_matches_pcg_image_within_mc_error():
    """The pixel estimates of the two samplers differ by Monte Carlo noise only: measured against
    the PCG paths' per-pixel standard errors, the Halton image is no farther from a PCG image than
    a second PCG image (another seed) is; the radiance is heavy-tailed (rare light hits), so the
    comparison is relative rather than to a unit normal."""
    sc = scenes.box_scene(seed=0, width=12, height=10)
    o = oracle.Scene.from_dict(sc)
    cam = sc["camera"]
    spp, n_pix = 256, 12 * 10
    img_h, _ = o.render_pixels(cam, spp, 4, 3, sampler="halton")
    L = o.render_paths(cam, spp, 4, 5, np.arange(n_pix * spp))["L"].reshape(n_pix, spp, 3)
    L2 = o.render_paths(cam, spp, 4, 9, np.arange(n_pix * spp))["L"].reshape(n_pix, spp, 3)
    img_p, img_p2 = L.mean(1), L2.mean(1)
    se = np.sqrt((L.var(1, ddof=1) + L2.var(1, ddof=1)) / spp)
    z_h = (img_h - img_p) / (se + 1e-9)
    z_p = (img_p2 - img_p) / (se + 1e-9)
    assert np.sqrt(np.mean(z_h ** 2)) < 1.25 * np.sqrt(np.mean(z_p ** 2))
    assert np.median(np.abs(z_h)) < 1.0             # 0.67 for normal noise
    # no bias in the image mean: within 4 standard errors of the mean of 2 x 120 x 3 estimates
    assert abs(img_h.mean() - img_p.mean()) < 4 * np.sqrt(np.sum(se ** 2)) / se.size
