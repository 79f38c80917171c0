"""Pins for the oracle's delta-tracking transport (Sec. 5.1's scattering trace).

  * zero density: every path escapes;
  * delta tracking is unbiased: with a homogeneous sigma the chance of
    leaving without a real collision is exp(-sigma L) whatever the majorant
    (null collisions must not change it);
  * the first real collision absorbs with probability 0.2 (albedo 0.8);
  * Henyey-Greenstein sampling has mean cosine g = 0.3 and unit directions;
  * the noise generator vanishes on its lattice and the volume recipe has
    the stated mean optical depth.
"""
import math

import numpy as np
from scipy import stats

import oracle
from paper_2605_30294_gb300 import inputs


def _cam_axis(n, w=1, h=1):
    # a narrow camera on the -z side looking along +z through the centre
    c = n / 2.0
    return inputs.camera((c, c, -10.0 * n), (c, c, c), (0.0, 1.0, 0.0), 0.01, w, h)


def test_zero_density_escapes():
    n = 16
    vol = np.zeros((n, n, n), np.float32)
    cam = inputs.c0_camera(n, 8, 8)
    img, _ = oracle.c4_render_crop(vol, 0.5, cam, 8, 0, 0, 0, 8, 8, 4)
    assert np.all(img == 1.0)


def _first_collision_stats(n, sigma, sigma_max, paths=20000):
    vol = np.full((n, n, n), sigma, np.float32)
    cam = _cam_axis(n)
    escaped_clean = absorbed_first = collided = 0
    for s in range(paths):
        score, ev, b = oracle.c4_path(vol, sigma_max, cam, 1, 0, 0, 0, s)
        if b == 0 and score == 1:
            escaped_clean += 1
        else:
            collided += 1
            if b == 0 and score == 0:
                absorbed_first += 1
    return escaped_clean / paths, absorbed_first / max(collided, 1), collided


def test_delta_tracking_is_unbiased_beer_lambert():
    n, sigma = 16, 0.05
    p_escape = math.exp(-sigma * n)  # the axis ray crosses n cells
    for smax in (sigma, 4 * sigma):
        frac, _, _ = _first_collision_stats(n, sigma, smax)
        assert abs(frac - p_escape) < 5 * math.sqrt(p_escape * (1 - p_escape) / 20000)


def test_albedo():
    n, sigma = 16, 0.2
    _, absorbed, collided = _first_collision_stats(n, sigma, 2 * sigma)
    assert abs(absorbed - 0.2) < 5 * math.sqrt(0.16 / collided)


def test_henyey_greenstein_mean_cosine():
    rng = np.random.default_rng(3)
    d = np.array([0.3, -0.5, 0.81], np.float32)
    d /= np.linalg.norm(d)
    cs = []
    for xi, xp in rng.random((20000, 2)):
        o = oracle.c4_hg_sample(d, xi, xp)
        assert abs(np.linalg.norm(o) - 1.0) < 1e-5
        cs.append(float(np.dot(o, d)))
    cs = np.array(cs)
    assert abs(cs.mean() - 0.3) < 5 * cs.std() / math.sqrt(len(cs))
    # the HG density of cos theta: (1 - g^2) / (2 (1 + g^2 - 2 g mu)^{3/2})
    g = 0.3
    cdf = lambda mu: (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    assert stats.kstest(cs, cdf).pvalue > 1e-4


def test_noise_vanishes_on_lattice_and_volume_recipe():
    for p in ((0.25, 0.5, 0.75), (0.0, 0.0, 0.0), (1.0, 0.25, 0.5)):
        assert abs(inputs.noise_at(p, octaves=1, base=4.0)) < 1e-12
    assert abs(inputs.noise_at((0.13, 0.41, 0.77), octaves=1, base=4.0)) > 1e-6
    vol, smax = inputs.c4_volume(64)
    assert abs(vol.astype(np.float64).mean() - 8.0 / 64) < 1e-5
    assert smax == vol.max() and vol.min() >= 0.0
    assert 0.2 < (vol > 0).mean() < 0.8


def test_views_recipe():
    views = inputs.c4_views(1024)
    assert [(w, h) for _, w, h, _ in views] == [(2048, 2048), (1024, 768), (512, 512), (3840, 2160)]
    assert sum(w * h for _, w, h, _ in views) == 13537280
    assert [b for _, _, _, b in views] == [0, 2048 * 2048, 2048 * 2048 + 1024 * 768, 2048 * 2048 + 1024 * 768 + 512 * 512]
