"""Pins for the oracle's absorption marching (trace step of Sec. 5.1).

What fixes it independently of the oracle's own code:
  * sigma(p): scipy's linear ``map_coordinates`` with nearest-edge clamping
    on coordinates p - 0.5 (voxel centres) is the same interpolant;
  * a field linear in one axis is reproduced exactly by trilinear
    interpolation, and the fixed-step midpoint sum of a linear function equals
    its integral: tau has a closed form;
  * a constant field gives T = exp(-sigma * 0.5 * n_samples);
  * straight rays cross a convex brick grid monotonically, so the hop
    sequence visits each brick once and moves by at most one brick per axis.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_2605_30294_gb300 import inputs


def _sigma_scipy(vol, pts):
    # vol[z, y, x]; map_coordinates wants (z, y, x) coordinates
    c = np.stack([pts[:, 2] - 0.5, pts[:, 1] - 0.5, pts[:, 0] - 0.5]).astype(np.float64)
    return ndimage.map_coordinates(vol.astype(np.float64), c, order=1, mode="nearest")


@pytest.mark.parametrize("n", [4, 8, 64])
def test_sigma_matches_library_trilinear(n):
    rng = np.random.default_rng(n)
    vol = rng.random((n, n, n), dtype=np.float32) * 0.1
    # interior, edge and outside-the-grid points (clamp to edge)
    pts = rng.uniform(-0.7, n + 0.7, size=(400, 3)).astype(np.float32)
    pts[:5] = [[0, 0, 0], [n, n, n], [0.5, 0.5, 0.5], [n - 0.5, 1.5, 2.25], [n / 2, n / 2, n / 2]]
    got = np.array([oracle.c0_sigma(vol, p) for p in pts])
    want = _sigma_scipy(vol, pts)
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-8)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sigma_reproduces_linear_field(axis):
    n = 16
    c = np.arange(n, dtype=np.float64) + 0.5
    shape = [1, 1, 1]
    shape[2 - axis] = n
    vol = np.broadcast_to((0.01 * c + 0.02).reshape(shape), (n, n, n)).astype(np.float32)
    rng = np.random.default_rng(axis)
    pts = rng.uniform(0.5, n - 0.5, size=(200, 3)).astype(np.float32)
    got = np.array([oracle.c0_sigma(vol, p) for p in pts])
    want = 0.01 * pts[:, axis].astype(np.float64) + 0.02
    np.testing.assert_allclose(got, want, rtol=1e-5)


def _cam_skew(n, w, h):
    # far eye, narrow field, rays slanted in x (dx/dz ~ 0.3): every ray enters z = 0 and
    # leaves z = n while x stays inside [0.5, n - 0.5], where the linear field is unclamped
    c = n / 2.0
    eye = (c - 10.0 * n * 0.3, c, c - 10.0 * n)
    return inputs.camera(eye, (c, c, c), (0.0, 1.0, 0.0), 2.0, w, h)


def test_tau_linear_field_closed_form():
    n, w, h = 32, 8, 8
    cam = _cam_skew(n, w, h)
    cx = np.arange(n, dtype=np.float64) + 0.5
    a, b = 0.003, 0.01
    vol = np.broadcast_to((a * cx + b)[None, None, :], (n, n, n)).astype(np.float32)
    res = oracle.c0_render(vol, cam, w, h)
    for y in range(h):
        for x in range(w):
            hit, d, t0, t1 = oracle.c0_primary(cam, n, x, y)
            assert hit and 0.25 < d[0] / d[2] < 0.35
            pix = y * w + x
            m = int(res["nsamp"][pix])
            assert m > 0
            # midpoint rule over [t0, t0 + 0.5 m] is exact for a linear integrand
            ta, tb = float(t0), float(t0) + 0.5 * m
            ox, dx = float(cam[0]), float(d[0])
            integral = a * (ox * (tb - ta) + dx * (tb * tb - ta * ta) / 2.0) + b * (tb - ta)
            assert abs(res["tau"][pix] - integral) <= 2e-5 * integral
            assert abs(res["T"][pix] - math.exp(-integral)) <= 2e-5


def test_sample_count_and_constant_field():
    n, w, h = 8, 16, 16
    cam = inputs.c0_camera(n, w, h)
    sig = np.float32(0.07)
    vol = np.full((n, n, n), sig, np.float32)
    res = oracle.c0_render(vol, cam, w, h)
    for y in range(h):
        for x in range(w):
            hit, d, t0, t1 = oracle.c0_primary(cam, n, x, y)
            # brute-force sample count: k with t0 + (k + 0.5) * 0.5 < t1, in float32
            k = 0
            if hit:
                while np.float32(t0) + (np.float32(k) + np.float32(0.5)) * np.float32(0.5) < np.float32(t1):
                    k += 1
            pix = y * w + x
            assert res["nsamp"][pix] == k
            # trilinear weights of a constant field sum to 1 up to rounding
            assert abs(float(res["tau"][pix]) - 0.5 * float(sig) * k) <= 1e-6 * max(1, k)
            assert abs(res["T"][pix] - math.exp(-0.5 * float(sig) * k)) < 1e-5 * max(1, k)
            if not hit:
                assert res["T"][pix] == 1.0


def test_primary_ray_geometry():
    n, w, h = 64, 128, 128
    cam = inputs.c0_camera(n, w, h)
    # the two centre pixels straddle the optical axis symmetrically
    _, d1, _, _ = oracle.c0_primary(cam, n, 63, 63)
    _, d2, _, _ = oracle.c0_primary(cam, n, 64, 64)
    assert abs(d1[0] + d2[0]) < 1e-6 and abs(d1[1] + d2[1]) < 1e-6 and d1[2] > 0.999
    # the top-left pixel is 20 deg (minus half a pixel) off axis, vertically
    _, d, _, _ = oracle.c0_primary(cam, n, 0, 0)
    assert d[1] > 0 and d[0] < 0
    ang_y = math.atan2(d[1], d[2])
    assert abs(ang_y - math.atan(math.tan(math.radians(20)) * 127 / 128)) < 1e-5
    # a ray that enters through z = 0 at the centre starts at t0 = 64
    hit, d, t0, t1 = oracle.c0_primary(cam, n, 64, 64)
    assert hit and abs(t0 * d[2] - 64.0) < 1e-3
    # ... and leaves through z = 64 at t1 = 128 / dz
    assert abs(t1 * d[2] - 128.0) < 1e-3
    # a ray that misses the box has no sample
    far = inputs.camera((32.0, 32.0, -64.0), (32.0, 300.0, 32.0), (0.0, 0.0, 1.0), 5.0, 4, 4)
    assert not oracle.c0_primary(far, n, 1, 1)[0]


@pytest.mark.parametrize("brick", [16, 32, 64])
def test_hop_sequence_is_monotone_brick_walk(brick):
    n, w, h = 64, 32, 32
    cam = inputs.c0_camera(n, w, h)
    vol = inputs.c0_volume(n)
    res = oracle.c0_render(vol, cam, w, h, brick=brick, max_hops=16)
    nb = n // brick
    for pix in range(w * h):
        cnt = int(res["hop_count"][pix])
        seq = res["hops"][pix, :cnt]
        assert cnt <= 3 * (nb - 1) + 1
        assert len(set(seq.tolist())) == cnt
        co = np.stack([seq % nb, (seq // nb) % nb, seq // (nb * nb)], 1)
        if cnt > 1:
            step = np.diff(co, axis=0)
            assert np.all(np.abs(step) <= 1)
            for ax in range(3):
                s = step[:, ax]
                assert np.all(s >= 0) or np.all(s <= 0)
        assert (cnt == 0) == (res["nsamp"][pix] == 0)


def test_render_independent_of_brick_size():
    # the oracle's T does not depend on the owner bookkeeping
    n, w, h = 64, 32, 32
    cam = inputs.c0_camera(n, w, h)
    vol = inputs.c0_volume(n)
    a = oracle.c0_render(vol, cam, w, h, brick=64)
    b = oracle.c0_render(vol, cam, w, h, brick=16)
    np.testing.assert_array_equal(a["T"], b["T"])


def test_blob_volume_recipe():
    n = 64
    vol = inputs.c0_volume(n)
    assert vol.shape == (n, n, n) and vol.dtype == np.float32
    cen, s = inputs.c0_blobs(n)
    assert np.all((s >= 4) & (s <= 10))
    assert np.all(cen >= s[:, None]) and np.all(cen <= n - s[:, None])
    # at a voxel centre the value is the blob sum, float64 -> float32
    z, y, x = 10, 20, 30
    pc = np.array([x + 0.5, y + 0.5, z + 0.5])
    want = sum(0.05 * math.exp(-np.sum((pc - cen[b]) ** 2) / (2 * s[b] ** 2)) for b in range(8))
    assert vol[z, y, x] == np.float32(want)
    assert 0 < vol.max() <= 0.05 * 8


def test_first_hop_is_the_entry_brick_x_fastest():
    # rank = bx + nb * (by + nb * bz): the entry point eye + t0 * dir, computed
    # here in float64, fixes which brick the first sample lies in
    n, w, h, brick = 64, 16, 16, 32
    cam = inputs.c0_camera(n, w, h)
    vol = inputs.c0_volume(n)
    res = oracle.c0_render(vol, cam, w, h, brick=brick)
    checked = 0
    for y in range(h):
        for x in range(w):
            hit, d, t0, t1 = oracle.c0_primary(cam, n, x, y)
            if not hit:
                continue
            p = cam[:3].astype(np.float64) + d.astype(np.float64) * (t0 + 0.25)
            if np.any(np.abs(p - np.round(p / brick) * brick) < 1e-3):
                continue  # too close to a brick face to call in float64
            b = np.clip(np.floor(p / brick), 0, n // brick - 1).astype(int)
            nb = n // brick
            assert res["hops"][y * w + x, 0] == b[0] + nb * (b[1] + nb * b[2])
            checked += 1
    assert checked > 100
