"""Pins for the oracle's emission-absorption renderer and its FP64 adjoint.

  * constant density: C = 20 sigma (1 - exp(-sigma n / 2)) for a ray with n
    samples (the geometric series of T alpha c);
  * the float forward agrees with the FP64 recomputation inside the adjoint
    (one-hot dL/dC returns a ray's C in double);
  * the FP64 adjoint is the derivative of the FP64 forward: central finite
    differences of sum(dL/dC * C) match it voxel by voxel;
  * jittered samples stay inside their pixel.
"""
import math

import numpy as np

import oracle
from paper_2605_30294_gb300 import inputs


def test_constant_density_closed_form():
    n, w, h, spp = 16, 12, 10, 2
    sig = 0.03
    vol = np.full((n, n, n), sig, np.float32)
    cam = inputs.c0_camera(n, w, h)
    img, rayC = oracle.c3_render(vol, cam, w, h, spp)
    # sample counts from the marching oracle's ray setup (same camera, no jitter there),
    # so compare with the closed form through the density-independent count:
    # C depends on the sample count only, and every count gives 20 s (1 - e^{-s n/2})
    vals = np.unique(np.round(rayC, 6))
    ns = np.arange(0, 200)
    closed = 20 * sig * (1 - np.exp(-sig * ns / 2.0))
    for v in vals:
        assert np.min(np.abs(closed - v)) < 2e-6 * max(1.0, v)
    assert rayC.max() > 0 and np.isclose(img, rayC.reshape(-1, spp).mean(1), rtol=1e-6).all()


def test_float_forward_matches_double_recomputation():
    n, w, h, spp = 16, 8, 8, 2
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    img, rayC = oracle.c3_render(vol, cam, w, h, spp)
    for ray in (0, 17, 40, w * h * spp - 1):
        g = np.zeros(w * h * spp)
        g[ray] = 1.0
        _, acc = oracle.c3_adjoint_f64(vol, cam, w, h, spp, g)
        assert abs(acc - rayC[ray]) <= 2e-5 * max(1.0, abs(acc))


def test_adjoint_is_the_derivative_of_the_forward():
    n, w, h, spp = 12, 8, 6, 2
    vol = inputs.c0_volume(n) * 4.0
    cam = inputs.c0_camera(n, w, h)
    rng = np.random.default_rng(4)
    g = rng.normal(size=w * h * spp)
    grad, _ = oracle.c3_adjoint_f64(vol, cam, w, h, spp, g)
    idx = np.argsort(np.abs(grad).ravel())[-12:]
    eps = 1e-3
    for flat in idx:
        vp = vol.astype(np.float64).copy().ravel()
        vm = vp.copy()
        vp[flat] += eps
        vm[flat] -= eps
        # the functional is evaluated in double inside the adjoint; perturb a float copy
        _, ap = oracle.c3_adjoint_f64(vp.reshape(vol.shape).astype(np.float32), cam, w, h, spp, g)
        _, am = oracle.c3_adjoint_f64(vm.reshape(vol.shape).astype(np.float32), cam, w, h, spp, g)
        fd = (ap - am) / (np.float32(vp[flat]) - np.float32(vm[flat]))
        assert abs(fd - grad.ravel()[flat]) <= 2e-3 * np.abs(grad).max()


def test_jitter_stays_inside_the_pixel():
    # Philox(key {seed,5}, ctr {pixel, s}) top 24 bits: u, v in [0, 1)
    r = oracle.philox4x32_10(np.array([[5, s, 0, 0] for s in range(16)], np.uint32), np.array([3, 5], np.uint32))
    u = (r[:, 0] >> 8) / 2**24
    v = (r[:, 1] >> 8) / 2**24
    assert np.all((u >= 0) & (u < 1) & (v >= 0) & (v < 1)) and len(set(u.tolist())) == 16


def test_target_volume_recipe():
    vol = inputs.c0_volume(16)
    t = inputs.c3_target_volume(vol)
    ratio = t / np.maximum(vol, 1e-30)
    assert np.all((ratio >= 0.9 - 1e-6) & (ratio <= 1.1 + 1e-6))
    assert abs(ratio.mean() - 1.0) < 0.01


def test_fp64_adjoint_absolute_sums():
    # gabs (a sum over the magnitudes of each contribution's two parts) bounds
    # |grad| voxel by voxel, does not change with the sign of dL/dC while grad
    # flips, and scales with |dL/dC|
    n, w, h, spp = 16, 12, 12, 2
    vol = inputs.c0_volume(n) * 4.0
    cam = inputs.c0_camera(n, w, h)
    g = np.random.default_rng(5).normal(size=w * h * spp)
    grad, _, ab, cnt = oracle.c3_adjoint_f64(vol, cam, w, h, spp, g, with_abs=True)
    grad2, _, ab2, cnt2 = oracle.c3_adjoint_f64(vol, cam, w, h, spp, -2.0 * g, with_abs=True)
    # eight corners per sample (clamped corners count on the voxel they land on)
    assert cnt.sum() % 8 == 0 and np.array_equal(cnt, cnt2)
    assert np.all((cnt > 0) >= (ab > 0))
    grad3, _ = oracle.c3_adjoint_f64(vol, cam, w, h, spp, g)
    np.testing.assert_array_equal(grad, grad3)
    assert np.all(ab >= np.abs(grad) - 1e-15 * ab.max())
    assert np.count_nonzero(ab) > 0 and np.any(ab > np.abs(grad) * (1 + 1e-9))
    np.testing.assert_allclose(ab2, 2.0 * ab, rtol=1e-12)
    np.testing.assert_allclose(grad2, -2.0 * grad, rtol=1e-12, atol=1e-15 * ab.max())
