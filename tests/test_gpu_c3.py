"""GPU parity: the differentiable partitioned emission-absorption renderer.

Forward: images and per-sample colours against the oracle's float render
(max relative error 1e-5; the sums are in the same order, expf may differ by
an ulp).  Adjoint: against the oracle's FP64 reverse-accumulation adjoint
(max-norm relative error 1e-4) and, at the configured size (256^3 over 2x2x2
ranks, 512x512 at 4 spp), against central finite differences (eps = 1e-3,
loss summed in FP64) on 32 voxels (relative error 1e-2).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import ea_autograd, inputs, rafi

from gpu_util import dev, stream, to_dev

pytestmark = pytest.mark.gpu


def gpu_render(vol, cam, brick, w, h, spp, seed=3):
    n = vol.shape[0]
    R = (n // brick) ** 3
    s = stream()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c0_make_bricks(to_dev(vol.reshape(-1)), n, brick, bricks, s)
    rayC = torch.zeros(w * h * spp, dtype=torch.float32, device=dev())
    img = torch.zeros(w * h, dtype=torch.float32, device=dev())
    with rafi.Context(R, 64, w * h * spp) as ctx:
        rounds = rafi.rf_c3_render(ctx.handle, bricks, cam, n, brick, w, h, spp, seed, rayC, img, stream=s)
    return img.cpu().numpy(), rayC.cpu().numpy(), bricks, rayC, rounds


def test_forward_matches_oracle():
    n, brick, w, h, spp = 64, 32, 64, 48, 4
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    img, rayC, _, _, rounds = gpu_render(vol, cam, brick, w, h, spp)
    wimg, wray = oracle.c3_render(vol, cam, w, h, spp)
    assert rounds <= 4
    np.testing.assert_allclose(rayC, wray, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(img, wimg, rtol=1e-5, atol=1e-7)
    assert wimg.max() > 0.05


def test_forward_partition_independent():
    n, w, h, spp = 64, 48, 48, 2
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    a = gpu_render(vol, cam, 64, w, h, spp)[0]
    b = gpu_render(vol, cam, 32, w, h, spp)[0]
    c = gpu_render(vol, cam, 16, w, h, spp)[0]
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    np.testing.assert_array_equal(a.view(np.uint32), c.view(np.uint32))


def test_adjoint_matches_fp64_oracle():
    n, brick, w, h, spp = 32, 16, 32, 32, 4
    vol = inputs.c0_volume(n) * 3.0
    cam = inputs.c0_camera(n, w, h)
    _, _, bricks, rayC, _ = gpu_render(vol, cam, brick, w, h, spp)
    gimg = np.random.default_rng(2).normal(size=w * h).astype(np.float32)
    grad = torch.zeros(n ** 3, dtype=torch.float32, device=dev())
    s = stream()
    with rafi.Context((n // brick) ** 3, 64, w * h * spp) as ctx:
        rafi.rf_c3_adjoint(ctx.handle, bricks, cam, n, brick, w, h, spp, 3, rayC, to_dev(gimg), grad, stream=s)
    got = grad.cpu().numpy().reshape(n, n, n)
    dLdC = np.repeat(gimg.astype(np.float64) / spp, spp)
    want, _ = oracle.c3_adjoint_f64(vol, cam, w, h, spp, dLdC)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 1e-4, err


def test_autograd_and_finite_differences_at_full_size():
    # 256^3 blobs over 2x2x2 ranks of 128^3, 512x512 at 4 spp, L2 loss against
    # a target rendered from the perturbed density
    n, brick, w, h, spp = 256, 128, 512, 512, 4
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    target = ea_autograd.render(to_dev(inputs.c3_target_volume(vol)), cam, brick, w, h, spp).detach()
    v = to_dev(vol).requires_grad_(True)
    img = ea_autograd.render(v, cam, brick, w, h, spp)
    loss = ((img - target) ** 2).mean()
    loss.backward()
    grad = v.grad.detach().cpu().numpy()
    assert np.abs(grad).max() > 0

    def loss64(volume):
        im = ea_autograd.render(volume, cam, brick, w, h, spp).detach().cpu().numpy().astype(np.float64)
        return ((im - target.cpu().numpy().astype(np.float64)) ** 2).mean()

    rng = np.random.default_rng(7)
    strong = np.argwhere(np.abs(grad) > 0.1 * np.abs(grad).max())
    picks = strong[rng.choice(len(strong), size=32, replace=False)]
    eps = 1e-3
    base = to_dev(vol)
    worst = 0.0
    for z, y, x in picks:
        vp = base.clone()
        vm = base.clone()
        vp[z, y, x] += eps
        vm[z, y, x] -= eps
        step = float(vp[z, y, x].item()) - float(vm[z, y, x].item())
        fd = (loss64(vp) - loss64(vm)) / step
        worst = max(worst, abs(fd - grad[z, y, x]) / abs(grad[z, y, x]))
    assert worst <= 1e-2, worst
