"""GPU parity: the differentiable partitioned emission-absorption renderer.

Forward: images and per-sample colours against the oracle's float render
(max relative error 1e-5; the sums are in the same order, expf may differ by
an ulp); the compensated forward returns the same colours bit for bit.

Adjoint, voxel by voxel against the oracle's FP64 reverse-accumulation
adjoint: |got - want| <= 1e-4 |want| + (3 Kmax + m + 16) 2^-24 K, where K
(from the oracle) sums over the voxel's contributions |dL/dC| (|T (0.5 e c +
20 alpha)| + |0.5 S|) times the trilinear weight, m is the number of those
contributions and Kmax the most samples a ray can take.  That is float
arithmetic's error: each contribution is the difference of its two parts,
T after k samples is a product of k expf values (up to 2 ulp each, one
rounding per product: 3 k 2^-24 relative), a part adds a few more roundings
(the 16), and the m float adds that build the voxel's sum round each partial
sum again; contributions of both signs cancel, so the scale is K, not the
gradient.  Checked on a 32^3 copy and at the configured size (256^3 over
2x2x2 ranks, 512x512 at 4 spp), where the late samples of opaque rays have
the longest, smallest suffixes.  Also at the configured size: central finite
differences of the FP64 loss (eps = 1e-3) on 32 of the strongest voxels
(relative 1e-2), and Richardson-extrapolated central differences ((4 D(eps/2)
- D(eps)) / 3, which removes the eps^2 term) on 32 voxels drawn from every
voxel the rays touch, within 1e-2 |g| + 2e-4 max|g|: a weak voxel's
difference of two float renders carries their rounding, measured at up to
7e-5 max|g| over 64 such voxels.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import ea_autograd, inputs, rafi

from gpu_util import dev, stream, to_dev

pytestmark = pytest.mark.gpu


def gpu_render(vol, cam, brick, w, h, spp, seed=3, lo=False):
    n = vol.shape[0]
    R = (n // brick) ** 3
    s = stream()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c0_make_bricks(to_dev(vol.reshape(-1)), n, brick, bricks, s)
    rayC = torch.zeros(w * h * spp, dtype=torch.float32, device=dev())
    rayClo = torch.zeros(w * h * spp, dtype=torch.float32, device=dev()) if lo else None
    img = torch.zeros(w * h, dtype=torch.float32, device=dev())
    with rafi.Context(R, 64, w * h * spp) as ctx:
        rounds = rafi.rf_c3_render(ctx.handle, bricks, cam, n, brick, w, h, spp, seed, rayC, img, stream=s,
                                   ray_c_lo=rayClo)
    if lo:
        return img.cpu().numpy(), rayC.cpu().numpy(), bricks, rayC, rounds, rayClo
    return img.cpu().numpy(), rayC.cpu().numpy(), bricks, rayC, rounds


def gpu_adjoint(vol, cam, brick, w, h, spp, gimg, lo=True):
    n = vol.shape[0]
    _, _, bricks, rayC, _, rayClo = gpu_render(vol, cam, brick, w, h, spp, lo=True)
    grad = torch.zeros(n ** 3, dtype=torch.float32, device=dev())
    with rafi.Context((n // brick) ** 3, 64, w * h * spp) as ctx:
        rafi.rf_c3_adjoint(ctx.handle, bricks, cam, n, brick, w, h, spp, 3, rayC, to_dev(gimg), grad,
                           stream=stream(), ray_c_lo=rayClo if lo else None)
    return grad.cpu().numpy().reshape(n, n, n).astype(np.float64)


def adjoint_excess(got, want, kappa, count, n):
    """Largest |got - want| / bound over the voxels (1 = at the bound), bound =
    1e-4 |want| + (3 Kmax + count + 16) 2^-24 kappa, Kmax = ceil(2 sqrt(3) n)."""
    kmax = int(np.ceil(2.0 * np.sqrt(3.0) * n))
    bound = 1e-4 * np.abs(want) + (3 * kmax + count + 16) * 2.0 ** -24 * kappa
    return float(np.max(np.abs(got - want) / (bound + 1e-300)))


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


def test_compensated_forward_keeps_the_colours():
    # with the low parts requested, C is still the plain float sum, bit for
    # bit, and each low part is below the rounding the sum can have made
    n, brick, w, h, spp = 64, 32, 64, 48, 4
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    img, rayC, _, _, _ = gpu_render(vol, cam, brick, w, h, spp)
    img2, rayC2, _, _, _, lo = gpu_render(vol, cam, brick, w, h, spp, lo=True)
    np.testing.assert_array_equal(rayC.view(np.uint32), rayC2.view(np.uint32))
    np.testing.assert_array_equal(img.view(np.uint32), img2.view(np.uint32))
    lo = lo.cpu().numpy()
    assert np.all(np.abs(lo) <= 1e-4 * np.abs(rayC) + 1e-30)
    assert np.any(lo != 0)


def test_forward_partition_independent():
    n, w, h, spp = 64, 48, 48, 2
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    a = gpu_render(vol, cam, 64, w, h, spp)[0]
    b = gpu_render(vol, cam, 32, w, h, spp)[0]
    c = gpu_render(vol, cam, 16, w, h, spp)[0]
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    np.testing.assert_array_equal(a.view(np.uint32), c.view(np.uint32))


@pytest.mark.parametrize("n,brick,w,h,scale", [(32, 16, 32, 32, 3.0), (256, 128, 512, 512, 1.0)],
                         ids=["32^3_dense", "configured_256^3"])
def test_adjoint_matches_fp64_oracle_voxel_by_voxel(n, brick, w, h, scale):
    spp = 4
    vol = (inputs.c0_volume(n) * scale).astype(np.float32)
    cam = inputs.c0_camera(n, w, h)
    gimg = np.random.default_rng(2).normal(size=w * h).astype(np.float32)
    got = gpu_adjoint(vol, cam, brick, w, h, spp, gimg)
    dLdC = np.repeat(gimg.astype(np.float64) / spp, spp)
    want, _, kappa, count = oracle.c3_adjoint_f64(vol, cam, w, h, spp, dLdC, with_abs=True)
    assert np.all(kappa >= np.abs(want) * (1 - 1e-12))
    assert np.count_nonzero(want) > 0.5 * np.count_nonzero(kappa)
    ex = adjoint_excess(got, want, kappa, count, n)
    assert ex <= 1.0, ex
    # and in the max-norm over the grid
    assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()


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
    gmax = float(np.abs(grad).max())
    strong = np.argwhere(np.abs(grad) > 0.1 * gmax)
    touched = np.argwhere(grad != 0)
    eps = 1e-3
    base = to_dev(vol)

    def fd_at(z, y, x, e=eps):
        vp = base.clone()
        vm = base.clone()
        vp[z, y, x] += e
        vm[z, y, x] -= e
        step = float(vp[z, y, x].item()) - float(vm[z, y, x].item())
        return (loss64(vp) - loss64(vm)) / step

    def richardson_at(z, y, x):
        return (4.0 * fd_at(z, y, x, eps / 2) - fd_at(z, y, x, eps)) / 3.0

    worst_strong = max(abs(fd_at(*v) - grad[tuple(v)]) / abs(grad[tuple(v)])
                       for v in strong[rng.choice(len(strong), size=32, replace=False)])
    assert worst_strong <= 1e-2, worst_strong
    # voxels drawn from all the rays touch, weak ones included
    worst_any = max(abs(richardson_at(*v) - grad[tuple(v)]) / (1e-2 * abs(grad[tuple(v)]) + 2e-4 * gmax)
                    for v in touched[rng.choice(len(touched), size=32, replace=False)])
    assert worst_any <= 1.0, worst_any
