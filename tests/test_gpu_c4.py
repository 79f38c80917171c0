"""GPU parity: delta-tracking transport over 8x8x8 ranks against the oracle.

The oracle follows every path through the unpartitioned grid with the same
Philox keys; the GPU forwards it between bricks, carrying its event index and
any pending tentative collision, so paths are the same up to transcendental
ulps (logf/sinf/cosf differ between the device and the host).  The stated
tolerance is the image mean absolute error: below 1e-3 on 64x64 crops.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import inputs, rafi

from gpu_util import dev, stream, to_dev

pytestmark = pytest.mark.gpu

SMALL_VIEWS = ((64, 64), (48, 32), (32, 32), (80, 45))


def gpu_render(vol, smax, views, brick, spp, batched=True, seed=4, shape=0):
    n = vol.shape[0]
    R = (n // brick) ** 3
    s = stream()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    dv = to_dev(vol.reshape(-1))
    rafi.rf_c0_make_bricks(dv, n, brick, bricks, s)
    del dv
    npix = sum(w * h for _, w, h, _ in views)
    score = torch.zeros(npix, dtype=torch.float32, device=dev())
    paths = npix * spp
    with rafi.Context(R, 64, paths) as ctx:
        rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_TRANSPORT, rafi.RF_FORM_PERSISTENT, shape)
        rounds, fwd = rafi.rf_c4_render(ctx.handle, bricks, n, brick, smax, views, spp, seed, score, batched,
                                        stream=s)
    return score.cpu().numpy() / spp, rounds, fwd


def test_small_grid_matches_oracle():
    n, brick, spp = 128, 16, 16
    vol, smax = inputs.c4_volume(n)
    views = inputs.c4_views(n, SMALL_VIEWS)
    img, rounds, fwd = gpu_render(vol, smax, views, brick, spp)
    assert rounds > 3 and fwd > 0
    for cam, w, h, base in views[:2]:
        want, _ = oracle.c4_render_crop(vol, smax, cam, w, base, 0, 0, w, h, spp)
        got = img[base:base + w * h].reshape(h, w)
        mae = np.abs(got - want).mean()
        assert mae < 1e-3, mae
        assert (got == want).mean() > 0.98


def test_partition_independence_and_forms():
    n, spp = 128, 8
    vol, smax = inputs.c4_volume(n)
    views = inputs.c4_views(n, SMALL_VIEWS)
    a = gpu_render(vol, smax, views, 128, spp)[0]
    b = gpu_render(vol, smax, views, 32, spp)[0]
    c, rc, fc = gpu_render(vol, smax, views, 16, spp, batched=1)
    d, rd, fd = gpu_render(vol, smax, views, 16, spp, batched=0)
    e, re_, fe = gpu_render(vol, smax, views, 16, spp, batched=2)  # the graph loop
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(c, d)
    np.testing.assert_array_equal(c, e)
    assert (rc, fc) == (rd, fd) == (re_, fe)


def test_full_size_crop():
    # 1024^3 fractal noise, mean optical depth 8, 8x8x8 ranks of 128^3, the four
    # views (13,537,280 pixels) at 16 spp = 216,596,480 paths in one run
    n, brick, spp = 1024, 128, 16
    vol, smax = inputs.c4_volume(n)
    views = inputs.c4_views(n)
    img, rounds, fwd = gpu_render(vol, smax, views, brick, spp)
    assert img.size == 13537280 and 0.0 <= img.min() and img.max() <= 1.0
    cam, w, h, base = views[0]
    x0, y0 = w // 2 - 32, h // 2 - 32
    want, _ = oracle.c4_render_crop(vol, smax, cam, w, base, x0, y0, 64, 64, spp)
    got = img[base:base + w * h].reshape(h, w)[y0:y0 + 64, x0:x0 + 64]
    mae = np.abs(got - want).mean()
    assert mae < 1e-3, mae


@pytest.mark.parametrize("shape", range(len(rafi.rf_rounds_shapes(rafi.RF_POLICY_TRANSPORT))))
def test_every_persistent_shape_gives_the_host_loop_image(shape):
    # paths are drawn from counter-based streams keyed by (pixel, sample, bounce,
    # event), so every shape of the persistent kernel renders the host loop's
    # image bit for bit
    n = 64
    vol, smax = inputs.c4_volume(n)
    views = inputs.c4_views(n, sizes=((48, 32), (24, 24)))
    a, ra, fa = gpu_render(vol, smax, views, 16, 4, batched=0)
    b, rb, fb = gpu_render(vol, smax, views, 16, 4, batched=rafi.RF_FORM_TUNED, shape=shape)
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    assert (ra, fa) == (rb, fb)
