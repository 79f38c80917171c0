"""GPU parity: brick-partitioned absorption marching against the oracle.

The oracle marches every ray through the unpartitioned grid; the GPU path
marches it brick by brick, forwarding it between ranks.  tau is the same sum
in the same float order, so T agrees to a few ulp of expf (tolerance: max
relative error 1e-5), the hop sequence of every ray equals the sequence of
bricks its samples cross, and the image does not depend on the partition.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import inputs, rafi

from gpu_util import dev, stream, to_dev

pytestmark = pytest.mark.gpu

RAY_BYTES = 48


def render(vol, cam, n, brick, w, h, max_hops=16):
    nb = n // brick
    R = nb ** 3
    s = stream()
    dvol = to_dev(vol.reshape(-1))
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c0_make_bricks(dvol, n, brick, bricks, s)
    image = torch.full((w * h,), -1.0, dtype=torch.float32, device=dev())
    hop_log = torch.full((w * h, max_hops), -1, dtype=torch.int32, device=dev())
    hop_count = torch.zeros(w * h, dtype=torch.int32, device=dev())
    with rafi.Context(R, RAY_BYTES, w * h) as ctx:
        rounds = rafi.rf_c0_render(ctx.handle, bricks, cam, n, brick, w, h, image, hop_log, max_hops, hop_count,
                                   stream=s)
        stats = rafi.rf_stats(ctx.handle)
    torch.cuda.synchronize()
    return dict(T=image.cpu().numpy(), hops=hop_log.cpu().numpy(), hop_count=hop_count.cpu().numpy(),
                rounds=rounds, stats=stats)


def test_blob_volume_8_ranks_matches_oracle():
    n, w, h, brick = 64, 128, 128, 32
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    got = render(vol, cam, n, brick, w, h)
    want = oracle.c0_render(vol, cam, w, h, brick=brick)
    assert np.all(got["T"] > 0)
    rel = np.abs(got["T"] - want["T"]) / want["T"]
    assert rel.max() <= 1e-5, rel.max()
    np.testing.assert_array_equal(got["hop_count"], want["hop_count"])
    np.testing.assert_array_equal(got["hops"], want["hops"])
    # a straight ray crosses at most 4 bricks of a 2x2x2 grid
    assert got["rounds"] <= 4 and want["hop_count"].max() <= 4
    assert got["stats"].exchanges == got["rounds"] + 1


@pytest.mark.parametrize("n,brick,w,h", [(64, 16, 96, 80), (32, 8, 64, 64), (16, 4, 33, 17)])
def test_other_partitions_match_oracle(n, brick, w, h):
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    got = render(vol, cam, n, brick, w, h, max_hops=32)
    want = oracle.c0_render(vol, cam, w, h, brick=brick, max_hops=32)
    rel = np.abs(got["T"] - want["T"]) / want["T"]
    assert rel.max() <= 1e-5, rel.max()
    np.testing.assert_array_equal(got["hops"], want["hops"])


def test_partition_independence():
    # forwarding does not change what is computed: 1, 8 and 64 ranks give identical bits
    n, w, h = 64, 128, 128
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    imgs = [render(vol, cam, n, b, w, h, max_hops=32)["T"] for b in (64, 32, 16)]
    np.testing.assert_array_equal(imgs[0].view(np.uint32), imgs[1].view(np.uint32))
    np.testing.assert_array_equal(imgs[0].view(np.uint32), imgs[2].view(np.uint32))


def test_missing_rays_and_constant_volume():
    # camera aimed past the box: every ray misses, T = 1, nothing is forwarded
    n = 16
    vol = np.full((n, n, n), 0.05, np.float32)
    cam = inputs.camera((8.0, 8.0, -32.0), (8.0, 200.0, 8.0), (0.0, 0.0, 1.0), 5.0, 16, 16)
    got = render(vol, cam, n, 8, 16, 16)
    assert np.all(got["T"] == 1.0) and got["rounds"] == 0 and got["stats"].numActive == 0
    # constant field: T = exp(-0.05 * 0.5 * samples)
    cam = inputs.c0_camera(n, 24, 24)
    got = render(vol, cam, n, 8, 24, 24)
    want = oracle.c0_render(vol, cam, 24, 24, brick=8)
    np.testing.assert_allclose(got["T"], np.exp(-0.025 * want["nsamp"]), rtol=2e-5)


def test_raygen_then_manual_rounds():
    # the step-by-step API gives the same image as rf_c0_render
    n, w, h, brick = 32, 40, 40, 16
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    ref = render(vol, cam, n, brick, w, h)
    s = stream()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c0_make_bricks(to_dev(vol.reshape(-1)), n, brick, bricks, s)
    image = torch.zeros(w * h, dtype=torch.float32, device=dev())
    with rafi.Context(8, RAY_BYTES, w * h) as ctx:
        rafi.rf_c0_raygen(ctx.handle, cam, n, brick, w, h, image, s)
        st, active = rafi.rf_exchange(ctx.handle, s)
        rounds = 0
        while active:
            rafi.rf_c0_march(ctx.handle, bricks, n, brick, image, stream=s)
            st, active = rafi.rf_exchange(ctx.handle, s)
            rounds += 1
    torch.cuda.synchronize()
    assert rounds == ref["rounds"]
    np.testing.assert_array_equal(image.cpu().numpy(), ref["T"])


def test_graph_form_matches_host_loop_and_is_relaunched():
    # the rounds in a kept CUDA graph (conditional while node) give the host
    # loop's image bit for bit, also when the kept graph is relaunched and
    # after an argument change rebuilds it
    n, w, h, brick = 64, 128, 128, 32
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    want = render(vol, cam, n, brick, w, h)
    s = stream()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c0_make_bricks(to_dev(vol.reshape(-1)), n, brick, bricks, s)
    image = torch.zeros(w * h, dtype=torch.float32, device=dev())
    hop_log = torch.full((w * h, 16), -1, dtype=torch.int32, device=dev())
    hop_count = torch.zeros(w * h, dtype=torch.int32, device=dev())
    with rafi.Context(8, RAY_BYTES, w * h) as ctx:
        for rep in range(3):
            image.fill_(-1.0)
            hop_log.fill_(-1)
            rounds = rafi.rf_c0_render_graph(ctx.handle, bricks, cam, n, brick, w, h, image, hop_log, 16, hop_count,
                                             stream=s)
            torch.cuda.synchronize()
            assert rounds == want["rounds"]
            np.testing.assert_array_equal(image.cpu().numpy().view(np.uint32), want["T"].view(np.uint32))
            np.testing.assert_array_equal(hop_log.cpu().numpy(), want["hops"])
        # another camera: the kept graph is rebuilt
        cam2 = inputs.camera((32.0, 90.0, -40.0), (32.0, 32.0, 32.0), (0.0, 1.0, 0.0), 40.0, w, h)
        want2 = render(vol, cam2, n, brick, w, h)
        rounds = rafi.rf_c0_render_graph(ctx.handle, bricks, cam2, n, brick, w, h, image, hop_log, 16, hop_count,
                                         stream=s)
        torch.cuda.synchronize()
        assert rounds == want2["rounds"]
        np.testing.assert_array_equal(image.cpu().numpy().view(np.uint32), want2["T"].view(np.uint32))


def render_tma(vol, cam, n, brick, w, h, form=rafi.RF_FORM_HOST_LOOP):
    s = stream()
    dvol = to_dev(vol.reshape(-1))
    sb = torch.zeros(rafi.c0_scalar_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c0_make_scalar_bricks(dvol, n, brick, sb, s)
    image = torch.full((w * h,), -1.0, dtype=torch.float32, device=dev())
    with rafi.Context((n // brick) ** 3, RAY_BYTES, w * h) as ctx:
        rounds = rafi.rf_c0_render_tma(ctx.handle, sb, cam, n, brick, w, h, image, stream=s, form=form)
        if form == rafi.RF_FORM_GRAPH:  # a second frame relaunches the kept graph
            image.fill_(-1.0)
            assert rafi.rf_c0_render_tma(ctx.handle, sb, cam, n, brick, w, h, image, stream=s, form=form) == rounds
    torch.cuda.synchronize()
    return image.cpu().numpy(), rounds, sb


@pytest.mark.parametrize("form", [rafi.RF_FORM_HOST_LOOP, rafi.RF_FORM_GRAPH], ids=["host_loop", "graph"])
@pytest.mark.parametrize("n,brick,w,h", [(64, 32, 128, 128), (64, 16, 96, 80), (16, 4, 33, 17)])
def test_tma_staged_bricks_give_the_same_image(n, brick, w, h, form):
    # bricks staged whole in shared memory by a 3-D tensor copy: same corners,
    # same float operations, so the image equals the quad-brick path's bit for
    # bit (and so the oracle's within its tolerance)
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    img, rounds, sb = render_tma(vol, cam, n, brick, w, h, form)
    ref = render(vol, cam, n, brick, w, h)
    np.testing.assert_array_equal(img.view(np.uint32), ref["T"].view(np.uint32))
    assert rounds == ref["rounds"]
    want = oracle.c0_render(vol, cam, w, h, brick=brick)
    assert np.max(np.abs(img - want["T"]) / want["T"]) <= 1e-5
    # the scalar bricks hold the clamped halo (rows padded to whole 16-byte units)
    nb, S, X = n // brick, brick + 2, rafi.c0_scalar_row(brick)
    b = sb.cpu().numpy().reshape(nb ** 3, S, S, X)
    r = nb ** 3 - 1  # the last brick: its halo leaves the volume on three faces
    bx = by = bz = nb - 1
    idx = lambda o, l: np.clip(o - 1 + l, 0, n - 1)  # noqa: E731
    zz, yy, xx = np.meshgrid(idx(bz * brick, np.arange(S)), idx(by * brick, np.arange(S)),
                             idx(bx * brick, np.arange(X)), indexing="ij")
    np.testing.assert_array_equal(b[r], vol[zz, yy, xx])


def test_tma_refuses_bricks_beyond_shared_memory():
    # a 128^3 brick with its halo (132 x 130 x 130 floats, 8.9 MB) cannot be staged whole
    n, brick = 256, 128
    sb = torch.zeros(16, dtype=torch.float32, device=dev())
    image = torch.zeros(16, dtype=torch.float32, device=dev())
    with rafi.Context(8, RAY_BYTES, 16) as ctx:
        st = rafi.lib().rf_c0_march_tma(ctx.handle, sb.data_ptr(), n, brick, image.data_ptr(), None)
    assert st == rafi.RF_ERR_ARG and "shared memory" in rafi.rf_last_error()
