"""torch.autograd.Function over the partitioned emission-absorption renderer.

Argument marshalling only: forward cuts the density grid into bricks and
calls rf_c3_render; backward calls rf_c3_adjoint, which forwards adjoint rays
through the same bricks and scatters dL/dsigma into the gradient grid.
"""
from __future__ import annotations

import torch

from . import rafi


class PartitionedEARender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, volume, cam, brick, width, height, spp, seed):
        n = volume.shape[0]
        ranks = (n // brick) ** 3
        vol = volume.detach().contiguous()
        s = torch.cuda.current_stream(vol.device)
        bricks = torch.empty(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device=vol.device)
        rafi.rf_c0_make_bricks(vol, n, brick, bricks, s)
        nrays = width * height * spp
        ray_c = torch.empty(nrays, dtype=torch.float32, device=vol.device)
        ray_c_lo = torch.empty(nrays, dtype=torch.float32, device=vol.device)
        image = torch.empty(width * height, dtype=torch.float32, device=vol.device)
        with rafi.Context(ranks, 64, nrays) as c:
            rafi.rf_c3_render(c.handle, bricks, cam, n, brick, width, height, spp, seed, ray_c, image, stream=s,
                              ray_c_lo=ray_c_lo)
        ctx.save_for_backward(bricks, ray_c, ray_c_lo)
        ctx.meta = (cam, n, brick, width, height, spp, seed)
        return image.view(height, width)

    @staticmethod
    def backward(ctx, grad_image):
        bricks, ray_c, ray_c_lo = ctx.saved_tensors
        cam, n, brick, width, height, spp, seed = ctx.meta
        s = torch.cuda.current_stream(bricks.device)
        grad = torch.zeros((n, n, n), dtype=torch.float32, device=bricks.device)
        g = grad_image.detach().contiguous().view(-1)
        with rafi.Context((n // brick) ** 3, 64, width * height * spp) as c:
            rafi.rf_c3_adjoint(c.handle, bricks, cam, n, brick, width, height, spp, seed, ray_c, g, grad, stream=s,
                               ray_c_lo=ray_c_lo)
        return grad, None, None, None, None, None, None


def render(volume: torch.Tensor, cam, brick: int, width: int, height: int, spp: int = 4, seed: int = 3):
    """Differentiable partitioned render of an N^3 density grid (index [z, y, x])."""
    return PartitionedEARender.apply(volume, cam, brick, width, height, spp, seed)
