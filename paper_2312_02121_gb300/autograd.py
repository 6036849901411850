"""``torch.autograd.Function`` over the CUDA forward and backward.

``render`` is the user-facing call: Gaussian parameters (tensors that may
require grad) and cameras in, one [H,W,3] image per view out; ``loss.backward()``
runs ``gs_rasterize_bwd`` and ``gs_project_bwd``.  The backward rebuilds Sigma',
the conic and alpha from the parameters instead of storing them per pixel;
only the per-pixel final transmittance and last index are kept.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import binding as B
from . import pipeline


class RasterizeGaussians(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, scales, opacities, colors, views: B.Views, eps2d: float,
                background: Optional[torch.Tensor], K_capacity: Optional[int]):
        p = pipeline.Params(means.detach().contiguous(), quats.detach().contiguous(),
                            scales.detach().contiguous(), opacities.detach().contiguous(),
                            colors.detach().contiguous())
        frame = pipeline.forward(views, p, eps2d, background, K_capacity)
        ctx.frame = frame
        ctx.params = p
        ctx.mark_non_differentiable(frame.T_final)
        return frame.out_rgb, frame.T_final

    @staticmethod
    def backward(ctx, dL_drgb, _dL_dT):
        g = pipeline.backward(ctx.frame, ctx.params, dL_drgb)
        return g["means"], g["quats"], g["scales"], g["opacities"], g["colors"], None, None, None, None


def render(means: torch.Tensor, quats: torch.Tensor, scales: torch.Tensor, opacities: torch.Tensor,
           colors: torch.Tensor, cameras: Sequence, g_ranges: Optional[Sequence[Tuple[int, int]]] = None,
           eps2d: float = 0.3, background: Optional[torch.Tensor] = None,
           K_capacity: Optional[int] = None) -> List[torch.Tensor]:
    """Renders every camera; returns a list of [H, W, 3] images (views of one
    packed buffer).  ``g_ranges[i] = (g_begin, g_count)`` selects the scene
    camera i sees (default: all Gaussians)."""
    if g_ranges is None:
        g_ranges = [(0, int(means.shape[0]))] * len(cameras)
    views = B.Views(cameras, g_ranges, device=means.device)
    rgb, _ = RasterizeGaussians.apply(means, quats, scales, opacities, colors, views, eps2d, background, K_capacity)
    out = []
    for i in range(views.V):
        off, w, h, _ = views.image_slice(i)
        out.append(rgb[off:off + w * h].view(h, w, 3))
    return out
