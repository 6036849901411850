"""``torch.autograd.Function`` over the CUDA forward and backward.

``render`` is the user-facing call: Gaussian parameters (tensors that may
require grad) and cameras in, one [H,W,3] image per view out; ``loss.backward()``
runs ``gs_rasterize_bwd`` and ``gs_project_bwd``.  The backward rebuilds Sigma',
the conic and alpha from the parameters instead of storing them per pixel;
only the per-pixel final transmittance and last index are kept.

Camera poses can be optimised too: pass ``viewmats`` [V, 4, 4] (world-to-camera
T_cw, which then replace the cameras' R and t) and it receives dL/dT_cw
(Eq. 20 plus the covariance route through R_cw).  The camera travels to the
GPU inside the view descriptors in fp32, so the pose is read on the host at
each forward.
"""
from __future__ import annotations

import types
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import binding as B
from . import pipeline


class RasterizeGaussians(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, scales, opacities, colors, viewmats, views: B.Views, eps2d: float,
                background: Optional[torch.Tensor], K_capacity: Optional[int]):
        p = pipeline.Params(means.detach().contiguous(), quats.detach().contiguous(),
                            scales.detach().contiguous(), opacities.detach().contiguous(),
                            colors.detach().contiguous())
        frame = pipeline.forward(views, p, eps2d, background, K_capacity)
        ctx.frame = frame
        ctx.params = p
        ctx.viewmats_dtype = None if viewmats is None else (viewmats.dtype, viewmats.device)
        ctx.mark_non_differentiable(frame.T_final)
        return frame.out_rgb, frame.T_final

    @staticmethod
    def backward(ctx, dL_drgb, _dL_dT):
        want_pose = ctx.viewmats_dtype is not None and ctx.needs_input_grad[5]
        g = pipeline.backward(ctx.frame, ctx.params, dL_drgb, viewmats=want_pose)
        gv = None
        if want_pose:
            dt, dev = ctx.viewmats_dtype
            gv = g["viewmats"].to(dtype=dt, device=dev)
        return g["means"], g["quats"], g["scales"], g["opacities"], g["colors"], gv, None, None, None, None


def _posed(cam, T: np.ndarray):
    """``cam``'s intrinsics with the extrinsics of the 4x4 world-to-camera T."""
    return types.SimpleNamespace(R=T[:3, :3], t=T[:3, 3], fx=cam.fx, fy=cam.fy, cx=cam.cx, cy=cam.cy,
                                 width=cam.width, height=cam.height, near=cam.near, far=cam.far)


def render(means: torch.Tensor, quats: torch.Tensor, scales: torch.Tensor, opacities: torch.Tensor,
           colors: torch.Tensor, cameras: Sequence, g_ranges: Optional[Sequence[Tuple[int, int]]] = None,
           eps2d: float = 0.3, background: Optional[torch.Tensor] = None,
           K_capacity: Optional[int] = None, viewmats: Optional[torch.Tensor] = None,
           views: Optional[B.Views] = None) -> List[torch.Tensor]:
    """Renders every camera; returns a list of [H, W, 3] images (views of one
    packed buffer).  ``g_ranges[i] = (g_begin, g_count)`` selects the scene
    camera i sees (default: all Gaussians).  ``viewmats`` (optional, [V, 4, 4])
    overrides the cameras' extrinsics and is differentiable.  A prepared
    ``views`` (``binding.Views``) may be passed instead of cameras and ranges.
    With ``K_capacity`` given, nothing in the call waits for the device."""
    if views is None:
        if g_ranges is None:
            g_ranges = [(0, int(means.shape[0]))] * len(cameras)
        if viewmats is not None:
            if tuple(viewmats.shape) != (len(cameras), 4, 4):
                raise ValueError(f"viewmats must be [{len(cameras)}, 4, 4], got {tuple(viewmats.shape)}")
            T = viewmats.detach().cpu().double().numpy()
            cameras = [_posed(c, T[i]) for i, c in enumerate(cameras)]
        views = B.Views(cameras, g_ranges, device=means.device)
    elif viewmats is not None:
        raise ValueError("pass viewmats with cameras, not with prepared views")
    rgb, _ = RasterizeGaussians.apply(means, quats, scales, opacities, colors, viewmats, views, eps2d, background,
                                      K_capacity)
    out = []
    for i in range(views.V):
        off, w, h, _ = views.image_slice(i)
        out.append(rgb[off:off + w * h].view(h, w, 3))
    return out


class L2Loss(torch.autograd.Function):
    """mean((rgb - target)^2) and its gradient in one kernel (gs_l2_loss)."""

    @staticmethod
    def forward(ctx, rgb, target):
        rgb, target = rgb.contiguous(), target.contiguous()
        loss = torch.zeros(1, dtype=rgb.dtype, device=rgb.device)
        dL = torch.empty_like(rgb)
        B.gs_l2_loss(rgb, target, 1.0 / max(rgb.numel(), 1), dL, loss)
        ctx.save_for_backward(dL)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dL,) = ctx.saved_tensors
        return dL * g, None


def l2_loss(rgb: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Mean squared error of an image against a target (no gradient to the target)."""
    if rgb.shape != target.shape:
        raise ValueError(f"shapes differ: {tuple(rgb.shape)} vs {tuple(target.shape)}")
    return L2Loss.apply(rgb, target.detach())
