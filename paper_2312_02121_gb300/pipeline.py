"""Sequencing of the C-ABI stages for one forward / backward pass.

Torch only provides device memory and the stream here; every stage is one
``gs_*`` call into the CUDA library.  ``Frame`` keeps the buffers a backward
pass needs (the forward's per-pixel T_final and last index, the sorted
intersection lists) so that nothing is recomputed but Sigma', the conic and
alpha, which the backward kernels rebuild on the fly.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import torch

from . import binding as B


@dataclasses.dataclass
class Params:
    """Gaussian parameters on the device, fp32 contiguous: means [N,3],
    quats [N,4] (w,x,y,z), scales [N,3], opacities [N], colors [N,C] (C
    channels per Gaussian, 3 for RGB; fp64 paths take C = 3)."""

    means: torch.Tensor
    quats: torch.Tensor
    scales: torch.Tensor
    opacities: torch.Tensor
    colors: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def channels(self) -> int:
        return int(self.colors.shape[1]) if self.colors.dim() == 2 else 3

    @staticmethod
    def from_scene(scene, device="cuda") -> "Params":
        t = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        return Params(t(scene.means), t(scene.quats), t(scene.scales), t(scene.opacities), t(scene.colors))


def _check_params(p: Params):
    dt = p.means.dtype
    for name in ("means", "quats", "scales", "opacities", "colors"):
        x = getattr(p, name)
        if not x.is_cuda:
            raise RuntimeError(f"gsplat103 runs on CUDA only; {name} is on {x.device}")
        if x.dtype not in (torch.float32, torch.float64) or x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous float32 (or all float64)")
    if p.colors.dim() != 2 or p.colors.shape[0] != p.n or p.colors.shape[1] < 1:
        raise ValueError("colors must be [N, C]")
    if dt == torch.float64 and p.channels != 3:
        raise ValueError("the fp64 path composites 3 channels")


@dataclasses.dataclass
class Frame:
    views: B.Views
    eps2d: float
    background: Optional[torch.Tensor]
    K_capacity: int
    means2d: torch.Tensor
    conics: torch.Tensor
    depths: torch.Tensor
    rects: torch.Tensor
    touched: torch.Tensor
    K_total: torch.Tensor
    isect_ids: torch.Tensor
    isect_pos: Optional[torch.Tensor]  # deterministic frames only
    emit_start: Optional[torch.Tensor]
    tile_ranges: torch.Tensor
    K: torch.Tensor
    flags: torch.Tensor
    out_rgb: torch.Tensor
    T_final: torch.Tensor
    last_idx: torch.Tensor
    sort_ws: torch.Tensor
    n_contrib: Optional[torch.Tensor] = None
    config: Optional[B.RasterConfig] = None  # the forward's tile walk, reused by the backward

    def overflowed(self) -> bool:
        """Reads the device error word (synchronises)."""
        return bool(int(self.flags.item()) & B.GS_FLAG_CAPACITY)

    def image(self, i: int = 0) -> torch.Tensor:
        off, w, h, _ = self.views.image_slice(i)
        return self.out_rgb[off:off + w * h].view(h, w, -1)


def project(views: B.Views, p: Params, eps2d: float, stream=None):
    dev, dt = p.means.device, p.means.dtype
    P = views.P
    out = dict(
        means2d=torch.empty(P, 2, device=dev, dtype=dt), conics=torch.empty(P, 3, device=dev, dtype=dt),
        depths=torch.empty(P, device=dev), rects=torch.empty(P, 4, dtype=torch.int16, device=dev),
        touched=torch.empty(P, dtype=torch.int32, device=dev), K_total=torch.empty(1, dtype=torch.int64, device=dev))
    B.gs_project(views, p.means, p.quats, p.scales, eps2d, out["means2d"], out["conics"], out["depths"],
                 out["rects"], out["touched"], out["K_total"], stream)
    return out


def forward(views: B.Views, p: Params, eps2d: float = 0.3, background: Optional[torch.Tensor] = None,
            K_capacity: Optional[int] = None, stream=None, count_contrib: bool = False,
            config: Optional[B.RasterConfig] = None, deterministic: bool = False) -> Frame:
    """Projection, binning + sort and compositing of every view.  Without
    ``K_capacity`` the exact intersection count is read back (one sync).
    ``deterministic`` also keeps what the deterministic backward needs (the
    sorted position of every pair in emission order); the fast backward does
    without it."""
    _check_params(p)
    dev = p.means.device
    if background is not None:
        background = background.to(device=dev, dtype=p.means.dtype).contiguous()
    pr = project(views, p, eps2d, stream)
    cap = int(pr["K_total"].item()) if K_capacity is None else int(K_capacity)
    cap = max(cap, 1)
    P, T = views.P, views.T
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, T), dtype=torch.uint8, device=dev)
    isect_ids = torch.empty(cap, dtype=torch.int32, device=dev)
    isect_pos = torch.empty(cap, dtype=torch.int32, device=dev) if deterministic else None
    emit_start = torch.empty(max(P, 1), dtype=torch.int32, device=dev) if deterministic else None
    tile_ranges = torch.empty(T, 2, dtype=torch.int32, device=dev)
    K = torch.empty(1, dtype=torch.int32, device=dev)
    flags = torch.zeros(1, dtype=torch.int32, device=dev)
    B.gs_bin_and_sort(views, pr["rects"], pr["depths"], pr["touched"], cap, ws, isect_ids, isect_pos, emit_start,
                      tile_ranges, K, flags, stream)
    pix = views.pixels
    dt = p.means.dtype
    C = p.channels
    out_rgb = torch.empty(pix, C, device=dev, dtype=dt)
    T_final = torch.empty(pix, device=dev, dtype=dt)
    last_idx = torch.empty(pix, dtype=torch.int32, device=dev)
    n_contrib = torch.empty(pix, dtype=torch.int32, device=dev) if count_contrib else None
    if config is None and C <= 3:
        # the forward records its per-pair warp-box cull for the backward
        config = B.RasterConfig(device=dev, warp_hits=torch.empty(cap, dtype=torch.int32, device=dev))
    if C == 3:
        B.gs_rasterize_fwd(views, pr["means2d"], pr["conics"], p.opacities, p.colors, isect_ids, tile_ranges,
                           background, out_rgb, T_final, last_idx, n_contrib, config, stream)
    else:
        B.gs_rasterize_fwd_nc(views, C, pr["means2d"], pr["conics"], p.opacities, p.colors, isect_ids, tile_ranges,
                              background, out_rgb, T_final, last_idx, n_contrib, config, stream)
    return Frame(views, eps2d, background, cap, pr["means2d"], pr["conics"], pr["depths"], pr["rects"],
                 pr["touched"], pr["K_total"], isect_ids, isect_pos, emit_start, tile_ranges, K, flags, out_rgb,
                 T_final, last_idx, ws, n_contrib, config)


def backward(f: Frame, p: Params, dL_drgb: torch.Tensor, stream=None, deterministic: bool = False,
             config: Optional[B.RasterConfig] = None, viewmats: bool = False) -> dict:
    """Gradients of L w.r.t. means, quats, scales, opacities, colors (and the
    2D intermediates means2d, conics) given dL/dC [pixels, C].
    ``deterministic`` selects the run-to-run identical reduction (3 channels
    only).  With ``viewmats`` the result also holds dL/dT_cw of every view
    ([V, 4, 4])."""
    dev, dt = p.means.device, p.means.dtype
    views = f.views
    P, N = views.P, p.n
    if config is None:
        config = f.config
    dL_drgb = dL_drgb.contiguous().to(dt)
    C = p.channels
    # every gradient in one allocation, zeroed by one fill (the outputs are views of it)
    Pm, Nm = max(P, 1), max(N, 1)
    shapes = [(Pm, 2), (Pm, 3), (Nm,), (Nm, C), (Nm, 3), (Nm, 4), (Nm, 3)]
    if viewmats:
        shapes.append((max(views.V, 1), 4, 4))
    sizes = [math.prod(sh) for sh in shapes]
    flat = torch.zeros(sum(sizes), device=dev, dtype=dt)
    parts, off = [], 0
    for sh, n in zip(shapes, sizes):
        parts.append(flat[off:off + n].view(*sh))
        off += n
    g2, gc, go, gcol, gm, gq, gs = parts[:7]
    if deterministic and f.isect_pos is None:
        raise ValueError("the deterministic backward needs a frame from forward(..., deterministic=True)")
    if C == 3:
        nws = B.gs_rasterize_bwd_workspace_size(f.K_capacity, deterministic, dt == torch.float64)
        ws = torch.empty(nws, dtype=torch.uint8, device=dev) if nws else None
        B.gs_rasterize_bwd(views, f.means2d, f.conics, p.opacities, p.colors, f.isect_ids, f.isect_pos,
                           f.emit_start, f.touched, f.tile_ranges, f.K, f.K_capacity, f.background, f.T_final,
                           f.last_idx, dL_drgb, deterministic, ws, g2, gc, go, gcol, config, stream)
    else:
        if deterministic:
            raise ValueError("the deterministic backward composites 3 channels")
        B.gs_rasterize_bwd_nc(views, C, f.means2d, f.conics, p.opacities, p.colors, f.isect_ids, f.tile_ranges,
                              f.background, f.T_final, f.last_idx, dL_drgb, g2, gc, go, gcol, config, stream)
    gv = parts[7] if viewmats else None
    B.gs_project_bwd(views, p.means, p.quats, p.scales, f.eps2d, f.touched, g2, gc, gm, gq, gs, stream, gv)
    out = dict(means=gm[:N], quats=gq[:N], scales=gs[:N], opacities=go[:N], colors=gcol[:N], means2d=g2[:P],
               conics=gc[:P])
    if viewmats:
        out["viewmats"] = gv[:views.V]
    return out
