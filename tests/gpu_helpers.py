"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on a
workload and collect numpy copies of everything the oracle is compared with."""
import numpy as np
import torch

import oracle
from oracle import compare
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline


def run_gpu(workload, dL_drgb=None, background=None, K_capacity=None, views_subset=None, deterministic=False):
    """Forward (and backward when dL_drgb is given) of every view of the workload.
    ``deterministic``: the deterministic backward, and a frame that keeps the
    pairs' inverse positions.  Returns (frame, params, grads or None)."""
    B.load()
    dev = "cuda"
    offs = np.cumsum([0] + [s.n for s in workload.scenes])
    params = pipeline.Params(*[torch.as_tensor(np.concatenate([getattr(s, k) for s in workload.scenes]),
                                               dtype=torch.float32).contiguous().to(dev)
                               for k in ("means", "quats", "scales", "opacities", "colors")])
    vs = workload.views if views_subset is None else [workload.views[i] for i in views_subset]
    views = B.Views([v.camera for v in vs], [(int(offs[v.scene]), workload.scenes[v.scene].n) for v in vs], device=dev)
    bg = None if background is None else torch.as_tensor(background, dtype=torch.float32, device=dev)
    frame = pipeline.forward(views, params, workload.eps2d, bg, K_capacity, deterministic=deterministic)
    grads = None
    if dL_drgb is not None:
        grads = pipeline.backward(frame, params, torch.as_tensor(dL_drgb, dtype=torch.float32, device=dev),
                                  deterministic=deterministic)
    torch.cuda.synchronize()
    return frame, params, grads


def np_(t):
    return t.detach().cpu().numpy()


def gpu_projection(frame, i=0):
    """The CUDA projection of view i as an oracle ``proj`` dict (fp32 values upcast; the conic packed
    from the library's factors, which ``conic_factors`` keeps)."""
    v = frame.views.host[i]
    s, e = v.proj_offset, v.proj_offset + v.g_count
    factors = np_(frame.conics[s:e]).astype(np.float64)
    return dict(means2d=np_(frame.means2d[s:e]).astype(np.float64), conics=compare.conic_from_factors(factors),
                conic_factors=factors, depths=np_(frame.depths[s:e]).astype(np.float64),
                rects=np_(frame.rects[s:e]).astype(np.int32), valid=(np_(frame.touched[s:e]) > 0).astype(np.int32),
                depths32=np_(frame.depths[s:e]))


def view_image(frame, i=0):
    off, w, h, _ = frame.views.image_slice(i)
    return (np_(frame.out_rgb[off:off + w * h]).reshape(h, w, 3), np_(frame.T_final[off:off + w * h]).reshape(h, w),
            np_(frame.last_idx[off:off + w * h]).reshape(h, w))


def last_gaussian_ids(frame, i=0):
    """GPU last composited Gaussian of each pixel of view i, as a projection
    index local to the view (-1 = none)."""
    off, w, h, toff = frame.views.image_slice(i)
    v = frame.views.host[i]
    last = np_(frame.last_idx[off:off + w * h]).reshape(h, w).astype(np.int64)
    ranges = np_(frame.tile_ranges)
    ids = np_(frame.isect_ids)
    TX = v.tiles_x
    ys, xs = np.mgrid[0:h, 0:w]
    tiles = toff + (ys // 16) * TX + xs // 16
    start = ranges[tiles, 0]
    out = np.full((h, w), -1, np.int64)
    has = last >= start
    has &= last >= 0
    out[has] = ids[last[has]] - v.proj_offset
    return out


def uncertain_pixels(oracle_fwd, proj, W, H, opacities=None, margin_rel=1e-4, rect_margin_px=1e-3):
    """Pixels whose result may legitimately differ between fp32 and fp64 (see
    ``oracle.compare.uncertain_pixels``), from an oracle forward of the whole
    image."""
    return compare.uncertain_pixels(oracle_fwd["margin"], proj, W, H, opacities, None, margin_rel, rect_margin_px)


rel_l2 = compare.rel_l2
