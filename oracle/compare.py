"""Comparison of an fp32 result with the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests, the smoke
check and the benchmark's CPU-baseline leg (which also reports the GPU
result's error against the oracle it times) use it.  It holds no arithmetic of
the method; it decides which pixels an fp32 and an fp64 evaluation of Eq. 7
may legitimately disagree on, and measures the distance between two results.

Where fp32 and fp64 may disagree (Reading O10): a threshold test of Sec. 2.2
(alpha >= 1/255, the 0.99 clamp, the 1e-4 transmittance cut-off) that lies
within ``margin_rel`` (relative) of its threshold, or a Gaussian whose 3-sigma
box edge lies within ``rect_margin_px`` of a tile line, so that the tile beyond
that line may or may not list it -- there only the pixels where the Gaussian's
alpha reaches 1/255 can change.
"""
from __future__ import annotations

import numpy as np

from . import ALPHA_MIN, TILE, tiles


def uncertain_pixels(margin, proj: dict, width: int, height: int, opacities=None, pixels=None,
                     margin_rel: float = 1e-4, rect_margin_px: float = 1e-3) -> np.ndarray:
    """Mask of the pixels an fp32 evaluation may legitimately composite
    differently from the oracle.

    ``margin``: the oracle's per-pixel threshold margin (``rasterize``'s
    ``margin``), shaped [height, width] for a whole image or [n] for the
    linear pixel ids ``pixels``.  ``proj``: the oracle projection (needs
    means2d, cov2d, conics, rects, valid, rect_margin).  The result has the
    shape of ``margin``."""
    margin = np.asarray(margin)
    bad = margin < margin_rel
    if "cov2d" not in proj:
        return bad
    TX, TY = tiles(width, height)
    flat = bad.reshape(-1)
    if pixels is None:
        xs_all = ys_all = None
    else:
        pixels = np.asarray(pixels, np.int64)
        xs_all, ys_all = pixels % width, pixels // width
    m2, cov, con = proj["means2d"], proj["cov2d"], proj["conics"]
    op = np.ones(len(m2)) if opacities is None else np.asarray(opacities, np.float64)
    near = np.nonzero((np.asarray(proj["rect_margin"]) < rect_margin_px) & (np.asarray(proj["valid"]) > 0))[0]
    for n in near:
        x0, y0, x1, y1 = (int(v) for v in proj["rects"][n])
        rx, ry = 3 * np.sqrt(cov[n, 0]), 3 * np.sqrt(cov[n, 2])
        for axis, side, edge in ((0, 0, m2[n, 0] - rx), (0, 1, m2[n, 0] + rx), (1, 0, m2[n, 1] - ry),
                                 (1, 1, m2[n, 1] + ry)):
            k = int(np.floor(edge / TILE + 0.5))
            if abs(edge - TILE * k) >= rect_margin_px:
                continue
            t = k - 1 if side == 0 else k  # the tile that may flip
            if axis == 0:
                if not 0 <= t < TX:
                    continue
                xa, xb = TILE * t, min(TILE * (t + 1), width)
                ya, yb = TILE * max(y0 - 1, 0), min(TILE * min(y1 + 1, TY), height)
            else:
                if not 0 <= t < TY:
                    continue
                ya, yb = TILE * t, min(TILE * (t + 1), height)
                xa, xb = TILE * max(x0 - 1, 0), min(TILE * min(x1 + 1, TX), width)
            if xa >= xb or ya >= yb:
                continue
            if pixels is None:
                ys, xs = np.mgrid[ya:yb, xa:xb]
                idx = (ys * width + xs).ravel()
                xs, ys = xs.ravel(), ys.ravel()
            else:
                sel = np.nonzero((xs_all >= xa) & (xs_all < xb) & (ys_all >= ya) & (ys_all < yb))[0]
                if not len(sel):
                    continue
                idx, xs, ys = sel, xs_all[sel], ys_all[sel]
            dx, dy = m2[n, 0] - (xs + 0.5), m2[n, 1] - (ys + 0.5)
            sigma = 0.5 * (con[n, 0] * dx * dx + 2 * con[n, 1] * dx * dy + con[n, 2] * dy * dy)
            hit = op[n] * np.exp(-sigma) >= ALPHA_MIN * (1 - 1e-3)
            flat[idx[hit]] = True
    return bad


def rel_l2(a, b) -> float:
    """||a - b|| / ||b|| over all entries (float64)."""
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
