"""Comparison of an fp32 result with the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests, the smoke
check and the benchmark's CPU-baseline leg (which also reports the GPU
result's error against the oracle it times) use it.  It holds no arithmetic of
the method; it decides which pixels an fp32 and an fp64 evaluation of Eq. 7
may legitimately disagree on, and measures the distance between two results.

Where fp32 and fp64 may disagree (Reading O10):
  - a threshold test of Sec. 2.2 (alpha >= 1/255, the 0.99 clamp, the 1e-4
    transmittance cut-off) that lies within ``margin_rel`` (relative) of its
    threshold;
  - a Gaussian whose 3-sigma box edge lies within ``rect_margin_px`` of a tile
    line, so that the tile beyond that line may or may not list it -- there
    only the pixels where the Gaussian's alpha reaches 1/255 can change;
  - two Gaussians that both pass the alpha test at a pixel with depths within
    ``depth_rel`` (relative) of each other: the fp32 depths that order a tile's
    list (Sec. 2.2; ties by index, Reading O12) may order them the other way
    round, and Eq. 7 composites them in that order.  This only matters end to
    end: given the same fp32 projection both sides sort the same depths.
"""
from __future__ import annotations

import numpy as np

from . import ALPHA_MIN, TILE, tiles


def uncertain_pixels(margin, proj: dict, width: int, height: int, opacities=None, pixels=None,
                     margin_rel: float = 1e-4, rect_margin_px: float = 1e-3, depth_gap=None,
                     depth_rel: float = 1e-6) -> np.ndarray:
    """Mask of the pixels an fp32 evaluation may legitimately composite
    differently from the oracle.

    ``margin``: the oracle's per-pixel threshold margin (``rasterize``'s
    ``margin``), shaped [height, width] for a whole image or [n] for the
    linear pixel ids ``pixels``.  ``proj``: the oracle projection (needs
    means2d, cov2d, conics, rects, valid, rect_margin).  ``depth_gap``:
    ``rasterize``'s per-pixel depth gap, same shape as ``margin`` (None: depth
    order not considered).  The result has the shape of ``margin``."""
    margin = np.asarray(margin)
    bad = margin < margin_rel
    if depth_gap is not None:
        bad |= np.asarray(depth_gap) < depth_rel
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


# --------------------------------------------------------------------------
# the conic's two forms
# --------------------------------------------------------------------------
# The oracle packs the conic Y = Sigma'^-1 as (Y00, Y01, Y11) (Reading O13).
# The CUDA library stores its LDL^T factors (a, k, d): sigma = (a (dx + k dy)^2 + d dy^2) / 2,
# i.e. (Y00, Y01, Y11) = (a, a k, a k^2 + d).  These convert between the two in fp64, for the
# conic and for the gradient of L with respect to it (the chain rule through that map).

def conic_from_factors(f) -> np.ndarray:
    """Packed (Y00, Y01, Y11) [n,3] from the factors (a, k, d) [n,3]."""
    f = np.asarray(f, np.float64)
    a, k, d = f[:, 0], f[:, 1], f[:, 2]
    return np.stack([a, a * k, a * k * k + d], 1)


def conic_factors(packed) -> np.ndarray:
    """Factors (a, k, d) [n,3] of packed conics (a = Y00, k = Y01 / Y00, d = Y11 - Y01^2 / Y00);
    rows with Y00 = 0 (culled projections) give zeros."""
    y = np.asarray(packed, np.float64)
    a = y[:, 0]
    safe = np.where(a != 0, a, 1.0)
    k = np.where(a != 0, y[:, 1] / safe, 0.0)
    d = np.where(a != 0, y[:, 2] - y[:, 1] * y[:, 1] / safe, 0.0)
    return np.stack([a, k, d], 1)


def conic_grad_to_factors(g_packed, packed) -> np.ndarray:
    """dL/d(a, k, d) from dL/d(Y00, Y01, Y11) at the conic ``packed``."""
    g = np.asarray(g_packed, np.float64)
    f = conic_factors(packed)
    a, k = f[:, 0], f[:, 1]
    return np.stack([g[:, 0] + k * g[:, 1] + k * k * g[:, 2], a * g[:, 1] + 2 * a * k * g[:, 2], g[:, 2]], 1)


def conic_grad_from_factors(g_factors, factors) -> np.ndarray:
    """dL/d(Y00, Y01, Y11) from dL/d(a, k, d) at the factors ``factors``; zero rows where a = 0."""
    g = np.asarray(g_factors, np.float64)
    f = np.asarray(factors, np.float64)
    a, k = f[:, 0], f[:, 1]
    inv = np.where(a != 0, 1.0 / np.where(a != 0, a, 1.0), 0.0)
    return np.stack([g[:, 0] - k * inv * g[:, 1] + k * k * g[:, 2], inv * g[:, 1] - 2 * k * g[:, 2], g[:, 2]], 1)


def with_factored_conic_grad(grads: dict, packed) -> dict:
    """A copy of an oracle gradient dict whose "conics" entry is dL/d(a, k, d) at ``packed``."""
    out = dict(grads)
    out["conics"] = conic_grad_to_factors(grads["conics"], packed)
    return out
