"""Invariant checks of the binning and compositing outputs, for debugging.

With ``GS_DEBUG=1`` in the environment the binding runs them after every
``gs_bin_and_sort``, ``gs_rasterize_fwd*`` and ``gs_rasterize_bwd*`` call (it
waits for the device to do so, and skips them while a CUDA graph is being
captured).  A violated invariant raises ``GsError``.  They catch an
out-of-range index or a broken sort where it happens instead of as a wrong
image later.  The checks only read the outputs; they compute nothing of the
method.

Binning (Sec. 2.2): the non-empty tile ranges, in tile order, cut [0, K) into
consecutive pieces, and every sorted pair names a projection below P.
Compositing (Eq. 7): images are finite, the final transmittance lies in
(0, 1], and each pixel's last composited index lies in its own tile's range
(or one before it, for a pixel that composited nothing).  Backward: every
gradient is finite.
"""
from __future__ import annotations

import os
from typing import Iterable

import torch

GS_ERR_INVALID_ARG = 1
GS_FLAG_CAPACITY = 1


def enabled() -> bool:
    """Checks run when GS_DEBUG=1 and the current stream is not being captured."""
    if os.environ.get("GS_DEBUG") != "1":
        return False
    return not (torch.cuda.is_available() and torch.cuda.is_current_stream_capturing())


def _sync():
    if torch.cuda.is_available():
        torch.cuda.synchronize()  # the call may have run on another stream


def _fail(msg: str):
    from .binding import GsError
    raise GsError(GS_ERR_INVALID_ARG, f"GS_DEBUG: {msg}")


def check_binning(P: int, K_capacity: int, isect_ids: torch.Tensor, tile_ranges: torch.Tensor, K: torch.Tensor,
                  flags: torch.Tensor) -> None:
    _sync()
    k = int(K.reshape(-1)[0].item())
    if int(flags.reshape(-1)[0].item()) & GS_FLAG_CAPACITY:
        return  # the outputs are documented as incomplete
    if k < 0 or k > K_capacity:
        _fail(f"pair count {k} outside [0, {K_capacity}]")
    r = tile_ranges.reshape(-1, 2).long().cpu()
    start, end = r[:, 0], r[:, 1]
    nonempty = end > start
    s, e = start[nonempty], end[nonempty]
    if len(s) == 0:
        if k != 0:
            _fail(f"{k} pairs but every tile range is empty")
    else:
        if int(s[0]) != 0 or int(e[-1]) != k:
            _fail(f"tile ranges span [{int(s[0])}, {int(e[-1])}), not [0, {k})")
        gaps = torch.nonzero(s[1:] != e[:-1]).reshape(-1)
        if len(gaps):
            i = int(gaps[0])
            _fail(f"tile ranges not consecutive: one ends at {int(e[i])}, the next starts at {int(s[i + 1])}")
    if k:
        ids = isect_ids.reshape(-1)[:k]
        lo, hi = int(ids.min().item()), int(ids.max().item())
        if lo < 0 or hi >= P:
            _fail(f"a sorted pair names projection {lo if lo < 0 else hi}, outside [0, {P})")


def _pixel_tiles(views, device) -> torch.Tensor:
    """Global tile id of every packed pixel of the views."""
    parts = []
    for i in range(views.V):
        v = views.host[i]
        W, H = v.cam.width, v.cam.height
        y = torch.arange(H, device=device).view(H, 1) // 16
        x = torch.arange(W, device=device).view(1, W) // 16
        parts.append((v.tile_offset + y * v.tiles_x + x).reshape(-1))
    return torch.cat(parts) if parts else torch.zeros(0, dtype=torch.int64, device=device)


def check_forward(views, tile_ranges: torch.Tensor, out: torch.Tensor, T_final: torch.Tensor,
                  last_idx: torch.Tensor) -> None:
    _sync()
    if not bool(torch.isfinite(out).all()):
        _fail("the image holds a non-finite value")
    T = T_final.reshape(-1)
    if bool(((T <= 0) | (T > 1) | ~torch.isfinite(T)).any()):
        _fail("a final transmittance lies outside (0, 1]")
    tiles = _pixel_tiles(views, last_idx.device)
    r = tile_ranges.reshape(-1, 2).long()
    start, end = r[tiles, 0], r[tiles, 1]
    last = last_idx.reshape(-1).long()
    bad = (last < start - 1) | (last >= torch.maximum(end, start))
    if bool(bad.any()):
        i = int(torch.nonzero(bad)[0])
        _fail(f"pixel {i}: last index {int(last[i])} outside its tile's range [{int(start[i])}, {int(end[i])})")


def check_gradients(named: Iterable) -> None:
    _sync()
    for name, t in named:
        if t is not None and not bool(torch.isfinite(t).all()):
            _fail(f"the gradient {name} holds a non-finite value")
