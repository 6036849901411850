"""Binning (Sec. 2.2) on synthetic tile rectangles and depths, bit-exact against
the oracle's brute-force binning.  The depth sort runs only the radix passes
the spread of the visible depth keys needs, so the cases span that spread:
depths over four decades (all passes), a narrow band, equal depths (ties, in
projection order) and no visible projection at all."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import workloads as wl

W, H = 256, 128  # 16 x 8 tiles


def synthetic(spread: str, P: int = 6000, seed: int = 3):
    rng = np.random.default_rng(seed)
    TX, TY = (W + 15) // 16, (H + 15) // 16
    x0 = rng.integers(0, TX, P)
    y0 = rng.integers(0, TY, P)
    x1 = np.minimum(x0 + rng.integers(1, 5, P), TX)
    y1 = np.minimum(y0 + rng.integers(1, 4, P), TY)
    rects = np.stack([x0, y0, x1, y1], axis=1).astype(np.int16)
    visible = rng.random(P) > 0.1
    if spread == "wide":
        depths = 10.0 ** rng.uniform(-1.9, 1.99, P)  # 0.013 .. 98: a 30-bit key spread
    elif spread == "narrow":
        depths = rng.uniform(5.0, 5.01, P)
    elif spread == "equal":
        depths = np.full(P, 3.0)
    else:  # nothing visible
        depths = rng.uniform(1.0, 50.0, P)
        visible[:] = False
    depths = depths.astype(np.float32)
    touched = np.where(visible, (x1 - x0) * (y1 - y0), 0).astype(np.int32)
    return rects, depths, touched, TX, TY


def key_spread_bits(depths, touched):
    k = depths[touched > 0].view(np.int32).astype(np.int64)
    return int(k.max() - k.min()).bit_length() if len(k) else 0


@pytest.mark.gpu
@pytest.mark.parametrize("spread", ["wide", "narrow", "equal", "none"])
def test_depth_sort_passes_follow_the_key_spread(spread):
    rects, depths, touched, TX, TY = synthetic(spread)
    bits = key_spread_bits(depths, touched)
    assert {"wide": bits > 24, "narrow": 8 < bits <= 24, "equal": bits == 0, "none": bits == 0}[spread]
    ids_o, ranges_o = oracle.bin_tiles(rects, depths, (touched > 0).astype(np.int32), TX, TY)
    dev = "cuda"
    views = B.Views([wl.camera_at_distance(3.0, W, H, 100.0)], [(0, len(depths))], device=dev)
    P, T = views.P, views.T
    cap = max(int(touched.sum()), 1)
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, T), dtype=torch.uint8, device=dev)
    ids = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    pos = torch.empty(cap, dtype=torch.int32, device=dev)
    es = torch.empty(P, dtype=torch.int32, device=dev)
    tr = torch.full((T, 2), -7, dtype=torch.int32, device=dev)
    K = torch.empty(1, dtype=torch.int32, device=dev)
    fl = torch.zeros(1, dtype=torch.int32, device=dev)
    t = lambda a: torch.as_tensor(a, device=dev)
    for isect_pos, emit_start in ((None, None), (pos, es)):
        B.gs_bin_and_sort(views, t(rects), t(depths), t(touched), cap, ws, ids, isect_pos, emit_start, tr, K, fl)
        torch.cuda.synchronize()
        k = int(K.item())
        assert k == len(ids_o) == int(touched.sum()) and int(fl.item()) == 0
        np.testing.assert_array_equal(ids.cpu().numpy()[:k], ids_o)
        rng_gpu = tr.cpu().numpy()
        nonempty = ranges_o[:, 1] > ranges_o[:, 0]
        np.testing.assert_array_equal(rng_gpu[nonempty], ranges_o[nonempty])
        assert (rng_gpu[~nonempty, 1] - rng_gpu[~nonempty, 0] <= 0).all()


def _bin(views, rects, depths, touched, cap):
    dev = "cuda"
    P, T = views.P, views.T
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, T), dtype=torch.uint8, device=dev)
    ids = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    tr = torch.full((T, 2), -7, dtype=torch.int32, device=dev)
    K = torch.empty(1, dtype=torch.int32, device=dev)
    fl = torch.zeros(1, dtype=torch.int32, device=dev)
    B.gs_bin_and_sort(views, rects, depths, touched, cap, ws, ids, None, None, tr, K, fl)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), tr.cpu().numpy(), int(K.item()), int(fl.item())


@pytest.mark.gpu
def test_binning_over_several_views_matches_the_oracle():
    # two 16x8-tile views (256 tiles in all), uneven projection counts, rectangles up to 4x3 tiles: global
    # tile ids follow each view's tile offset, and the depth sort runs over both views at once
    parts = [synthetic("wide", P=5000, seed=5), synthetic("narrow", P=3500, seed=6)]
    rects = np.concatenate([p[0] for p in parts])
    depths = np.concatenate([p[1] for p in parts])
    touched = np.concatenate([p[2] for p in parts])
    TX, TY = parts[0][3], parts[0][4]
    cams = [wl.camera_at_distance(3.0, W, H, 100.0)] * 2
    views = B.Views(cams, [(0, 5000), (0, 3500)], device="cuda")
    t = lambda a: torch.as_tensor(a, device="cuda")
    cap = int(touched.sum())
    got = _bin(views, t(rects), t(depths), t(touched), cap)
    # the oracle bins each view on its own; global tile ids follow the views' tile offsets, and the
    # pairs of view 1 follow those of view 0
    ids0, rng0 = oracle.bin_tiles(rects[:5000], depths[:5000], (touched[:5000] > 0).astype(np.int32), TX, TY)
    ids1, rng1 = oracle.bin_tiles(rects[5000:], depths[5000:], (touched[5000:] > 0).astype(np.int32), TX, TY)
    ids_o = np.concatenate([ids0, ids1 + 5000])
    rng_o = np.concatenate([rng0, rng1 + len(ids0)])
    ids, tr, k, fl = got
    assert k == len(ids_o) == cap and fl == 0
    np.testing.assert_array_equal(ids[:k], ids_o)
    ne = rng_o[:, 1] > rng_o[:, 0]
    np.testing.assert_array_equal(tr[ne], rng_o[ne])
    assert (tr[~ne, 1] - tr[~ne, 0] <= 0).all()

