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
