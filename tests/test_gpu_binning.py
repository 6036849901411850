"""Binning (Sec. 2.2) on synthetic tile rectangles and depths, bit-exact against
the oracle's brute-force binning.  The depth sort runs only the radix passes
the spread of the visible depth keys needs, so the cases span that spread:
depths over four decades (all passes), a narrow band, equal depths (ties, in
projection order) and no visible projection at all.  Long tile lists (about
3000 pairs a tile, and 63,000 in one) with many equal depths, and a capacity
overflow, complete the cases."""
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



def _tile_of_pair(rects, p, j, TX, tile_offset=0):
    x0, y0, x1, _ = rects[p]
    w = x1 - x0
    return tile_offset + (y0 + j // w) * TX + x0 + j % w


def _long_lists(case, seed=11):
    # a 4x2-tile view; "long": about 3000 pairs per tile; "xl": every rectangle holds tile 0 (63,000
    # visible pairs) and half of them tile 1
    rng = np.random.default_rng(seed)
    TX, TY = 4, 2
    if case == "long":
        P = 12000
        x0, y0 = rng.integers(0, TX, P), rng.integers(0, TY, P)
        x1, y1 = np.minimum(x0 + rng.integers(1, 3, P), TX), np.minimum(y0 + rng.integers(1, 3, P), TY)
    else:
        P = 70000
        x0, y0 = np.zeros(P, np.int64), np.zeros(P, np.int64)
        x1, y1 = rng.integers(1, 3, P), np.ones(P, np.int64)
    rects = np.stack([x0, y0, x1, y1], axis=1).astype(np.int16)
    # half the depths from eight values (ties, broken by projection index), half spread over four decades
    depths = np.where(rng.random(P) < 0.5, rng.choice(np.linspace(1.0, 2.0, 8), P),
                      10.0 ** rng.uniform(-1.5, 2.5, P)).astype(np.float32)
    visible = rng.random(P) > 0.1
    touched = np.where(visible, (x1 - x0) * (y1 - y0), 0).astype(np.int32)
    return rects, depths, touched, TX, TY


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["long", "xl"])
def test_long_lists_match_the_oracle(case):
    rects, depths, touched, TX, TY = _long_lists(case)
    P = len(depths)
    ids_o, rng_o = oracle.bin_tiles(rects, depths, (touched > 0).astype(np.int32), TX, TY)
    lengths = rng_o[:, 1] - rng_o[:, 0]
    assert lengths.max() > (16384 * 2 if case == "xl" else 2048)
    dev = "cuda"
    views = B.Views([wl.camera_at_distance(3.0, 16 * TX, 16 * TY, 100.0)], [(0, P)], device=dev)
    assert views.T == TX * TY
    cap = int(touched.sum())
    t = lambda a: torch.as_tensor(a, device=dev)
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, views.T), dtype=torch.uint8, device=dev)
    ids = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    pos = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    es = torch.full((P,), -7, dtype=torch.int32, device=dev)
    tr = torch.full((views.T, 2), -7, dtype=torch.int32, device=dev)
    K = torch.empty(1, dtype=torch.int32, device=dev)
    fl = torch.zeros(1, dtype=torch.int32, device=dev)
    for isect_pos, emit_start in ((None, None), (pos, es)):
        B.gs_bin_and_sort(views, t(rects), t(depths), t(touched), cap, ws, ids, isect_pos, emit_start, tr, K, fl)
        torch.cuda.synchronize()
        assert int(K.item()) == len(ids_o) == cap and int(fl.item()) == 0
        np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
        r = tr.cpu().numpy()
        ne = lengths > 0
        np.testing.assert_array_equal(r[ne], rng_o[ne])
        assert (r[~ne, 1] == r[~ne, 0]).all()
    # pair j of projection p (emission emit_start[p] + j) sits in its own tile's list
    e_s, p_s, sid = es.cpu().numpy(), pos.cpu().numpy(), ids.cpu().numpy()
    tile_of_slot = np.repeat(np.arange(views.T), lengths)
    for p in np.nonzero(touched)[0][:: max(1, P // 3000)]:
        for j in range(touched[p]):
            i = p_s[e_s[p] + j]
            assert sid[i] == p and tile_of_slot[i] == _tile_of_pair(rects, p, j, TX)


@pytest.mark.gpu
def test_capacity_overflow_stays_in_bounds():
    # half the pairs fit: the flag is set, K counts all of them, every range and written index stays in
    # its buffer, and every inverse position the deterministic reduction may read is a valid slot
    rects, depths, touched, TX, TY = _long_lists("long", seed=12)
    P = len(depths)
    dev = "cuda"
    views = B.Views([wl.camera_at_distance(3.0, 16 * TX, 16 * TY, 100.0)], [(0, P)], device=dev)
    total = int(touched.sum())
    cap = total // 2
    t = lambda a: torch.as_tensor(a, device=dev)
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, views.T), dtype=torch.uint8, device=dev)
    ids = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    pos = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    es = torch.full((P,), -7, dtype=torch.int32, device=dev)
    tr = torch.full((views.T, 2), -7, dtype=torch.int32, device=dev)
    K = torch.empty(1, dtype=torch.int32, device=dev)
    fl = torch.zeros(1, dtype=torch.int32, device=dev)
    B.gs_bin_and_sort(views, t(rects), t(depths), t(touched), cap, ws, ids, pos, es, tr, K, fl)
    torch.cuda.synchronize()
    assert int(K.item()) == total and int(fl.item()) & B.GS_FLAG_CAPACITY
    r = tr.cpu().numpy()
    assert (r >= 0).all() and (r <= cap).all() and (r[:, 0] <= r[:, 1]).all()
    ids_h, pos_h = ids.cpu().numpy(), pos.cpu().numpy()
    assert ((ids_h >= 0) & (ids_h < P)).all()
    assert ((pos_h >= 0) & (pos_h < cap)).all()
