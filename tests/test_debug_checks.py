"""The GS_DEBUG invariant checks (paper_2312_02121_gb300/debug.py) on host
tensors: valid binning and compositing outputs pass, and each kind of
corruption the checks exist for is reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2312_02121_gb300 import build as gsbuild
from paper_2312_02121_gb300 import debug

W, H = 40, 20  # 3 x 2 tiles, the last column and row partial


@pytest.fixture(scope="module")
def binding():
    from paper_2312_02121_gb300 import binding
    gsbuild.build()
    binding.load()
    return binding


def _binning():
    rng = np.random.default_rng(1)
    P, TX, TY = 50, 3, 2
    x0 = rng.integers(0, TX, P)
    y0 = rng.integers(0, TY, P)
    rects = np.stack([x0, y0, np.minimum(x0 + rng.integers(1, 3, P), TX),
                      np.minimum(y0 + rng.integers(1, 3, P), TY)], 1).astype(np.int32)
    depths = rng.uniform(1, 5, P).astype(np.float32)
    valid = (rng.random(P) > 0.2).astype(np.int32)
    ids, ranges = oracle.bin_tiles(rects, depths, valid, TX, TY)
    ranges = np.where((ranges[:, 1] > ranges[:, 0])[:, None], ranges, 0)  # empty tiles as the sort leaves them
    return P, torch.tensor(ids, dtype=torch.int32), torch.tensor(ranges, dtype=torch.int32), len(ids)


def test_valid_binning_passes_and_corruptions_are_reported(binding):
    P, ids, ranges, K = _binning()
    cap = K + 5
    Kt, fl = torch.tensor([K], dtype=torch.int32), torch.zeros(1, dtype=torch.int32)
    debug.check_binning(P, cap, ids, ranges, Kt, fl)
    bad = ids.clone()
    bad[K // 2] = P  # a projection that does not exist
    with pytest.raises(binding.GsError, match="names projection"):
        debug.check_binning(P, cap, bad, ranges, Kt, fl)
    gap = ranges.clone()
    t = int(torch.nonzero(gap[:, 1] > gap[:, 0])[0])
    gap[t, 1] -= 1  # the next tile no longer starts where this one ends
    with pytest.raises(binding.GsError, match="not consecutive|span"):
        debug.check_binning(P, cap, ids, gap, Kt, fl)
    with pytest.raises(binding.GsError, match="pair count"):
        debug.check_binning(P, K - 1, ids, ranges, Kt, fl)
    # an overflowed sort is documented as incomplete: nothing to check
    debug.check_binning(P, cap, bad, gap, Kt, torch.tensor([binding.GS_FLAG_CAPACITY], dtype=torch.int32))


def _frame(binding):
    from paper_2312_02121_gb300 import workloads as wl
    views = binding.Views([wl.camera_at_distance(3.0, W, H, 50.0)], [(0, 1)], device="cpu")
    T = 6
    lens = np.array([3, 0, 2, 4, 1, 0])
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    ranges = np.stack([np.where(lens > 0, starts, 0), np.where(lens > 0, starts + lens, 0)], 1)
    rng = np.random.default_rng(2)
    last = np.empty((H, W), np.int32)
    for y in range(H):
        for x in range(W):
            s, e = ranges[(y // 16) * 3 + x // 16]
            last[y, x] = rng.integers(s - 1, e) if e > s else s - 1
    out = torch.rand(W * H, 3)
    Tf = torch.rand(W * H) * 0.9 + 0.05
    assert views.T == T and views.pixels == W * H
    return views, torch.tensor(ranges, dtype=torch.int32), out, Tf, torch.tensor(last.reshape(-1))


def test_valid_frame_passes_and_corruptions_are_reported(binding):
    views, ranges, out, Tf, last = _frame(binding)
    debug.check_forward(views, ranges, out, Tf, last)
    nan = out.clone()
    nan[7, 1] = float("nan")
    with pytest.raises(binding.GsError, match="non-finite"):
        debug.check_forward(views, ranges, nan, Tf, last)
    t0 = Tf.clone()
    t0[3] = 0.0
    with pytest.raises(binding.GsError, match="transmittance"):
        debug.check_forward(views, ranges, out, t0, last)
    far = last.clone()
    far[W * 17 + 33] = 100  # pixel (33, 17) in tile 5, whose list is empty
    with pytest.raises(binding.GsError, match="last index"):
        debug.check_forward(views, ranges, out, Tf, far)
    debug.check_gradients([("a", torch.zeros(4)), ("b", None)])
    with pytest.raises(binding.GsError, match="gradient g"):
        debug.check_gradients([("g", torch.tensor([0.0, float("inf")]))])


def test_codes_match_the_binding(binding):
    assert (debug.GS_FLAG_CAPACITY, debug.GS_ERR_INVALID_ARG) == (binding.GS_FLAG_CAPACITY, binding.GS_ERR_INVALID_ARG)


def test_checks_are_off_unless_asked(monkeypatch):
    monkeypatch.delenv("GS_DEBUG", raising=False)
    assert not debug.enabled()
    monkeypatch.setenv("GS_DEBUG", "1")
    assert debug.enabled() is (not (torch.cuda.is_available() and torch.cuda.is_current_stream_capturing()))


def test_pixel_tiles_follow_the_view_layout(binding):
    # two views of different sizes: packed pixels map to their own view's tiles, offset by the
    # tiles of the views before
    from paper_2312_02121_gb300 import workloads as wl
    cams = [wl.camera_at_distance(3.0, 40, 20, 50.0), wl.camera_at_distance(3.0, 17, 33, 50.0)]
    views = binding.Views(cams, [(0, 1), (0, 1)], device="cpu")
    tiles = debug._pixel_tiles(views, "cpu").numpy()
    assert len(tiles) == views.pixels == 40 * 20 + 17 * 33
    expect = [(y // 16) * 3 + x // 16 for y in range(20) for x in range(40)]
    expect += [6 + (y // 16) * 2 + x // 16 for y in range(33) for x in range(17)]
    assert tiles.tolist() == expect and views.T == 6 + 2 * 3
