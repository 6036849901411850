"""gs_bin_and_sort_static: the binning entry point for callers that cannot
allocate device memory (it takes no workspace; its scratch is a fixed array in
the library).  Its outputs must equal those of gs_bin_and_sort, which takes a
caller-allocated workspace, exactly -- these are integer lists -- on two calls
in a row with different inputs, since the fixed array keeps the previous
call's contents.  This file is named to be collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline
from paper_2312_02121_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _projected(w):
    sc = w.scenes[0]
    params = pipeline.Params.from_scene(sc, "cuda")
    views = B.Views([w.views[0].camera], [(0, sc.n)], device="cuda")
    pr = pipeline.project(views, params, w.eps2d)
    K = int(pr["K_total"].item())
    return views, pr, K


def _outputs(views, K):
    dev = "cuda"
    cap = max(K, 1)
    return dict(isect_ids=torch.full((cap,), -7, dtype=torch.int32, device=dev),
                isect_pos=torch.full((cap,), -7, dtype=torch.int32, device=dev),
                emit_start=torch.full((max(views.P, 1),), -7, dtype=torch.int32, device=dev),
                tile_ranges=torch.full((views.T, 2), -7, dtype=torch.int32, device=dev),
                K=torch.full((1,), -7, dtype=torch.int32, device=dev),
                flags=torch.zeros(1, dtype=torch.int32, device=dev))


def _with_workspace(views, pr, K):
    o = _outputs(views, K)
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(views.P, max(K, 1), views.T), dtype=torch.uint8, device="cuda")
    B.gs_bin_and_sort(views, pr["rects"], pr["depths"], pr["touched"], max(K, 1), ws, o["isect_ids"], o["isect_pos"],
                      o["emit_start"], o["tile_ranges"], o["K"], o["flags"])
    return o


def _static(views, pr, K):
    o = _outputs(views, K)
    B.gs_bin_and_sort_static(views, pr["rects"], pr["depths"], pr["touched"], max(K, 1), o["isect_ids"],
                             o["isect_pos"], o["emit_start"], o["tile_ranges"], o["K"], o["flags"])
    return o


def _same(a, b, pr, K):
    vis = pr["touched"] > 0
    assert int(a["K"].item()) == int(b["K"].item()) == K
    assert int(a["flags"].item()) == int(b["flags"].item()) == 0
    for k in ("isect_ids", "isect_pos", "tile_ranges"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(a["emit_start"][vis], b["emit_start"][vis])


def test_static_scratch_entry_point_matches_workspace_entry_point():
    cases = [wl.fwdbwd_100k_1024x768(seed=3), wl.small_case(21, 5000, 333, 211, log_scale_mu=-2.5)]
    prepared = [_projected(w) for w in cases]
    for views, pr, K in prepared:
        assert views.P <= 131072 and K <= 1048576
    ref = [_with_workspace(*p) for p in prepared]
    got = [_static(*p) for p in prepared]  # two calls in a row, different inputs
    torch.cuda.synchronize()
    for (views, pr, K), a, b in zip(prepared, ref, got):
        _same(a, b, pr, K)
    # and again in the other order: the fixed scratch holds the other case's data
    again = _static(*prepared[0])
    torch.cuda.synchronize()
    _same(ref[0], again, prepared[0][1], prepared[0][2])


def test_static_scratch_entry_point_rejects_oversized_problems():
    views, pr, K = _projected(wl.small_case(22, 100, 64, 64))
    o = _outputs(views, K)
    with pytest.raises(B.GsError) as e:
        B.gs_bin_and_sort_static(views, pr["rects"], pr["depths"], pr["touched"], 1048577, o["isect_ids"],
                                 o["isect_pos"], o["emit_start"], o["tile_ranges"], o["K"], o["flags"])
    assert e.value.code == B.GS_ERR_INVALID_ARG and "must not exceed" in str(e.value)
