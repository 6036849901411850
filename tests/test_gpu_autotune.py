"""gs_autotune through the C ABI: it times every candidate tile walk and
backward batch shape of a projected and sorted batch, returns the fastest
(the least of the times it reports), refuses a candidate whose shape is not
compiled, and its choice renders exactly what the default walk renders."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import batch as GB
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import workloads as wl
from gpu_helpers import np_, rel_l2

pytestmark = pytest.mark.gpu


def _batch():
    a = wl.small_case(71, 2500, 120, 90, log_scale_mu=-2.6)
    b = wl.small_case(72, 1800, 96, 64, log_scale_mu=-2.8)
    cams = wl.sphere_cameras(np.random.default_rng(73), 3, 4.0, [(64, 48), (50, 37), (80, 80)],
                             focal_range=(60.0, 120.0))
    views = [wl.View(0, a.views[0].camera), wl.View(1, b.views[0].camera)] + [wl.View(i % 2, c) for i, c in
                                                                          enumerate(cams)]
    trng = np.random.default_rng(74)
    w = wl.Workload("tune", [a.scenes[0], b.scenes[0]], views, [wl.target_image(trng, v.camera) for v in views])
    params, vs, ranges, targets = GB.workload_views(w)
    cap = GB.exact_capacity(params, vs, w.eps2d)
    return w, params, vs, targets, cap


def test_autotune_picks_the_fastest_of_every_candidate_and_renders_the_same():
    w, params, views, targets, cap = _batch()
    r = GB.BatchRenderer(params, views, cap, targets, w.eps2d, deterministic=True)
    best = GB.autotune(r, key="test", use_cache=False)
    cands = B.gs_autotune_default_candidates()
    assert len(best["all"]) == len(cands) == 20
    assert [{k: c[k] for k in B.TUNING_FIELDS} for c in best["all"]] == cands
    assert all(c["ms"] > 0 for c in best["all"])
    assert best["ms"] == min(c["ms"] for c in best["all"])
    assert {k: best[k] for k in B.TUNING_FIELDS} in cands
    # the tuned renderer renders what the default one renders
    r.step_eager()
    tuned = GB.BatchRenderer(params, views, cap, targets, w.eps2d, GB.config(best), bool(best["longest_first"]),
                             deterministic=True)
    tuned.step_eager()
    torch.cuda.synchronize()
    assert torch.equal(r.rgb, tuned.rgb) and torch.equal(r.last_idx, tuned.last_idx)
    for k, v in r.grads().items():
        assert rel_l2(np_(tuned.grads()[k]), np_(v)) <= 1e-5, k


def test_autotune_takes_an_explicit_list_and_refuses_an_unknown_shape():
    w, params, views, targets, cap = _batch()
    r = GB.BatchRenderer(params, views, cap, targets, w.eps2d)
    r.forward()
    ws = torch.empty(B.gs_autotune_workspace_size(views.P, params.n, views.T, cap, views.pixels), dtype=torch.uint8,
                     device="cuda")
    two = [dict(persistent=0, ctas_per_sm=0, longest_first=0, bwd_pixels=1, bwd_batch=96),
           dict(persistent=1, ctas_per_sm=2, longest_first=1, bwd_pixels=2, bwd_batch=64)]
    best, res = B.gs_autotune(views, params.n, r.means2d, r.conics, params.opacities, params.colors, r.isect_ids,
                              r.tile_ranges, r.K, cap, ws, two, repeats=2)
    assert [{k: x[k] for k in B.TUNING_FIELDS} for x in res] == two
    assert best["ms"] == min(x["ms"] for x in res)
    bad = [dict(persistent=0, ctas_per_sm=0, longest_first=0, bwd_pixels=3, bwd_batch=0)]
    with pytest.raises(B.GsError) as e:
        B.gs_autotune(views, params.n, r.means2d, r.conics, params.opacities, params.colors, r.isect_ids,
                      r.tile_ranges, r.K, cap, ws, bad)
    assert e.value.code == B.GS_ERR_INVALID_ARG
    with pytest.raises(B.GsError):  # too small a workspace
        B.gs_autotune(views, params.n, r.means2d, r.conics, params.opacities, params.colors, r.isect_ids,
                      r.tile_ranges, r.K, cap, ws[:1024], two)
