"""gs_project_bwd_exclusive: with every Gaussian in exactly one view, the 3D
gradients it writes over whatever the buffers held equal, bit for bit, those
gs_project_bwd adds to zeroed buffers (zeros for culled projections); the
binding refuses views that share Gaussians; and a BatchRenderer over such
views takes this path and skips the fill of the 3D gradients without
changing its gradients (Sec. 3.2, 3.2.1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import batch as GB
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline
from paper_2312_02121_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _scenes(views_ranges, n=20000, seed=3):
    w = wl.small_case(seed, n, 200, 120)
    sc, cam = w.scenes[0], w.views[0].camera
    params = pipeline.Params.from_scene(sc, "cuda")
    views = B.Views([cam] * len(views_ranges), views_ranges, device="cuda")
    return params, views, w.eps2d


def _both(params, views, eps2d):
    pr = pipeline.project(views, params, eps2d)
    P, N = views.P, params.n
    gen = torch.Generator("cuda").manual_seed(5)
    g2 = torch.randn(P, 2, device="cuda", generator=gen)
    gc = torch.randn(P, 3, device="cuda", generator=gen)
    out = []
    for exclusive in (False, True):
        fill = 7.0 if exclusive else 0.0
        gm, gq, gs = (torch.full((N, k), fill, device="cuda") for k in (3, 4, 3))
        fn = B.gs_project_bwd_exclusive if exclusive else B.gs_project_bwd
        fn(views, params.means, params.quats, params.scales, eps2d, pr["touched"], g2, gc, gm, gq, gs)
        torch.cuda.synchronize()
        out.append((gm, gq, gs))
    return pr, out


def test_exclusive_writes_what_the_accumulating_call_adds_to_zero():
    params, views, eps2d = _scenes([(0, 20000)])
    pr, ((a_m, a_q, a_s), (b_m, b_q, b_s)) = _both(params, views, eps2d)
    assert torch.equal(a_m, b_m) and torch.equal(a_q, b_q) and torch.equal(a_s, b_s)
    culled = pr["touched"] == 0
    assert culled.any() and (~culled).any()
    assert (b_m[culled] == 0).all() and (b_q[culled] == 0).all() and (b_s[culled] == 0).all()


def test_exclusive_over_disjoint_views_and_refusal_of_shared_gaussians():
    # two views of two halves of the Gaussians (one scene drawn twice, disjoint ranges)
    params, views, eps2d = _scenes([(0, 12000), (12000, 8000)])
    _, ((a_m, a_q, a_s), (b_m, b_q, b_s)) = _both(params, views, eps2d)
    assert torch.equal(a_m, b_m) and torch.equal(a_q, b_q) and torch.equal(a_s, b_s)
    params, views, eps2d = _scenes([(0, 12000), (8000, 12000)])
    pr = pipeline.project(views, params, eps2d)
    z = lambda *s: torch.zeros(*s, device="cuda")
    with pytest.raises(B.GsError, match="overlap"):
        B.gs_project_bwd_exclusive(views, params.means, params.quats, params.scales, eps2d, pr["touched"],
                                   z(views.P, 2), z(views.P, 3), z(params.n, 3), z(params.n, 4), z(params.n, 3))


def test_batch_renderer_skips_the_fill_with_the_same_gradients():
    w = wl.small_case(4, 20000, 200, 120)
    params, views, ranges, targets = GB.workload_views(w, "cuda")
    cap = GB.exact_capacity(params, views, w.eps2d)
    grads = []
    for exclusive in (True, False):
        r = GB.BatchRenderer(params, views, cap, targets, w.eps2d, deterministic=True)
        assert r.exclusive
        if not exclusive:  # the accumulating path, with the step's fill over the whole buffer
            r.exclusive, r.step_fill = False, r.grad_flat
        for _ in range(2):  # the second step finds the first one's gradients in the buffers
            r.step_eager()
        torch.cuda.synchronize()
        grads.append({k: v.clone() for k, v in r.grads().items()})
    for k in grads[0]:
        assert torch.equal(grads[0][k], grads[1][k]), k
    # views that share Gaussians keep the accumulating path
    two = B.Views([w.views[0].camera] * 2, [(0, 20000), (0, 20000)], device="cuda")
    assert not GB.BatchRenderer(params, two, 2 * cap, None, w.eps2d).exclusive
