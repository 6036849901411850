"""gs_rasterize_fwd_l2: the forward with the L2 loss folded in gives the same
image, final transmittance and last indices as gs_rasterize_fwd, the same
dL/dC as gs_l2_loss on that image (bit for bit), and a loss as close to the
exact sum as gs_l2_loss's (their fp32 sums run in different orders).  On one
view with a background, and on a 64-view batch walked as the tuner may walk
it (persistent grid, longest first)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import batch as GB
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline
from paper_2312_02121_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _both(views, f, params, target, inv_norm, background=None, config=None):
    pix = views.pixels
    out = []
    for fused in (False, True):
        rgb, Tf = torch.empty(pix, 3, device="cuda"), torch.empty(pix, device="cuda")
        last = torch.empty(pix, dtype=torch.int32, device="cuda")
        dL, loss = torch.empty(pix, 3, device="cuda"), torch.zeros(1, device="cuda")
        args = (views, f.means2d, f.conics, params.opacities, params.colors, f.isect_ids, f.tile_ranges, background,
                rgb, Tf, last)
        if fused:
            B.gs_rasterize_fwd_l2(*args, target, inv_norm, dL, loss, config=config)
        else:
            B.gs_rasterize_fwd(*args, None, config)
            B.gs_l2_loss(rgb, target, inv_norm, dL, loss)
        torch.cuda.synchronize()
        out.append((rgb, Tf, last, dL, float(loss.item())))
    (r0, t0, l0, g0, s0), (r1, t1, l1, g1, s1) = out
    assert torch.equal(r0, r1) and torch.equal(t0, t1) and torch.equal(l0, l1)
    assert torch.equal(g0, g1)
    # both sums are fp32 over millions of terms in different orders: each within 1e-5 of the exact sum
    exact = inv_norm * float(((r0.double() - target.double()) ** 2).sum())
    assert abs(s0 - exact) <= 1e-5 * exact and abs(s1 - exact) <= 1e-5 * exact, (s0, s1, exact)


def test_folded_loss_one_view_with_background():
    w = wl.fwdbwd_100k_1024x768()
    cam, sc = w.views[0].camera, w.scenes[0]
    params = pipeline.Params.from_scene(sc, "cuda")
    views = B.Views([cam], [(0, sc.n)], device="cuda")
    f = pipeline.forward(views, params, w.eps2d)
    target = torch.as_tensor(w.targets[0], device="cuda").reshape(-1, 3).contiguous()
    bg = torch.tensor([0.2, 0.5, 0.9], device="cuda")
    _both(views, f, params, target, 1.0 / target.numel(), background=bg)


def test_folded_loss_batched_views_persistent_longest_first():
    w = wl.batch_views_500k_64()
    params, views, ranges, targets = GB.workload_views(w, "cuda")
    f = pipeline.forward(views, params, w.eps2d)
    order = torch.empty(views.T, dtype=torch.int32, device="cuda")
    ws = torch.empty(max(B.gs_tile_order_workspace_size(views.T), 1), dtype=torch.uint8, device="cuda")
    B.gs_tile_order(f.tile_ranges, views.T, ws, order)
    cfg = B.RasterConfig(True, 0, order, device="cuda")
    target = targets.reshape(-1, 3).contiguous()
    _both(views, f, params, target, 1.0 / target.numel(), config=cfg)


def test_folded_loss_refuses_what_it_does_not_compute():
    w = wl.forward_1k_128()
    cam, sc = w.views[0].camera, w.scenes[0]
    params = pipeline.Params.from_scene(sc, "cuda")
    views = B.Views([cam], [(0, sc.n)], device="cuda")
    f = pipeline.forward(views, params, w.eps2d)
    pix = views.pixels
    rgb, Tf = torch.empty(pix, 3, device="cuda"), torch.empty(pix, device="cuda")
    last = torch.empty(pix, dtype=torch.int32, device="cuda")
    args = (views, f.means2d, f.conics, params.opacities, params.colors, f.isect_ids, f.tile_ranges, None, rgb, Tf,
            last)
    with pytest.raises(B.GsError):
        B.gs_rasterize_fwd_l2(*args, None, 1.0, torch.empty(pix, 3, device="cuda"), None)
    with pytest.raises(B.GsError):
        B.gs_rasterize_fwd_l2(*args, torch.zeros(pix, 3, device="cuda"), 1.0, None, None)
