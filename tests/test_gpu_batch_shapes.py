"""Every compiled batch shape of the compositing backward (pixels per thread x
staged batch, GsRasterConfig.bwd_pixels / bwd_batch) computes the gradients
of Sec. 3.1: against the FP64 oracle given the CUDA projection, bit-identical
run to run in the deterministic mode, and equal to the default shape up to the
fp32 order of the fast mode's atomics -- with the forward's warp ballots and
with the cull recomputed, on a one-CTA-per-tile and a persistent walk."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import compare
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline
from paper_2312_02121_gb300 import workloads as wl
from gpu_helpers import gpu_projection, np_

pytestmark = pytest.mark.gpu

SHAPES = [(1, 64), (1, 96), (2, 64), (2, 128)]
KEYS = ("means2d", "conics", "opacities", "colors", "means", "quats", "scales")


@pytest.fixture(scope="module")
def frame():
    # a ragged image (partial tiles at the right and bottom), dense enough that tiles hold several batches
    w = wl.small_case(51, 6000, 203, 141, log_scale_mu=-2.5, opacity_logit_mu=0.6)
    sc = w.scenes[0]
    params = pipeline.Params.from_scene(sc, "cuda")
    views = B.Views([w.views[0].camera], [(0, sc.n)], device="cuda")
    G = torch.tensor(np.random.default_rng(52).standard_normal((views.pixels, 3)).astype(np.float32), device="cuda")
    return w, params, views, G


def _run(frame, px, batch, deterministic, persistent=False, hits=True):
    w, params, views, G = frame
    cap = None
    f = pipeline.forward(views, params, w.eps2d, deterministic=True)
    cfg = B.RasterConfig(persistent, 2, device="cuda", bwd_pixels=px, bwd_batch=batch,
                         warp_hits=f.config.warp_hits if hits else None)
    if hits:  # refill the ballots under this walk (same forward, same words)
        f = pipeline.forward(views, params, w.eps2d, deterministic=True, config=cfg)
    g = pipeline.backward(f, params, G, deterministic=deterministic, config=cfg)
    torch.cuda.synchronize()
    return f, {k: np_(v).astype(np.float64) for k, v in g.items()}


@pytest.mark.parametrize("px,batch", SHAPES)
def test_shape_matches_oracle_and_is_deterministic(frame, px, batch):
    w, params, views, G = frame
    cam, sc = w.views[0].camera, w.scenes[0]
    f, g1 = _run(frame, px, batch, True)
    _, g2 = _run(frame, px, batch, True)
    for k in KEYS:
        np.testing.assert_array_equal(g1[k], g2[k], err_msg=k)
    gp = gpu_projection(f)
    o = oracle.rasterize(gp, sc.opacities, sc.colors, cam.width, cam.height)
    ok = (o["margin"] >= 1e-4).reshape(-1)
    assert ok.mean() > 0.99
    Gm = np.where(ok[:, None], np_(G), 0.0)
    # the masked gradient through the same shape
    G_saved = G.clone()
    G.copy_(torch.as_tensor(Gm, dtype=torch.float32, device="cuda"))
    try:
        _, gm = _run(frame, px, batch, True)
    finally:
        G.copy_(G_saved)
    ob = compare.with_factored_conic_grad(oracle.rasterize_bwd(gp, sc.opacities, sc.colors, cam.width, cam.height, Gm),
                                          gp["conics"])
    for k in ("means2d", "conics", "opacities", "colors"):
        assert compare.rel_l2(gm[k], ob[k]) <= 1e-4, (px, batch, k)


@pytest.mark.parametrize("px,batch", SHAPES)
@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("hits", [True, False])
def test_shape_agrees_with_default_shape(frame, px, batch, persistent, hits):
    _, ref = _run(frame, 1, 96, True)
    _, det = _run(frame, px, batch, True, persistent, hits)
    _, fast = _run(frame, px, batch, False, persistent, hits)
    for k in KEYS:
        # the deterministic mode sums each tile's warps in a fixed order, but the warps differ between
        # shapes; the fast mode also varies in the order of its atomics
        assert compare.rel_l2(det[k], ref[k]) <= (5e-5 if k == "quats" else 1e-5), (k, px, batch)
        assert compare.rel_l2(fast[k], ref[k]) <= (5e-5 if k == "quats" else 1e-5), (k, px, batch)


def test_cull_off_leaves_each_shape_unchanged(frame):
    outs = {}
    for cull in (True, False):
        if not cull:
            os.environ["GS_NO_CULL"] = "1"
        try:
            for px, batch in SHAPES:
                outs[(cull, px, batch)] = _run(frame, px, batch, True, hits=False)[1]
        finally:
            os.environ.pop("GS_NO_CULL", None)
    for px, batch in SHAPES:
        for k in KEYS:
            np.testing.assert_array_equal(outs[(True, px, batch)][k], outs[(False, px, batch)][k], err_msg=k)


def test_unknown_shape_is_refused(frame):
    w, params, views, G = frame
    f = pipeline.forward(views, params, w.eps2d)
    for px, batch in ((3, 0), (1, 128), (2, 96), (1, 32)):
        cfg = B.RasterConfig(device="cuda", bwd_pixels=px, bwd_batch=batch)
        with pytest.raises(B.GsError) as e:
            pipeline.backward(f, params, G, config=cfg)
        assert e.value.code == B.GS_ERR_INVALID_ARG
