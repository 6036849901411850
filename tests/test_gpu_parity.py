"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (fp32 kernels against the fp64 oracle): projected means within
2e-4 px (+1e-6 relative), conics and depths within 1e-5 relative; tile lists
and sorted order bit-exact; images and final transmittance within 1e-5
max-abs; gradients within 1e-4 relative L2.  Pixels where a threshold test
(alpha 1/255, alpha 0.99, T 1e-4, tile-box edge) lies within fp32 reach of its
threshold may legitimately differ; they are excluded, counted, and must stay
rare.  dL/dC is zeroed there for the gradient comparisons.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline
from paper_2312_02121_gb300 import workloads as wl
from oracle import compare
from gpu_helpers import (gpu_projection, last_gaussian_ids, np_, rel_l2, run_gpu, uncertain_pixels, view_image)

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GRAD_TOL = 1e-4


def _workloads():
    return {
        "forward_1k_128": lambda: wl.forward_1k_128(),
        "ragged_2k_100x75": lambda: wl.small_case(5, 2000, 100, 75),
        "dense_3k_160x120": lambda: wl.small_case(6, 3000, 160, 120, log_scale_mu=-2.6, opacity_logit_mu=1.0),
        "gradcheck_64_32": lambda: wl.gradcheck_64_32(),
        "fwdbwd_100k_1024x768": lambda: wl.fwdbwd_100k_1024x768(),
    }


CASES = list(_workloads())


@pytest.fixture(scope="module", params=CASES)
def case(request):
    w = _workloads()[request.param]()
    cam, sc = w.views[0].camera, w.scenes[0]
    rng = np.random.default_rng(42)
    G = rng.standard_normal((cam.height, cam.width, 3)).astype(np.float32)
    ofwd = oracle.render(cam, sc, w.eps2d)
    frame, params, _ = run_gpu(w, deterministic=True)  # the binning tests read the inverse positions
    # uncertain pixels: end to end (oracle projection) or given the CUDA projection
    bad = uncertain_pixels(ofwd, ofwd["proj"], cam.width, cam.height, sc.opacities)
    ogp = oracle.rasterize(gpu_projection(frame), sc.opacities, sc.colors, cam.width, cam.height)
    bad_gp = ogp["margin"] < 1e-4
    Gm = np.where((bad | bad_gp)[..., None], 0.0, G).astype(np.float32)
    grads = pipeline.backward(frame, params, torch.as_tensor(Gm.reshape(-1, 3), device="cuda"))
    torch.cuda.synchronize()
    return dict(name=request.param, w=w, cam=cam, sc=sc, G=Gm, ofwd=ofwd, bad=bad, ogp=ogp, bad_gp=bad_gp,
                frame=frame, grads=grads, params=params)


def test_projection(case):
    cam, sc, w = case["cam"], case["sc"], case["w"]
    op = case["ofwd"]["proj"]
    gp = gpu_projection(case["frame"])
    sure = op["rect_margin"] > 1e-3
    assert sure.mean() > 0.99
    np.testing.assert_array_equal(gp["valid"][sure], op["valid"][sure])
    v = (op["valid"] > 0) & (gp["valid"] > 0)
    np.testing.assert_allclose(gp["means2d"][v], op["means2d"][v], rtol=1e-6, atol=2e-4)
    np.testing.assert_allclose(gp["depths"][v], op["depths"][v], rtol=1e-6)
    # per Gaussian, error relative to its largest conic entry (elongated ellipses lose a few digits)
    rel = np.abs(gp["conics"][v] - op["conics"][v]).max(axis=1) / np.abs(op["conics"][v]).max(axis=1)
    assert (rel <= 1e-5).mean() > 0.999 and rel.max() <= 1e-3
    # the factors themselves: a and d to fp32 precision whatever the elongation, k relative to 1 + |k|
    of, gf = compare.conic_factors(op["conics"][v]), gp["conic_factors"][v]
    for j in (0, 2):
        assert (np.abs(gf[:, j] - of[:, j]) / np.abs(of[:, j])).max() <= 1e-5, j
    assert (np.abs(gf[:, 1] - of[:, 1]) / (1 + np.abs(of[:, 1]))).max() <= 1e-5
    np.testing.assert_array_equal(gp["rects"][v & sure], op["rects"][v & sure])


def test_binning_bit_exact(case):
    f = case["frame"]
    gp = gpu_projection(f)
    TX, TY = oracle.tiles(case["cam"])
    ids, ranges = oracle.bin_tiles(gp["rects"], gp["depths32"], gp["valid"], TX, TY)
    K = int(np_(f.K)[0])
    assert K == len(ids) == int(np_(f.K_total)[0])
    assert not f.overflowed()
    np.testing.assert_array_equal(np_(f.isect_ids)[:K], ids)
    np.testing.assert_array_equal(np_(f.tile_ranges), ranges)
    # every projection finds its own pairs through emit_start / isect_pos
    touched = np_(f.touched)
    es, pos, sid = np_(f.emit_start), np_(f.isect_pos)[:K], np_(f.isect_ids)[:K]
    vis = np.nonzero(touched)[0]
    owner = np.repeat(vis, touched[vis])
    e = np.concatenate([es[p] + np.arange(touched[p]) for p in vis]) if len(vis) else np.zeros(0, np.int64)
    np.testing.assert_array_equal(sid[pos[e]], owner)


def test_binning_without_inverse_positions_is_the_same(case):
    # without isect_pos (the fast backward's case) the tile sort carries the owners directly
    f = case["frame"]
    v, P, T = f.views, f.views.P, f.views.T
    cap = f.K_capacity
    dev = "cuda"
    ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, T), dtype=torch.uint8, device=dev)
    ids = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    tr = torch.full((T, 2), -7, dtype=torch.int32, device=dev)
    K = torch.empty(1, dtype=torch.int32, device=dev)
    fl = torch.zeros(1, dtype=torch.int32, device=dev)
    B.gs_bin_and_sort(v, f.rects, f.depths, f.touched, cap, ws, ids, None, None, tr, K, fl)
    torch.cuda.synchronize()
    k = int(K.item())
    assert k == int(np_(f.K)[0]) and int(fl.item()) == 0
    np.testing.assert_array_equal(np_(ids)[:k], np_(f.isect_ids)[:k])
    np.testing.assert_array_equal(np_(tr), np_(f.tile_ranges))


def test_forward_given_projection(case):
    # compositing alone: the oracle composites the CUDA path's own fp32 projection
    cam, sc, f = case["cam"], case["sc"], case["frame"]
    o, bad = case["ogp"], case["bad_gp"]
    img, Tf, _ = view_image(f)
    assert bad.mean() < 0.01
    assert np.abs(img - o["rgb"])[~bad].max() <= IMG_TOL
    assert np.abs(Tf - o["T_final"])[~bad].max() <= IMG_TOL
    np.testing.assert_array_equal(last_gaussian_ids(f)[~bad], o["last_id"][~bad])


def test_forward_end_to_end(case):
    cam, f, bad = case["cam"], case["frame"], case["bad"]
    img, Tf, _ = view_image(f)
    assert bad.mean() < 0.02, bad.mean()
    o = case["ofwd"]
    assert np.abs(img - o["rgb"])[~bad].max() <= IMG_TOL
    assert np.abs(Tf - o["T_final"])[~bad].max() <= IMG_TOL


def test_backward_2d_given_projection(case):
    cam, sc, f, g = case["cam"], case["sc"], case["frame"], case["grads"]
    gp = gpu_projection(f)
    ob = compare.with_factored_conic_grad(
        oracle.rasterize_bwd(gp, sc.opacities, sc.colors, cam.width, cam.height, case["G"]), gp["conics"])
    for k in ("means2d", "conics", "opacities", "colors"):
        assert rel_l2(np_(g[k]), ob[k]) <= GRAD_TOL, k


def test_backward_3d_given_2d_gradients(case):
    # projection backward alone: the oracle maps the CUDA 2D gradients to 3D
    cam, sc, f, g = case["cam"], case["sc"], case["frame"], case["grads"]
    gp = gpu_projection(f)
    ob = oracle.project_bwd(cam, sc.means, sc.quats, sc.scales, gp["valid"], np_(g["means2d"]),
                            compare.conic_grad_from_factors(np_(g["conics"]), gp["conic_factors"]), case["w"].eps2d)
    for k in ("means", "quats", "scales"):
        assert rel_l2(np_(g[k]), ob[k]) <= GRAD_TOL, k


def test_backward_end_to_end(case):
    cam, sc, g = case["cam"], case["sc"], case["grads"]
    ob = oracle.backward(cam, sc, case["G"], case["w"].eps2d)
    for k in ("means", "quats", "scales", "opacities", "colors"):
        assert rel_l2(np_(g[k]), ob[k]) <= GRAD_TOL, k


def _project_bwd_with_viewmats(frame, params, g2, gc, eps2d):
    z = lambda *shape: torch.zeros(*shape, device="cuda")
    N = params.n
    gm, gq, gs, gv = z(max(N, 1), 3), z(max(N, 1), 4), z(max(N, 1), 3), z(frame.views.V, 4, 4)
    B.gs_project_bwd(frame.views, params.means, params.quats, params.scales, eps2d, frame.touched, g2, gc, gm, gq,
                     gs, None, gv)
    torch.cuda.synchronize()
    return dict(means=gm[:N], quats=gq[:N], scales=gs[:N], viewmats=gv)


def test_view_matrix_gradient_given_2d_gradients(case):
    # projection backward with dL/dT_cw: the oracle maps the CUDA 2D gradients (Eq. 20, Reading O14)
    cam, sc, f, g = case["cam"], case["sc"], case["frame"], case["grads"]
    P = f.views.P
    out = _project_bwd_with_viewmats(f, case["params"], g["means2d"][:P].contiguous(), g["conics"][:P].contiguous(),
                                     case["w"].eps2d)
    gp = gpu_projection(f)
    ob = oracle.project_bwd(cam, sc.means, sc.quats, sc.scales, gp["valid"], np_(g["means2d"]),
                            compare.conic_grad_from_factors(np_(g["conics"]), gp["conic_factors"]), case["w"].eps2d)
    gv = np_(out["viewmats"][0])
    assert not gv[3].any()
    assert rel_l2(gv, ob["viewmat"]) <= GRAD_TOL
    for k in ("means", "quats", "scales"):  # the kernel variant leaves the per-Gaussian outputs as they were
        assert rel_l2(np_(out[k]), np_(g[k])) <= 1e-6, k


def test_view_matrix_gradient_end_to_end_rotated_cameras():
    # three rotated cameras of uneven sizes on one scene; one batched call, per-view dL/dT_cw
    base = wl.small_case(12, 2500, 64, 64, log_scale_mu=-2.6)
    sc = base.scenes[0]
    cams = wl.sphere_cameras(np.random.default_rng(13), 3, 4.0, [(80, 60), (47, 33), (64, 64)],
                             focal_range=(60.0, 110.0))
    w = wl.Workload("rotated", [sc], [wl.View(0, c) for c in cams], None)
    rng = np.random.default_rng(14)
    Gs = []
    for c in cams:
        o = oracle.render(c, sc, w.eps2d)
        G = rng.standard_normal((c.height, c.width, 3)).astype(np.float32)
        G[uncertain_pixels(o, o["proj"], c.width, c.height, sc.opacities)] = 0
        Gs.append(G)
    frame, params, _ = run_gpu(w)
    g = pipeline.backward(frame, params, torch.as_tensor(np.concatenate([G.reshape(-1, 3) for G in Gs]),
                                                         device="cuda"), viewmats=True)
    torch.cuda.synchronize()
    for i, (c, G) in enumerate(zip(cams, Gs)):
        ob = oracle.backward(c, sc, G, w.eps2d)
        assert rel_l2(np_(g["viewmats"][i]), ob["viewmat"]) <= GRAD_TOL, i


def test_background():
    w = wl.small_case(7, 400, 48, 40)
    cam, sc = w.views[0].camera, w.scenes[0]
    bg = np.array([0.25, 0.5, 0.75], np.float32)
    G = np.random.default_rng(0).standard_normal((40, 48, 3)).astype(np.float32)
    o = oracle.render(cam, sc, w.eps2d, background=bg)
    bad = uncertain_pixels(o, o["proj"], 48, 40, sc.opacities)
    G[bad] = 0
    f, p, g = run_gpu(w, dL_drgb=G.reshape(-1, 3), background=bg)
    img, _, _ = view_image(f)
    assert np.abs(img - o["rgb"])[~bad].max() <= IMG_TOL
    ob = oracle.backward(cam, sc, G, w.eps2d, background=bg)
    for k in ("means", "quats", "scales", "opacities", "colors"):
        assert rel_l2(np_(g[k]), ob[k]) <= GRAD_TOL, k


def test_batch_of_views_equals_single_views():
    # three views of two scenes, uneven sizes, one call == one call per view (bit-exact)
    a = wl.small_case(8, 300, 40, 24)
    b = wl.small_case(9, 500, 57, 33)
    c = wl.small_case(10, 300, 64, 48)
    c.scenes = a.scenes
    w = wl.Workload("mix", [a.scenes[0], b.scenes[0]],
                    [wl.View(0, a.views[0].camera), wl.View(1, b.views[0].camera), wl.View(0, c.views[0].camera)],
                    None)
    Gall = np.random.default_rng(1).standard_normal((w.pixels, 3)).astype(np.float32)
    fb, pb, gb = run_gpu(w, dL_drgb=Gall)
    off = 0
    tot = {k: 0 for k in ("means", "quats", "scales", "opacities", "colors")}
    n0 = a.scenes[0].n
    for i, v in enumerate(w.views):
        pix = v.camera.pixels
        single = wl.Workload("one", [w.scenes[v.scene]], [wl.View(0, v.camera)], None)
        fs, ps, gs = run_gpu(single, dL_drgb=Gall[off:off + pix])
        img_b, T_b, _ = view_image(fb, i)
        img_s, T_s, _ = view_image(fs, 0)
        np.testing.assert_array_equal(img_b, img_s)
        np.testing.assert_array_equal(T_b, T_s)
        sl = slice(0, n0) if v.scene == 0 else slice(n0, n0 + b.scenes[0].n)
        for k in tot:
            exp = np.zeros_like(np_(gb[k]))
            exp[sl] = np_(gs[k])
            tot[k] = tot[k] + exp
        off += pix
    for k in tot:
        np.testing.assert_allclose(np_(gb[k]), tot[k], rtol=1e-5, atol=1e-7 * np.abs(tot[k]).max())


def test_deterministic_and_cull_invariant():
    # deterministic mode: bit-identical across runs and with the pair cull disabled;
    # atomic mode: equal to it up to fp32 summation order (1e-5 relative L2; 5e-5 for the
    # quaternion gradient, which sums terms of both signs, so reordering shows most there)
    w = wl.small_case(11, 3000, 150, 110, log_scale_mu=-2.4, opacity_logit_mu=0.8)
    G = np.random.default_rng(3).standard_normal((w.pixels, 3)).astype(np.float32)
    f1, _, g1 = run_gpu(w, dL_drgb=G, deterministic=True)
    f2, _, g2 = run_gpu(w, dL_drgb=G, deterministic=True)
    os.environ["GS_NO_CULL"] = "1"
    try:
        f3, _, g3 = run_gpu(w, dL_drgb=G, deterministic=True)
        f5, _, g5 = run_gpu(w, dL_drgb=G)
    finally:
        del os.environ["GS_NO_CULL"]
    f4, _, g4 = run_gpu(w, dL_drgb=G)
    for f in (f2, f3, f4, f5):
        np.testing.assert_array_equal(np_(f1.out_rgb), np_(f.out_rgb))
        np.testing.assert_array_equal(np_(f1.last_idx), np_(f.last_idx))
        np.testing.assert_array_equal(np_(f1.isect_ids), np_(f.isect_ids))
    for g in (g2, g3):
        for k in ("means2d", "conics", "means", "quats", "scales", "opacities", "colors"):
            np.testing.assert_array_equal(np_(g1[k]), np_(g[k]), err_msg=k)
    for g in (g4, g5):
        for k in ("means2d", "conics", "means", "quats", "scales", "opacities", "colors"):
            assert rel_l2(np_(g[k]), np_(g1[k])) <= (5e-5 if k == "quats" else 1e-5), k


def test_edge_case_no_gaussians_visible():
    w = wl.small_case(12, 50, 40, 30)
    w.scenes[0].means[:, 2] = -20.0  # all behind the camera
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    f, p, g = run_gpu(w, dL_drgb=np.ones((w.pixels, 3), np.float32), background=bg)
    assert int(np_(f.K)[0]) == 0 and int(np_(f.touched).sum()) == 0
    img, Tf, _ = view_image(f)
    np.testing.assert_array_equal(img, np.broadcast_to(bg, img.shape))
    np.testing.assert_array_equal(Tf, 1.0)
    for k in ("means", "quats", "scales", "opacities", "colors"):
        assert not np_(g[k]).any()


def test_edge_case_empty_scene():
    w = wl.small_case(13, 1, 33, 17)
    for k in ("means", "quats", "scales", "opacities", "colors"):
        setattr(w.scenes[0], k, getattr(w.scenes[0], k)[:0])
    f, p, g = run_gpu(w, dL_drgb=np.ones((w.pixels, 3), np.float32))
    img, Tf, last = view_image(f)
    assert not img.any() and (Tf == 1).all()


def test_edge_case_one_gaussian_over_every_tile():
    w = wl.small_case(14, 1, 70, 50)
    sc = w.scenes[0]
    sc.means[:] = [[0.0, 0.0, 0.0]]
    sc.scales[:] = [[2.0, 1.5, 1.0]]
    sc.opacities[:] = [0.8]
    G = np.random.default_rng(4).standard_normal((50, 70, 3)).astype(np.float32)
    cam = w.views[0].camera
    o = oracle.render(cam, sc, w.eps2d)
    assert o["proj"]["rects"][0].tolist() == [0, 0, 5, 4]
    f, p, g = run_gpu(w, dL_drgb=G)
    img, _, _ = view_image(f)
    assert np.abs(img - o["rgb"]).max() <= IMG_TOL
    ob = oracle.backward(cam, sc, G, w.eps2d)
    for k in ("means", "quats", "scales", "opacities", "colors"):
        assert rel_l2(np_(g[k]), ob[k]) <= GRAD_TOL, k


def test_capacity_overflow_is_flagged():
    w = wl.small_case(15, 500, 64, 64)
    f, _, _ = run_gpu(w, K_capacity=16)
    assert int(np_(f.K_total)[0]) > 16
    assert f.overflowed()
    f2, _, _ = run_gpu(w)
    assert not f2.overflowed()


def test_full_size_1080p_sampled_pixels():
    # 1,000,000 Gaussians at 1920x1080, in the benchmark's launch configuration;
    # the oracle composites a seeded sample of pixels from the CUDA projection.
    w = wl.fwdbwd_1m_1080p()
    cam, sc = w.views[0].camera, w.scenes[0]
    rng = np.random.default_rng(5)
    pix = np.sort(rng.choice(cam.pixels, 1500, replace=False))
    G = np.zeros((cam.pixels, 3), np.float32)
    G[pix] = rng.standard_normal((len(pix), 3))
    f, p, g = run_gpu(w, dL_drgb=G)
    assert not f.overflowed()
    gp = gpu_projection(f)
    o = oracle.rasterize(gp, sc.opacities, sc.colors, cam.width, cam.height, pixels=pix)
    img, Tf, _ = view_image(f)
    ok = o["margin"] >= 1e-4
    assert ok.mean() > 0.98
    assert np.abs(img.reshape(-1, 3)[pix] - o["rgb"])[ok].max() <= IMG_TOL
    assert np.abs(Tf.reshape(-1)[pix] - o["T_final"])[ok].max() <= IMG_TOL
    Gs = np.where(ok[:, None], G[pix], 0.0)
    G2 = np.zeros_like(G)
    G2[pix] = Gs
    f2, p2, g2 = run_gpu(w, dL_drgb=G2)
    ob = compare.with_factored_conic_grad(
        oracle.rasterize_bwd(gp, sc.opacities, sc.colors, cam.width, cam.height, Gs, pixels=pix), gp["conics"])
    for k in ("means2d", "conics", "opacities", "colors"):
        assert rel_l2(np_(g2[k]), ob[k]) <= GRAD_TOL, k
    # properties at every pixel
    assert np.isfinite(img).all() and (Tf > 0).all() and (Tf <= 1).all()


def test_non_finite_parameters_are_culled_or_skipped():
    # NaN / Inf means and scales, a zero quaternion (culled at projection, Reading O1) and a NaN
    # opacity (skipped at compositing, Reading O7) among ordinary Gaussians: the image equals the
    # oracle's and the one without those Gaussians; every gradient is finite
    w = wl.small_case(15, 400, 64, 48, log_scale_mu=-2.4)
    cam, sc = w.views[0].camera, w.scenes[0]
    bad_ids = [3, 17, 41, 77, 123]
    for k in ("means", "quats", "scales", "opacities", "colors"):
        setattr(sc, k, np.array(getattr(sc, k)))
    sc.means[3] = np.nan
    sc.scales[17] = [np.inf, 0.1, 0.1]
    sc.quats[41] = 0.0
    sc.opacities[77] = np.nan
    sc.means[123, 2] = np.inf
    G = np.random.default_rng(4).standard_normal((cam.height, cam.width, 3)).astype(np.float32)
    f, p, g = run_gpu(w, dL_drgb=G.reshape(-1, 3))
    touched = np_(f.touched)
    assert all(touched[i] == 0 for i in (3, 17, 41, 123))
    o = oracle.render(cam, sc, w.eps2d)
    bad = uncertain_pixels(o, o["proj"], cam.width, cam.height, sc.opacities)
    img, T, _ = view_image(f)
    assert np.isfinite(img).all() and np.isfinite(T).all()
    assert np.abs(img - o["rgb"])[~bad].max() <= IMG_TOL
    keep = np.setdiff1d(np.arange(sc.n), bad_ids)
    clean = wl.Workload("clean", [wl.Scene(*[np.ascontiguousarray(getattr(sc, k)[keep]) for k in
                                              ("means", "quats", "scales", "opacities", "colors")])],
                        w.views, None)
    fc, _, _ = run_gpu(clean)
    img_c, T_c, _ = view_image(fc)
    assert np.abs(img - img_c).max() <= 1e-6
    for k in ("means2d", "conics", "means", "quats", "scales", "opacities", "colors"):
        assert np.isfinite(np_(g[k])[keep if g[k].shape[0] == sc.n else slice(None)]).all(), k


def test_backward_with_forward_warp_hits_is_identical():
    # the backward may take the forward's per-pair warp-box cull (GsRasterConfig.warp_hits) instead of
    # repeating it: same pairs, same sums (deterministic mode: bit for bit), for both tile walks
    w = wl.small_case(16, 4000, 200, 150, log_scale_mu=-2.4, opacity_logit_mu=0.8)
    sc = w.scenes[0]
    params = pipeline.Params.from_scene(sc, "cuda")
    views = B.Views([w.views[0].camera], [(0, sc.n)], device="cuda")
    G = torch.tensor(np.random.default_rng(5).standard_normal((views.pixels, 3)).astype(np.float32), device="cuda")
    for persistent in (False, True):
        plain = B.RasterConfig(persistent, 2)
        f1 = pipeline.forward(views, params, w.eps2d, config=plain, deterministic=True)
        g1 = pipeline.backward(f1, params, G, deterministic=True, config=plain)
        K = int(f1.K.item())
        # words the forward does not write (chunks past a warp's last pixel) must never be read:
        # start from garbage
        hits = torch.randint(-2**31, 2**31 - 1, (f1.K_capacity,), dtype=torch.int32,
                             generator=torch.Generator().manual_seed(9)).cuda()
        with_hits = B.RasterConfig(persistent, 2, warp_hits=hits)
        f2 = pipeline.forward(views, params, w.eps2d, config=with_hits, deterministic=True)
        g2 = pipeline.backward(f2, params, G, deterministic=True, config=with_hits)
        torch.cuda.synchronize()
        assert int(hits[:K].count_nonzero()) > 0
        tile_len = (f1.tile_ranges[:, 1] - f1.tile_ranges[:, 0]).cpu()
        assert bool(((tile_len % 32 > 0) & (tile_len % 32 < 8)).any())  # chunks too short for 8 words
        np.testing.assert_array_equal(np_(f1.out_rgb), np_(f2.out_rgb))
        for k in ("means2d", "conics", "opacities", "colors", "means", "quats", "scales"):
            np.testing.assert_array_equal(np_(g1[k]), np_(g2[k]), err_msg=k)
