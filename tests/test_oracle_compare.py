"""The fp32-vs-fp64 comparison helpers (oracle.compare): the uncertain-pixel
mask against a plain whole-image evaluation of its definition, and its
pixel-subset form against the whole-image mask at those pixels (CPU only)."""
import numpy as np

import oracle
from oracle import compare
from paper_2312_02121_gb300 import workloads as wl


def _brute_force_mask(margin, proj, W, H, op, margin_rel, rect_px):
    # the definition, over every pixel of the image for every Gaussian near a tile line
    bad = margin < margin_rel
    TX, TY = oracle.tiles(W, H)
    ys, xs = np.mgrid[0:H, 0:W]
    for n in range(len(proj["means2d"])):
        if not (proj["valid"][n] and proj["rect_margin"][n] < rect_px):
            continue
        x0, y0, x1, y1 = proj["rects"][n]
        m, cov, con = proj["means2d"][n], proj["cov2d"][n], proj["conics"][n]
        rx, ry = 3 * np.sqrt(cov[0]), 3 * np.sqrt(cov[2])
        for axis, side, edge in ((0, 0, m[0] - rx), (0, 1, m[0] + rx), (1, 0, m[1] - ry), (1, 1, m[1] + ry)):
            k = int(np.floor(edge / 16 + 0.5))
            if abs(edge - 16 * k) >= rect_px:
                continue
            t = k - 1 if side == 0 else k
            if axis == 0:
                if not 0 <= t < TX:
                    continue
                sel = (xs // 16 == t) & (ys // 16 >= max(y0 - 1, 0)) & (ys // 16 < y1 + 1)
            else:
                if not 0 <= t < TY:
                    continue
                sel = (ys // 16 == t) & (xs // 16 >= max(x0 - 1, 0)) & (xs // 16 < x1 + 1)
            dx, dy = m[0] - (xs + 0.5), m[1] - (ys + 0.5)
            sig = 0.5 * (con[0] * dx * dx + 2 * con[1] * dx * dy + con[2] * dy * dy)
            bad |= sel & (op[n] * np.exp(-sig) >= (1 / 255) * (1 - 1e-3))
    return bad


def test_uncertain_pixels_follow_their_definition_whole_image_and_subset():
    w = wl.small_case(41, 600, 101, 67, log_scale_mu=-2.5)
    cam, sc = w.views[0].camera, w.scenes[0]
    o = oracle.render(cam, sc, w.eps2d)
    # wide margins so that many Gaussians count as near a tile line and every branch runs
    for margin_rel, rect_px in ((1e-4, 1e-3), (2e-2, 2.5), (5e-2, 6.0)):
        ref = _brute_force_mask(o["margin"], o["proj"], cam.width, cam.height, sc.opacities, margin_rel, rect_px)
        got = compare.uncertain_pixels(o["margin"], o["proj"], cam.width, cam.height, sc.opacities,
                                       margin_rel=margin_rel, rect_margin_px=rect_px)
        np.testing.assert_array_equal(got, ref)
        pix = np.sort(np.random.default_rng(3).choice(cam.pixels, 700, replace=False))
        sub = compare.uncertain_pixels(o["margin"].reshape(-1)[pix], o["proj"], cam.width, cam.height,
                                       sc.opacities, pixels=pix, margin_rel=margin_rel, rect_margin_px=rect_px)
        np.testing.assert_array_equal(sub, ref.reshape(-1)[pix])
    assert ref.any() and not ref.all()


def test_rel_l2():
    b = np.array([3.0, 4.0])
    assert compare.rel_l2(b, b) == 0.0
    assert compare.rel_l2(b + [0.0, 0.5], b) == 0.1
    assert compare.rel_l2(np.zeros(2), np.zeros(2)) == 0.0
