"""The fp32-vs-fp64 comparison helpers (oracle.compare): the uncertain-pixel
mask against a plain whole-image evaluation of its definition, and its
pixel-subset form against the whole-image mask at those pixels (CPU only)."""
import numpy as np
import pytest

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


def _proj_at_pixel_centre(depths, n):
    # n Gaussians centred on pixel (4, 4) of a 16x16 image, unit conics, listed in one tile
    return dict(means2d=np.tile([4.5, 4.5], (n, 1)), conics=np.tile([1.0, 0.0, 1.0], (n, 1)),
                depths=np.asarray(depths, np.float64), rects=np.tile([0, 0, 1, 1], (n, 1)).astype(np.int32),
                valid=np.ones(n, np.int32))


def test_depth_gap_is_the_closest_pair_of_consecutive_gaussians_that_pass_the_alpha_test():
    # depths 2.0, 2.0000001 (too transparent to pass the alpha test), 2.5, 2.6, 2.6000026:
    # the consecutive takers are (2.0, 2.5), (2.5, 2.6), (2.6, 2.6000026) -> the last gap, 1e-6 relative
    d = [2.0, 2.0000001, 2.5, 2.6, 2.6000026]
    op = np.array([0.3, 0.002, 0.3, 0.3, 0.3])
    out = oracle.rasterize(_proj_at_pixel_centre(d, 5), op, np.full((5, 3), 0.5), 16, 16, pixels=np.array([4 * 16 + 4]))
    assert out["depth_gap"][0] == pytest.approx(2.6e-6 / 2.6, rel=1e-6)
    assert out["n_contrib"][0] == 4


def test_depth_gap_stops_at_the_gaussian_that_ends_the_pixel():
    # opacities 0.99 x 3 then a close pair: the third Gaussian takes T below 1e-4 and stops the pixel,
    # so the pair after it (depth gap 1e-9) is never reached; the gaps met are 0.1 and 0.05 (relative)
    d = [1.0, 1.1, 1.155, 2.0, 2.000000002]
    op = np.array([0.99, 0.99, 0.99, 0.5, 0.5])
    out = oracle.rasterize(_proj_at_pixel_centre(d, 5), op, np.full((5, 3), 0.5), 16, 16, pixels=np.array([4 * 16 + 4]))
    assert out["n_contrib"][0] == 2
    assert out["depth_gap"][0] == pytest.approx(0.055 / 1.1, rel=1e-9)
    # fewer than two takers: no gap
    one = oracle.rasterize(_proj_at_pixel_centre([3.0], 1), np.array([0.5]), np.full((1, 3), 0.5), 16, 16,
                           pixels=np.array([4 * 16 + 4]))
    assert np.isinf(one["depth_gap"][0])


def test_uncertain_pixels_include_close_depths():
    d = [2.0, 2.000001, 3.0]
    proj = _proj_at_pixel_centre(d, 3)
    out = oracle.rasterize(proj, np.array([0.3, 0.3, 0.3]), np.full((3, 3), 0.5), 16, 16)
    bad_without = compare.uncertain_pixels(out["margin"], proj, 16, 16)
    bad_with = compare.uncertain_pixels(out["margin"], proj, 16, 16, depth_gap=out["depth_gap"])
    assert not bad_without[4, 4] and bad_with[4, 4]
    assert (bad_with == (bad_without | (out["depth_gap"] < 1e-6))).all()


def test_conic_forms_and_their_gradients_convert_both_ways():
    rng = np.random.default_rng(9)
    # random SPD conics, some thin (condition 1e5)
    n = 200
    th = rng.uniform(0, np.pi, n)
    l1, l2 = np.exp(rng.uniform(-3, 2, n)), np.exp(rng.uniform(-3, 2, n))
    l2[:20] = l1[:20] * 1e-5
    c, s_ = np.cos(th), np.sin(th)
    Y = np.stack([l1 * c * c + l2 * s_ * s_, (l1 - l2) * c * s_, l1 * s_ * s_ + l2 * c * c], 1)
    f = compare.conic_factors(Y)
    np.testing.assert_allclose(compare.conic_from_factors(f), Y, rtol=1e-9, atol=1e-12 * np.abs(Y).max())
    # sigma of both forms agrees at random offsets
    dx, dy = rng.standard_normal(n), rng.standard_normal(n)
    sig_p = 0.5 * (Y[:, 0] * dx * dx + 2 * Y[:, 1] * dx * dy + Y[:, 2] * dy * dy)
    sig_f = 0.5 * (f[:, 0] * (dx + f[:, 1] * dy) ** 2 + f[:, 2] * dy * dy)
    np.testing.assert_allclose(sig_f, sig_p, rtol=1e-8, atol=1e-12)
    # gradients: against finite differences of L = <G, sigma-sums> in each parameterisation
    gP = rng.standard_normal((n, 3))
    gF = compare.conic_grad_to_factors(gP, Y)
    np.testing.assert_allclose(compare.conic_grad_from_factors(gF, f), gP, rtol=1e-7, atol=1e-9)
    h = 1e-7
    for j in range(3):
        fp, fm = f.copy(), f.copy()
        fp[:, j] += h * np.maximum(np.abs(f[:, j]), 1e-3)
        fm[:, j] -= h * np.maximum(np.abs(f[:, j]), 1e-3)
        Lp = (gP * compare.conic_from_factors(fp)).sum(1)
        Lm = (gP * compare.conic_from_factors(fm)).sum(1)
        fd = (Lp - Lm) / (2 * h * np.maximum(np.abs(f[:, j]), 1e-3))
        np.testing.assert_allclose(gF[:, j], fd, rtol=1e-5, atol=1e-6 * np.abs(gF).max())
    # culled rows (all zero) give zero factors and finite gradients
    z = compare.conic_factors(np.zeros((2, 3)))
    assert not z.any() and np.isfinite(compare.conic_grad_from_factors(np.ones((2, 3)), z)).all()
