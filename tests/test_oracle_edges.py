"""Boundary and special-case pins of the oracle's projection, binning and
compositing (Sec. 2.1, 2.2, Eq. 7; readings O1, O7, O9, O12): each axis of the
3-sigma box, the tile grid of an image whose size is a multiple of the tile
(or one short of it), culling exactly at the near and far planes and at a
singular Sigma', off-screen boxes on every side, the depth output, equal depths
in index order, a Gaussian exactly at the alpha skip threshold and exactly
at the alpha clamp, and the threshold margin the parity tests use to set aside
undecidable pixels.
Expected values are worked by hand or enumerated by brute force."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_02121_gb300 import workloads as wl


def _axis_cam(W, H, f, cx, cy, near=0.01, far=100.0):
    """Camera at the world origin looking down +z (R = I, t = 0)."""
    c = wl.camera_at_distance(0.0, W, H, f, near=near, far=far)
    c.R = np.eye(3)
    c.t = np.zeros(3)
    c.cx, c.cy = cx, cy
    return c


def _on_axis(sx_px, sy_px, f=80.0, d=4.0):
    """Mean on the optical axis at depth d with world scales giving Sigma' =
    diag(sx_px^2, sy_px^2) exactly (J = diag(f/d) there, R = I)."""
    return [[0.0, 0.0, d]], [[1.0, 0.0, 0.0, 0.0]], [[sx_px * d / f, sy_px * d / f, 0.01]]


def test_three_sigma_box_on_each_axis():
    # sigma'_x = 6 px, sigma'_y = 3 px at mu' = (64.5, 40.5): the box is
    # [46.5, 82.5] x [31.5, 49.5], i.e. tiles x 2..5, y 1..3.  A 2-sigma box, or
    # one with the axes swapped, gives other tiles on both axes.
    cam = _axis_cam(160, 96, 80.0, 64.5, 40.5)
    m, q, s = _on_axis(6.0, 3.0)
    p = oracle.project(cam, m, q, s, eps2d=0.0)
    np.testing.assert_allclose(p["cov2d"][0], [36.0, 0.0, 9.0], rtol=1e-12, atol=1e-12)
    assert p["valid"][0] == 1
    np.testing.assert_array_equal(p["rects"][0], [2, 1, 6, 4])
    # nearest tile boundaries: 46.5 -> 48, 82.5 -> 80, 31.5 -> 32, 49.5 -> 48
    np.testing.assert_allclose(p["rect_margin"][0], 0.5, atol=1e-9)


def test_rect_margin_is_the_distance_to_the_nearest_tile_boundary():
    # brute force over every boundary line k * 16, k = 0 .. tiles, of each box edge
    w = wl.small_case(11, 400, 70, 45)
    cam = w.views[0].camera
    sc = w.scenes[0]
    p = oracle.project(cam, sc.means, sc.quats, sc.scales)
    TX, TY = oracle.tiles(cam)
    checked = 0
    for n in range(len(p["valid"])):
        if not p["valid"][n]:
            assert math.isinf(p["rect_margin"][n])
            continue
        mx, my = p["means2d"][n]
        rx, ry = 3.0 * math.sqrt(p["cov2d"][n][0]), 3.0 * math.sqrt(p["cov2d"][n][2])
        best = min([abs(e - 16.0 * k) for e in (mx - rx, mx + rx) for k in range(TX + 1)]
                   + [abs(e - 16.0 * k) for e in (my - ry, my + ry) for k in range(TY + 1)])
        assert p["rect_margin"][n] == pytest.approx(best, abs=1e-9)
        checked += 1
    assert checked > 50


@pytest.mark.parametrize("W,H,TX,TY", [(32, 48, 2, 3), (47, 31, 3, 2), (33, 17, 3, 2)])
def test_tile_grid_rounds_up_and_clamps_the_box(W, H, TX, TY):
    # A box far larger than the image covers exactly the whole grid: ceil(W/16) x ceil(H/16).
    cam = _axis_cam(W, H, 80.0, W / 2.0, H / 2.0)
    m, q, s = _on_axis(40.0, 40.0)
    p = oracle.project(cam, m, q, s, eps2d=0.0)
    assert oracle.tiles(cam) == (TX, TY)
    np.testing.assert_array_equal(p["rects"][0], [0, 0, TX, TY])


def test_depth_is_camera_space_z():
    # t = R_cw mu + t_cw (Eq. 2) with a 90-degree turn about x: camera z = world y + 2.
    cam = _axis_cam(64, 64, 50.0, 32.0, 32.0)
    cam.R = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])
    cam.t = np.array([0.1, -0.2, 2.0])
    means = [[0.3, 3.0, 0.2], [-0.1, 1.5, -0.1], [0.0, 7.25, 0.4]]
    p = oracle.project(cam, means, [[1, 0, 0, 0]] * 3, [[0.02] * 3] * 3)
    np.testing.assert_allclose(p["depths"], [5.0, 3.5, 9.25], rtol=0, atol=1e-14)
    assert p["valid"].tolist() == [1, 1, 1]


def test_cull_exactly_at_the_near_and_far_planes():
    # O1: kept only for near < t_z < far (strictly)
    cam = _axis_cam(64, 64, 64.0, 32.0, 32.0, near=0.5, far=10.0)
    z = [0.5, 10.0, 0.5 + 1e-9, 10.0 - 1e-9]
    p = oracle.project(cam, [[0, 0, d] for d in z], [[1, 0, 0, 0]] * 4, [[0.05] * 3] * 4)
    assert p["valid"].tolist() == [0, 0, 1, 1]


def test_singular_projected_covariance_is_culled():
    # zero scales: Sigma' = 0 has det 0 (O1) unless the eps2d dilation (O11) makes it eps2d * I
    cam = _axis_cam(64, 64, 64.0, 32.0, 32.0)
    args = ([[0, 0, 3.0]], [[1, 0, 0, 0]], [[0.0, 0.0, 0.0]])
    assert oracle.project(cam, *args, eps2d=0.0)["valid"][0] == 0
    p = oracle.project(cam, *args, eps2d=0.3)
    assert p["valid"][0] == 1
    np.testing.assert_allclose(p["conics"][0], [1 / 0.3, 0.0, 1 / 0.3], rtol=1e-13)


def test_offscreen_on_each_side_is_culled_with_an_empty_rect():
    # The box misses the image to the right, left, below and above: its clamped
    # rectangle is empty on one axis, so the Gaussian is culled and its rect zeroed.
    cam = _axis_cam(40, 20, 80.0, 20.0, 10.0)
    d = 4.0
    means = [[3.0, 0, d], [-3.0, 0, d], [0, 3.0, d], [0, -3.0, d], [0, 0, d]]
    p = oracle.project(cam, means, [[1, 0, 0, 0]] * 5, [[0.02] * 3] * 5, eps2d=0.0)
    assert p["valid"].tolist() == [0, 0, 0, 0, 1]
    np.testing.assert_array_equal(p["rects"][:4], np.zeros((4, 4), np.int32))
    assert np.isinf(p["rect_margin"][:4]).all()


def _proj2d(means2d, sigmas_px, depths, W, H):
    n = len(means2d)
    TX, TY = oracle.tiles(W, H)
    return dict(means2d=np.array(means2d, float), conics=np.array([[1 / s ** 2, 0.0, 1 / s ** 2] for s in sigmas_px]),
                depths=np.array(depths, float), rects=np.array([[0, 0, TX, TY]] * n, np.int32),
                valid=np.ones(n, np.int32))


def test_equal_depths_composite_in_index_order():
    # O12: two Gaussians centred on pixel (5, 5) at one depth; 0 is red with
    # alpha 0.6, 1 is green with alpha 0.3, so index order gives (0.6, 0.3 * 0.4, 0).
    c = [5.5, 5.5]
    proj = _proj2d([c, c], [2.0, 2.0], [3.0, 3.0], 16, 16)
    out = oracle.rasterize(proj, [0.6, 0.3], [[1, 0, 0], [0, 1, 0]], 16, 16)
    np.testing.assert_allclose(out["rgb"][5, 5], [0.6, 0.12, 0.0], atol=1e-15)
    out = oracle.rasterize(proj, [0.3, 0.6], [[0, 1, 0], [1, 0, 0]], 16, 16)
    np.testing.assert_allclose(out["rgb"][5, 5], [0.42, 0.3, 0.0], atol=1e-15)
    assert oracle.pixel_trace(proj, [0.6, 0.3], [[1, 0, 0], [0, 1, 0]], 5, 5)["ids"].tolist() == [0, 1]


def test_equal_depths_bin_in_index_order():
    # brute force: every (tile, depth, index) triple of a grid with many equal depths, sorted
    rng = np.random.default_rng(8)
    P, TX, TY = 60, 4, 3
    x0, y0 = rng.integers(0, TX, P), rng.integers(0, TY, P)
    rects = np.stack([x0, y0, np.minimum(x0 + rng.integers(1, 4, P), TX),
                      np.minimum(y0 + rng.integers(1, 3, P), TY)], 1).astype(np.int32)
    depths = rng.choice(np.array([1.0, 2.5, 4.0], np.float32), P)
    valid = (rng.random(P) > 0.15).astype(np.int32)
    ids, ranges = oracle.bin_tiles(rects, depths, valid, TX, TY)
    pairs = sorted((ty * TX + tx, float(depths[n]), n) for n in range(P) if valid[n]
                   for ty in range(rects[n][1], rects[n][3]) for tx in range(rects[n][0], rects[n][2]))
    assert ids.tolist() == [n for _, _, n in pairs]
    ties = sum(1 for a, b in zip(pairs, pairs[1:]) if a[:2] == b[:2])
    assert ties > 20


def test_alpha_exactly_at_the_skip_threshold_is_composited():
    # O7: skipped only when o exp(-sigma) < 1/255; at the Gaussian's centre sigma = 0 and o = 1/255 exactly
    # (and the thresholds the oracle exports are the ones it applies)
    assert (oracle.ALPHA_MIN, oracle.ALPHA_MAX, oracle.T_MIN) == (1.0 / 255.0, 0.99, 1e-4)
    proj = _proj2d([[8.5, 8.5]], [2.0], [3.0], 16, 16)
    out = oracle.rasterize(proj, [oracle.ALPHA_MIN], [[1.0, 0.5, 0.25]], 16, 16)
    np.testing.assert_allclose(out["rgb"][8, 8], np.array([1.0, 0.5, 0.25]) / 255.0, rtol=0, atol=1e-18)
    assert out["n_contrib"][8, 8] == 1
    out = oracle.rasterize(proj, [math.nextafter(oracle.ALPHA_MIN, 0.0)], [[1.0, 0.5, 0.25]], 16, 16)
    assert out["n_contrib"][8, 8] == 0 and out["T_final"][8, 8] == 1.0


def test_threshold_margin_is_the_nearest_relative_distance_to_a_threshold():
    # margin = smallest |x - threshold| / threshold over the alpha skip (1/255),
    # the alpha clamp (0.99) and the transmittance cut-off (1e-4) tests the pixel made.
    centre = [[4.5, 4.5]]
    proj = _proj2d(centre, [2.0], [3.0], 16, 16)
    # o = 0.005 at the centre: nearest is the skip threshold, (0.005 - 1/255) * 255 = 0.275
    out = oracle.rasterize(proj, [0.005], [[1, 1, 1]], 16, 16)
    assert out["margin"][4, 4] == pytest.approx(0.275, rel=1e-12)
    # o = 0.5: nearest is the clamp, 0.49 / 0.99
    out = oracle.rasterize(proj, [0.5], [[1, 1, 1]], 16, 16)
    assert out["margin"][4, 4] == pytest.approx(0.49 / 0.99, rel=1e-12)
    # fourteen alpha = 1/2 Gaussians stacked on the pixel: T = 2^-13 after thirteen
    # (kept, 0.2207 above 1e-4), the fourteenth would leave 2^-14 < 1e-4 and is
    # not composited; nearest is the cut-off, 2^-13 / 1e-4 - 1
    proj = _proj2d(centre * 14, [2.0] * 14, np.arange(1, 15, dtype=float), 16, 16)
    out = oracle.rasterize(proj, [0.5] * 14, [[1, 1, 1]] * 14, 16, 16)
    assert out["n_contrib"][4, 4] == 13 and out["T_final"][4, 4] == 2.0 ** -13
    assert out["margin"][4, 4] == pytest.approx(2.0 ** -13 / 1e-4 - 1.0, rel=1e-12)


def test_alpha_exactly_at_the_clamp_has_no_opacity_gradient():
    # O7: alpha = min(0.99, o e^-sigma) is held at 0.99 from o e^-sigma = 0.99 up,
    # so there dalpha/do = 0; just below it dL/do = e^-sigma dL/dalpha, which for one
    # white Gaussian at the pixel centre with dL/dC = (1, 1, 1) is 3.
    W = H = 16
    proj = _proj2d([[8.5, 8.5]], [2.0], [3.0], W, H)
    G = np.zeros((W * H, 3))
    G[8 * W + 8] = 1.0
    at = oracle.rasterize_bwd(proj, [0.99], [[1, 1, 1]], W, H, G)
    assert at["opacities"][0] == 0.0
    np.testing.assert_allclose(at["colors"][0], [0.99] * 3, rtol=1e-15)
    below = oracle.rasterize_bwd(proj, [math.nextafter(0.99, 0.0)], [[1, 1, 1]], W, H, G)
    assert below["opacities"][0] == pytest.approx(3.0, rel=1e-15)


def test_compositing_invariants_over_a_dense_frame():
    # Eq. 7 with the O7 stop rule: T never falls below 1e-4 (compositing stops before it would);
    # the weights alpha_n T_n telescope to 1 - T_final; colours in [0, 1] keep every channel in
    # [0, 1 - T_final]; the last composited index is -1 exactly when nothing was composited.
    w = wl.small_case(5, 600, 48, 40, log_scale_mu=-2.2, opacity_logit_mu=1.0)
    cam, sc = w.views[0].camera, w.scenes[0]
    out = oracle.render(cam, sc)
    Tf, rgb = out["T_final"], out["rgb"]
    assert Tf.min() >= oracle.T_MIN and Tf.max() <= 1.0
    assert (Tf < 0.01).mean() > 0.1  # the frame is dense enough for the cut-off to matter
    assert (rgb >= 0).all() and (rgb <= (1.0 - Tf)[..., None] + 1e-12).all()
    assert ((out["last_id"] < 0) == (out["n_contrib"] == 0)).all()
    rng = np.random.default_rng(0)
    for py, px in zip(rng.integers(0, 40, 25), rng.integers(0, 48, 25)):
        tr = oracle.pixel_trace(out["proj"], sc.opacities, sc.colors, int(px), int(py))
        assert np.sum(tr["alpha"] * tr["T"]) == pytest.approx(1.0 - tr["T_final"], abs=1e-12)
        assert tr["T_final"] == pytest.approx(Tf[py, px], abs=1e-15)
