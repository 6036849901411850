"""Pins of the oracle's binning and compositing (Sec. 2.2, Eq. 7) and of the
reverse recurrences of Sec. 3.1: hand-derived golden values, closed forms,
threshold special cases and a brute-force per-pixel evaluation."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2312_02121_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _proj2d(means2d, sigmas_px, depths, W, H, rects=None):
    """2D Gaussians given directly in pixel space (isotropic, sigma in px)."""
    n = len(means2d)
    TX, TY = oracle.tiles(W, H)
    conics = np.array([[1 / s ** 2, 0.0, 1 / s ** 2] for s in sigmas_px])
    if rects is None:
        rects = [[0, 0, TX, TY]] * n
    return dict(means2d=np.array(means2d, float), conics=conics, depths=np.array(depths, float),
                rects=np.array(rects, np.int32), valid=np.ones(n, np.int32))


def test_two_gaussians_golden():
    g = json.load(open(os.path.join(GOLDEN, "two_gaussians.json")))
    px, py = g["pixel"]
    m2 = [x["mean2d"] for x in g["gaussians"]]
    sg = [x["sigma_px"] for x in g["gaussians"]]
    op = [x["opacity"] for x in g["gaussians"]]
    col = [x["color"] for x in g["gaussians"]]
    for case in g["cases"]:
        proj = _proj2d(m2, sg, case["depths"], g["width"], g["height"])
        out = oracle.rasterize(proj, op, col, g["width"], g["height"])
        np.testing.assert_allclose(out["rgb"][py, px], case["rgb"], atol=1e-15)
        np.testing.assert_allclose(out["T_final"][py, px], case["T_final"], atol=1e-15)
        assert out["n_contrib"][py, px] == 2


def test_single_gaussian_falloff_is_textbook_gaussian():
    # One isotropic Gaussian (sigma' = 2.5 px): at offset Delta the pixel is c o exp(-|Delta|^2 / (2 sigma'^2)).
    W = H = 32
    proj = _proj2d([[16.5, 10.5]], [2.5], [1.0], W, H)
    o, c = 0.7, np.array([0.3, 0.6, 0.9])
    out = oracle.rasterize(proj, [o], [c], W, H)
    for (px, py) in [(16, 10), (18, 10), (16, 13), (14, 12), (20, 8)]:
        d2 = (16.5 - (px + 0.5)) ** 2 + (10.5 - (py + 0.5)) ** 2
        a = o * math.exp(-d2 / (2 * 2.5 ** 2))
        if a < 1 / 255:
            continue
        np.testing.assert_allclose(out["rgb"][py, px], c * a, rtol=1e-14)
        np.testing.assert_allclose(out["T_final"][py, px], 1 - a, rtol=1e-14)


def test_anisotropic_conic_quadratic_form():
    # sigma = 1/2 Delta^T Y Delta with a full conic, Delta = mu' - centre (O6: sign is immaterial here).
    Y = np.array([[0.3, -0.12], [-0.12, 0.5]])
    proj = dict(means2d=np.array([[7.25, 9.75]]), conics=np.array([[Y[0, 0], Y[0, 1], Y[1, 1]]]),
                depths=np.array([1.0]), rects=np.array([[0, 0, 1, 1]], np.int32), valid=np.array([1], np.int32))
    out = oracle.rasterize(proj, [0.9], [[1, 1, 1]], 16, 16)
    for (px, py) in [(7, 9), (5, 11), (9, 8)]:
        d = np.array([7.25 - px - 0.5, 9.75 - py - 0.5])
        np.testing.assert_allclose(out["rgb"][py, px, 0], 0.9 * math.exp(-0.5 * d @ Y @ d), rtol=1e-14)


def test_alpha_clamp_and_skip():
    W = H = 16
    # o = 1 at the centre -> alpha clamped to 0.99 (reading O7)
    out = oracle.rasterize(_proj2d([[8.5, 8.5]], [2.0], [1.0], W, H), [1.0], [[1, 1, 1]], W, H)
    np.testing.assert_allclose(out["rgb"][8, 8], [0.99] * 3, rtol=1e-15)
    np.testing.assert_allclose(out["T_final"][8, 8], 0.01, rtol=1e-12)
    # o below 1/255 -> skipped, nothing composited
    out = oracle.rasterize(_proj2d([[8.5, 8.5]], [2.0], [1.0], W, H), [0.003], [[1, 1, 1]], W, H)
    assert out["n_contrib"][8, 8] == 0 and out["T_final"][8, 8] == 1.0 and out["last_id"][8, 8] == -1


def test_transmittance_cutoff_stops_before_the_gaussian():
    # Five stacked Gaussians with alpha = 0.95: T goes 1, .05, .0025, 1.25e-4, and the fourth
    # would bring it to 6.25e-6 < 1e-4, so only three are composited (reading O7).
    W = H = 16
    n = 5
    proj = _proj2d([[8.5, 8.5]] * n, [3.0] * n, [1.0, 2.0, 3.0, 4.0, 5.0], W, H)
    col = np.eye(3)[[0, 1, 2, 0, 1]]
    out = oracle.rasterize(proj, [0.95] * n, col, W, H)
    assert out["n_contrib"][8, 8] == 3
    assert out["last_id"][8, 8] == 2
    np.testing.assert_allclose(out["rgb"][8, 8], [0.95, 0.95 * 0.05, 0.95 * 0.0025], rtol=1e-14)
    np.testing.assert_allclose(out["T_final"][8, 8], 0.05 ** 3, rtol=1e-12)


def test_background_adds_final_transmittance():
    W = H = 16
    proj = _proj2d([[8.5, 8.5]], [2.0], [1.0], W, H)
    bg = np.array([0.2, 0.1, 0.7])
    out = oracle.rasterize(proj, [0.6], [[1, 0, 0]], W, H, background=bg)
    np.testing.assert_allclose(out["rgb"][8, 8], [0.6, 0, 0] + 0.4 * bg, rtol=1e-14)
    # pixel (0, 0) is 8 sigma' away on each axis: alpha < 1/255, only the background shows
    np.testing.assert_allclose(out["rgb"][0, 0], bg, rtol=1e-15)


def test_tile_membership_decides_inclusion():
    # Reading O9: a Gaussian contributes only inside the tiles of its rectangle, even where alpha >= 1/255.
    W, H = 32, 16
    proj = _proj2d([[15.5, 8.5]], [4.0], [1.0], W, H, rects=[[0, 0, 1, 1]])
    out = oracle.rasterize(proj, [0.9], [[1, 1, 1]], W, H)
    assert out["n_contrib"][8, 15] == 1  # tile 0
    assert out["n_contrib"][8, 16] == 0  # tile 1: alpha would be 0.9 exp(-1/32) but the tile is not in the rect


def _brute_force(proj, opac, col, W, H):
    """Per-pixel evaluation written independently: the Gaussians of the pixel's tile
    sorted with Python's sort, alpha per Gaussian, T_n as an explicit product."""
    m2, con, dep, rects, valid = proj["means2d"], proj["conics"], proj["depths"], proj["rects"], proj["valid"]
    img = np.zeros((H, W, 3))
    Tf = np.ones((H, W))
    for py in range(H):
        for px in range(W):
            tx, ty = px // 16, py // 16
            cand = sorted((dep[n], n) for n in range(len(dep))
                          if valid[n] and rects[n][0] <= tx < rects[n][2] and rects[n][1] <= ty < rects[n][3])
            kept = []  # composited (n, alpha)
            for _, n in cand:
                d = m2[n] - [px + 0.5, py + 0.5]
                Y = np.array([[con[n][0], con[n][1]], [con[n][1], con[n][2]]])
                s = 0.5 * d @ Y @ d
                if s < 0:
                    continue
                a = min(0.99, opac[n] * math.exp(-s))
                if a < 1 / 255:
                    continue
                T_before = math.prod(1 - b for _, b in kept)
                if T_before * (1 - a) < 1e-4:
                    break
                kept.append((n, a))
            for j, (n, a) in enumerate(kept):
                img[py, px] += col[n] * a * math.prod(1 - b for _, b in kept[:j])
            Tf[py, px] = math.prod(1 - b for _, b in kept)
    return img, Tf


@pytest.mark.parametrize("seed,W,H", [(0, 40, 24), (1, 33, 17)])
def test_compositing_matches_brute_force(seed, W, H):
    w = wl.small_case(seed, 60, W, H, log_scale_mu=-2.2, opacity_logit_mu=1.0)
    cam, sc = w.views[0].camera, w.scenes[0]
    out = oracle.render(cam, sc)
    img, Tf = _brute_force(out["proj"], sc.opacities.astype(float), sc.colors.astype(float), W, H)
    assert out["n_contrib"].max() >= 3  # the case really composites several layers
    np.testing.assert_allclose(out["rgb"], img, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["T_final"], Tf, rtol=1e-12, atol=1e-14)


def test_pixel_subset_equals_full_image():
    w = wl.small_case(3, 80, 50, 30)
    cam, sc = w.views[0].camera, w.scenes[0]
    full = oracle.render(cam, sc)
    rng = np.random.default_rng(0)
    pix = rng.choice(50 * 30, 97, replace=False)
    sub = oracle.render(cam, sc, pixels=pix)
    np.testing.assert_array_equal(sub["rgb"], full["rgb"].reshape(-1, 3)[pix])
    np.testing.assert_array_equal(sub["last_id"], full["last_id"].reshape(-1)[pix])


def test_backward_on_a_pixel_subset_equals_the_masked_full_backward():
    # The gradients are sums over pixels (Sec. 3.1), so those of a pixel subset are the
    # full image's with dL/dC zero outside the subset.
    w = wl.small_case(3, 80, 50, 30)
    cam, sc = w.views[0].camera, w.scenes[0]
    rng = np.random.default_rng(1)
    pix = rng.choice(50 * 30, 97, replace=False)
    G = rng.standard_normal((97, 3))
    Gfull = np.zeros((50 * 30, 3))
    Gfull[pix] = G
    sub = oracle.backward(cam, sc, G, pixels=pix)
    full = oracle.backward(cam, sc, Gfull)
    assert np.abs(full["opacities"]).max() > 0
    for k in ("means", "quats", "scales", "opacities", "colors", "means2d", "conics", "viewmat"):
        np.testing.assert_allclose(sub[k], full[k], rtol=1e-12, atol=1e-15, err_msg=k)


def test_reverse_recurrences_rebuild_forward_quantities():
    # Sec. 3.1: starting from the saved final transmittance, T_{n-1} = T_n / (1 - alpha_{n-1})
    # recovers the running products, and S_{n-1} = c_n alpha_n T_n + S_n the suffix sums.
    w = wl.small_case(4, 150, 32, 32, log_scale_mu=-2.0, opacity_logit_mu=0.5)
    cam, sc = w.views[0].camera, w.scenes[0]
    proj = oracle.project(cam, sc.means, sc.quats, sc.scales)
    col = sc.colors.astype(float)
    checked = 0
    for (px, py) in [(16, 16), (10, 20), (25, 5), (3, 28)]:
        tr = oracle.pixel_trace(proj, sc.opacities, col, px, py)
        c = len(tr["ids"])
        if c < 2:
            continue
        checked += 1
        T = tr["T_final"]  # transmittance after the last composited Gaussian
        S = np.zeros(3)
        for j in range(c - 1, -1, -1):
            T = T / (1 - tr["alpha"][j])  # transmittance before Gaussian j
            np.testing.assert_allclose(T, tr["T"][j], rtol=1e-12)
            explicit = sum(col[tr["ids"][m]] * tr["alpha"][m] * tr["T"][m] for m in range(j + 1, c))
            np.testing.assert_allclose(S, explicit, rtol=1e-12, atol=1e-15)
            S = S + col[tr["ids"][j]] * tr["alpha"][j] * T
    assert checked >= 2


def test_binning_golden():
    g = json.load(open(os.path.join(GOLDEN, "bin_small.json")))
    ids, ranges = oracle.bin_tiles(g["rects"], np.array(g["depths"], np.float32), g["valid"], g["TX"], g["TY"])
    for t, expect in g["tile_lists"].items():
        s, e = ranges[int(t)]
        assert ids[s:e].tolist() == expect, t


def test_binning_matches_python_enumeration():
    w = wl.small_case(5, 300, 70, 45)
    cam = w.views[0].camera
    p = oracle.project(cam, w.scenes[0].means, w.scenes[0].quats, w.scenes[0].scales)
    TX, TY = oracle.tiles(cam)
    dep32 = p["depths"].astype(np.float32)
    ids, ranges = oracle.bin_tiles(p["rects"], dep32, p["valid"], TX, TY)
    pairs = sorted((ty * TX + tx, float(dep32[n]), n) for n in range(len(dep32)) if p["valid"][n]
                   for ty in range(p["rects"][n][1], p["rects"][n][3]) for tx in range(p["rects"][n][0], p["rects"][n][2]))
    assert ids.tolist() == [n for _, _, n in pairs]
    for t in range(TX * TY):
        s, e = ranges[t]
        assert all(pairs[i][0] == t for i in range(s, e))


# -- any channel count (Sec. 3.1 derives every term per channel) --------------

def _multichannel_case(C, seed=3):
    w = wl.small_case(seed, 300, 48, 40, log_scale_mu=-2.5)
    cam, sc = w.views[0].camera, w.scenes[0]
    proj = oracle.project(cam, sc.means, sc.quats, sc.scales, w.eps2d)
    col = np.random.default_rng(seed).uniform(size=(sc.n, C))
    return cam, sc, proj, col


def test_channels_are_composited_independently():
    cam, sc, proj, col = _multichannel_case(5)
    W, H = cam.width, cam.height
    bg = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    full = oracle.rasterize(proj, sc.opacities, col, W, H, background=bg)
    a = oracle.rasterize(proj, sc.opacities, col[:, :3], W, H, background=bg[:3])
    b = oracle.rasterize(proj, sc.opacities, col[:, 3:], W, H, background=bg[3:])
    assert full["rgb"].shape == (H, W, 5)
    np.testing.assert_array_equal(full["rgb"], np.concatenate([a["rgb"], b["rgb"]], axis=-1))
    np.testing.assert_array_equal(full["T_final"], a["T_final"])
    np.testing.assert_array_equal(full["last_id"], b["last_id"])


def test_single_unit_channel_is_the_alpha_mask():
    cam, sc, proj, _ = _multichannel_case(1)
    out = oracle.rasterize(proj, sc.opacities, np.ones((sc.n, 1)), cam.width, cam.height)
    np.testing.assert_allclose(out["rgb"][..., 0], 1.0 - out["T_final"], atol=1e-15)


def test_multichannel_gradients_are_linear_in_the_channels():
    cam, sc, proj, col = _multichannel_case(5, seed=4)
    W, H = cam.width, cam.height
    G = np.random.default_rng(9).standard_normal((H * W, 5))
    bg = np.array([0.3, 0.1, 0.7, 0.2, 0.9])
    full = oracle.rasterize_bwd(proj, sc.opacities, col, W, H, G, background=bg)
    parts = [oracle.rasterize_bwd(proj, sc.opacities, col[:, s], W, H, G[:, s], background=bg[s])
             for s in (slice(0, 2), slice(2, 5))]
    for k in ("means2d", "conics", "opacities"):
        np.testing.assert_allclose(full[k], parts[0][k] + parts[1][k], rtol=1e-12, atol=1e-15)
    # (threads sum their tiles in a scheduling-dependent order: equal to rounding, not bit for bit)
    np.testing.assert_allclose(full["colors"], np.concatenate([parts[0]["colors"], parts[1]["colors"]], 1),
                               rtol=1e-12, atol=1e-15)


def test_multichannel_gradients_match_finite_differences():
    cam, sc, proj, col = _multichannel_case(2, seed=5)
    W, H = cam.width, cam.height
    G = np.random.default_rng(10).standard_normal((H * W, 2))
    g = oracle.rasterize_bwd(proj, sc.opacities, col, W, H, G)
    out = oracle.rasterize(proj, sc.opacities, col, W, H)
    assert out["margin"].min() > 1e-6
    hit = np.nonzero(g["opacities"])[0][:4]
    h = 1e-7
    for n in hit:
        for j in range(2):
            cp, cm = col.copy(), col.copy()
            cp[n, j] += h
            cm[n, j] -= h
            fd = (np.sum(G * oracle.rasterize(proj, sc.opacities, cp, W, H)["rgb"].reshape(-1, 2)) -
                  np.sum(G * oracle.rasterize(proj, sc.opacities, cm, W, H)["rgb"].reshape(-1, 2))) / (2 * h)
            assert g["colors"][n, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        op_p, op_m = np.array(sc.opacities, np.float64), np.array(sc.opacities, np.float64)
        op_p[n] += h
        op_m[n] -= h
        fd = (np.sum(G * oracle.rasterize(proj, op_p, col, W, H)["rgb"].reshape(-1, 2)) -
              np.sum(G * oracle.rasterize(proj, op_m, col, W, H)["rgb"].reshape(-1, 2))) / (2 * h)
        assert g["opacities"][n] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_non_finite_opacity_is_skipped():
    # Reading O7: a Gaussian is composited only if o exp(-sigma) >= 1/255, a test NaN fails; the
    # clamp to 0.99 must not turn a NaN opacity into an opaque Gaussian
    w = wl.small_case(14, 60, 40, 32, log_scale_mu=-2.0)
    cam, sc = w.views[0].camera, w.scenes[0]
    proj = oracle.project(cam, sc.means, sc.quats, sc.scales, w.eps2d)
    op = np.array(sc.opacities, np.float64)
    hit = int(np.argmax(proj["valid"]))
    op_nan = op.copy()
    op_nan[hit] = np.nan
    op_zero = op.copy()
    op_zero[hit] = 0.0
    a = oracle.rasterize(proj, op_nan, sc.colors, cam.width, cam.height)
    b = oracle.rasterize(proj, op_zero, sc.colors, cam.width, cam.height)
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    np.testing.assert_array_equal(a["T_final"], b["T_final"])
    G = np.random.default_rng(2).standard_normal((cam.height, cam.width, 3))
    ga = oracle.rasterize_bwd(proj, op_nan, sc.colors, cam.width, cam.height, G)
    assert np.isfinite(ga["means2d"]).all() and ga["opacities"][hit] == 0.0
