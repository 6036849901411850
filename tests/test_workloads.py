"""The seeded synthetic inputs follow their stated recipe: the same seed gives
the same arrays, and the shapes, value ranges, distributions and camera rigs
are the ones each named workload states (Gaussians from the stated laws,
look-at cameras on the stated sphere, the stated resolutions and totals)."""
import math

import numpy as np
import pytest

from paper_2312_02121_gb300 import workloads as wl


def _check_scene(sc, n):
    for k, shape in (("means", (n, 3)), ("quats", (n, 4)), ("scales", (n, 3)), ("opacities", (n,)),
                     ("colors", (n, 3))):
        a = getattr(sc, k)
        assert a.shape == shape and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"], k
    np.testing.assert_allclose(np.linalg.norm(sc.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert (sc.scales > 0).all() and ((sc.opacities > 0) & (sc.opacities < 1)).all()
    assert ((sc.colors >= 0) & (sc.colors <= 1)).all()


def _logit(o):
    o = o.astype(np.float64)
    return np.log(o / (1 - o))


def test_same_seed_same_inputs_and_other_seed_other_inputs():
    a, b, c = wl.small_case(7, 500, 64, 48), wl.small_case(7, 500, 64, 48), wl.small_case(8, 500, 64, 48)
    for k in ("means", "quats", "scales", "opacities", "colors"):
        np.testing.assert_array_equal(getattr(a.scenes[0], k), getattr(b.scenes[0], k))
        assert not np.array_equal(getattr(a.scenes[0], k), getattr(c.scenes[0], k))
    np.testing.assert_array_equal(a.targets[0], b.targets[0])


def test_benchmark_frame_follows_its_recipe():
    # 1M Gaussians from a 64-component mixture (centres U[-5,5]^3, std 0.5), log s ~ N(-4.5, 1),
    # opacity logit ~ N(-1, 2), colours U[0,1]; a 1920x1080 camera, f = 1100, at distance 12
    w = wl.fwdbwd_1m_1080p()
    sc, cam = w.scenes[0], w.views[0].camera
    _check_scene(sc, 1_000_000)
    ls = np.log(sc.scales.astype(np.float64))
    assert abs(ls.mean() + 4.5) < 0.01 and abs(ls.std() - 1.0) < 0.01
    lo = _logit(sc.opacities)
    assert abs(lo.mean() + 1.0) < 0.02 and abs(lo.std() - 2.0) < 0.02
    assert abs(sc.colors.mean() - 0.5) < 0.01
    assert np.abs(sc.means).max() < 5.0 + 0.5 * 6  # centres in the cube, six sigma of spread
    assert (cam.width, cam.height, cam.fx, cam.fy) == (1920, 1080, 1100.0, 1100.0)
    np.testing.assert_array_equal(cam.t, [0, 0, 12.0])
    np.testing.assert_array_equal(cam.R, np.eye(3))
    assert w.targets[0].shape == (1080, 1920, 3)


def test_multi_view_workload_follows_its_recipe():
    # 64 look-at cameras on a radius-10 sphere, away from the up axis, resolutions from the stated
    # set, f ~ U[300, 1200]; 30.7 Mpixel in all
    w = wl.batch_views_500k_64()  # the cameras are drawn after the scene, from the same generator
    assert len(w.views) == 64 and len(w.scenes) == 1
    pix = 0
    for v in w.views:
        c = v.camera
        R, t = c.R.astype(np.float64), c.t.astype(np.float64)
        centre = -R.T @ t
        assert abs(np.linalg.norm(centre) - 10.0) < 1e-4
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
        np.testing.assert_allclose(R[2], -centre / np.linalg.norm(centre), atol=1e-6)  # looks at the origin
        assert abs(centre[1] / 10.0) <= 0.98 + 1e-6
        assert (c.width, c.height) in wl.BATCH_RESOLUTIONS and 300.0 <= c.fx <= 1200.0
        pix += c.width * c.height
    assert round(pix / 1e6, 1) == 30.7


def test_multi_scene_workload_follows_its_recipe():
    # 16 scenes with N log-uniform in [1e4, 2e6] (5.40 M in all), 4 cameras each at 960x540, f = 800,
    # radius 5: 33.2 Mpixel
    w = wl.batch_scenes_16x4()
    ns = [s.n for s in w.scenes]
    assert len(ns) == 16 and all(10_000 <= n <= 2_000_000 for n in ns)
    assert round(sum(ns) / 1e6, 2) == 5.40
    assert len(w.views) == 64 and [v.scene for v in w.views] == [s for s in range(16) for _ in range(4)]
    for v in w.views:
        c = v.camera
        assert (c.width, c.height, c.fx) == (960, 540, 800.0)
        assert abs(np.linalg.norm(c.R.astype(np.float64).T @ c.t.astype(np.float64)) - 5.0) < 1e-4
    assert round(sum(v.camera.width * v.camera.height for v in w.views) / 1e6, 1) == 33.2
    _check_scene(w.scenes[0], ns[0])


def test_gradcheck_and_small_cases():
    w = wl.gradcheck_64_32()
    c = w.views[0].camera
    assert w.scenes[0].n == 64 and (c.width, c.height) == (32, 32) and c.fx == pytest.approx(900.0 * 32 / 1024)
    ls = np.log(w.scenes[0].scales.astype(np.float64))
    assert abs(ls.mean() - (-4.0 + math.log(32.0))) < 0.3  # the 1024x768 law shifted by ln 32
    w = wl.small_case(3, 80, 33, 17)
    c = w.views[0].camera
    assert (c.width, c.height) == (33, 17) and (c.cx, c.cy) == (16.5, 8.5)
    _check_scene(w.scenes[0], 80)
