"""Seeded synthetic scenes and cameras.

This module only draws inputs: Gaussian parameters, cameras and target images,
from ``numpy.random.default_rng``.  It holds none of the rasteriser's
arithmetic, so that the CUDA path and the FP64 oracle can both be fed from it
without sharing any of the method.

Conventions (OpenCV camera): x right, y down, z forward; a camera "at distance
d" has R_cw = I and t_cw = (0, 0, d), i.e. it sits at (0, 0, -d) looking along
+z, with the principal point at the image centre.  Quaternions are stored
(w, x, y, z).  All arrays are C-contiguous float32 (the precision the CUDA path
computes in); the oracle upcasts them to float64.

Named workloads (the sizes are the ones the benchmark and the tests use):

* ``forward_1k_128``      1,000 Gaussians, one 128x128 camera (forward only)
* ``fwdbwd_100k_1024x768``  100,000 Gaussians, one 1024x768 camera + target
* ``gradcheck_64_32``     64 Gaussians, 32x32 (the 1024x768 scene scaled down)
* ``fwdbwd_1m_1080p``     1,000,000 Gaussians (64-component mixture), 1920x1080
* ``batch_views_500k_64`` one 500,000-Gaussian mixture seen by 64 uneven cameras
* ``batch_scenes_16x4``   16 scenes of log-uniform size in [1e4, 2e6], 4 views each
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Camera:
    """World-to-camera extrinsics (R row-major, t) and pinhole intrinsics."""

    R: np.ndarray  # [3,3] float32
    t: np.ndarray  # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01
    far: float = 100.0

    @property
    def pixels(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class Scene:
    """Gaussian parameters (float32): means [N,3], quats [N,4] (w,x,y,z),
    scales [N,3] (linear, not log), opacities [N], colors [N,3]."""

    means: np.ndarray
    quats: np.ndarray
    scales: np.ndarray
    opacities: np.ndarray
    colors: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


@dataclasses.dataclass
class View:
    scene: int
    camera: Camera


@dataclasses.dataclass
class Workload:
    name: str
    scenes: List[Scene]
    views: List[View]
    targets: Optional[List[np.ndarray]]  # per view [H,W,3] float32, or None
    eps2d: float = 0.3
    backward: bool = True

    @property
    def pixels(self) -> int:
        return sum(v.camera.pixels for v in self.views)

    @property
    def gaussians(self) -> int:
        return sum(s.n for s in self.scenes)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def sigmoid(x: np.ndarray) -> np.ndarray:
    return 1.0 / (1.0 + np.exp(-x))


def camera_at_distance(d: float, width: int, height: int, f: float,
                       near: float = 0.01, far: float = 100.0) -> Camera:
    """Identity rotation, camera centre at (0, 0, -d)."""
    return Camera(R=_f32(np.eye(3)), t=_f32([0.0, 0.0, d]), fx=float(f), fy=float(f),
                  cx=width / 2.0, cy=height / 2.0, width=int(width), height=int(height),
                  near=near, far=far)


def look_at_camera(centre: np.ndarray, target: np.ndarray, width: int, height: int,
                   f: float, near: float = 0.01, far: float = 100.0) -> Camera:
    """Camera at ``centre`` looking at ``target``; world 'up' is -y, so the
    camera's y axis (down) follows world +y."""
    z = np.asarray(target, np.float64) - np.asarray(centre, np.float64)
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    y = down - np.dot(down, z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    R = np.stack([x, y, z])  # rows: camera axes in world coordinates
    t = -R @ np.asarray(centre, np.float64)
    return Camera(R=_f32(R), t=_f32(t), fx=float(f), fy=float(f), cx=width / 2.0,
                  cy=height / 2.0, width=int(width), height=int(height), near=near, far=far)


def sphere_cameras(rng: np.random.Generator, count: int, radius: float,
                   resolutions, focal_range=None, focal=None) -> List[Camera]:
    """``count`` look-at cameras on a sphere around the origin; directions are
    normalised N(0,1)^3, re-drawn when nearly parallel to the up axis."""
    cams = []
    while len(cams) < count:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if abs(d[1]) > 0.98:
            continue
        if len(resolutions) == 1:
            w, h = resolutions[0]
        else:
            w, h = resolutions[int(rng.integers(len(resolutions)))]
        f = focal if focal is not None else float(rng.uniform(*focal_range))
        cams.append(look_at_camera(radius * d, np.zeros(3), w, h, f))
    return cams


def random_scene(rng: np.random.Generator, n: int, means: np.ndarray, log_scale_mu: float,
                 log_scale_sigma: float, opacity_logit_mu: float, opacity_logit_sigma: float) -> Scene:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return Scene(
        means=_f32(means),
        quats=_f32(q),
        scales=_f32(np.exp(rng.normal(log_scale_mu, log_scale_sigma, (n, 3)))),
        opacities=_f32(sigmoid(rng.normal(opacity_logit_mu, opacity_logit_sigma, n))),
        colors=_f32(rng.uniform(0.0, 1.0, (n, 3))),
    )


def mixture_means(rng: np.random.Generator, n: int, components: int = 64,
                  extent: float = 5.0, std: float = 0.5) -> np.ndarray:
    centres = rng.uniform(-extent, extent, (components, 3))
    which = rng.integers(components, size=n)
    return centres[which] + rng.normal(0.0, std, (n, 3))


def target_image(rng: np.random.Generator, cam: Camera) -> np.ndarray:
    return _f32(rng.uniform(0.0, 1.0, (cam.height, cam.width, 3)))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def forward_1k_128(seed: int = 0) -> Workload:
    rng = np.random.default_rng(seed)
    n = 1000
    means = rng.uniform(-1.0, 1.0, (n, 3))
    scene = random_scene(rng, n, means, -3.0, 0.5, 0.0, 1.0)
    cam = Camera(R=_f32(np.eye(3)), t=_f32([0, 0, 3.0]), fx=128.0, fy=128.0, cx=64.0, cy=64.0,
                 width=128, height=128)
    return Workload("forward_1k_128", [scene], [View(0, cam)], None, backward=False)


def fwdbwd_100k_1024x768(seed: int = 0, n: int = 100_000, width: int = 1024, height: int = 768,
                         f: float = 900.0, log_scale_shift: float = 0.0) -> Workload:
    rng = np.random.default_rng(seed)
    means = rng.uniform(-2.0, 2.0, (n, 3))
    scene = random_scene(rng, n, means, -4.0 + log_scale_shift, 0.7, 0.0, 1.5)
    cam = camera_at_distance(5.0, width, height, f)
    target = target_image(np.random.default_rng(seed + 1), cam)
    return Workload(f"fwdbwd_{n}_{width}x{height}", [scene], [View(0, cam)], [target])


def gradcheck_64_32(seed: int = 1) -> Workload:
    """The 1024x768 scene family shrunk to 64 Gaussians on 32x32 pixels: focal
    scaled by 32/1024, log-scales shifted by ln 32 so footprints in pixels match.
    Seed 1 keeps every threshold test (alpha_min, alpha_max, T_min, tile-box
    edges) at least 5e-4 (relative) away from its threshold, so finite
    differences never cross one; seed 0 has a pixel within 1e-5."""
    return fwdbwd_100k_1024x768(seed, n=64, width=32, height=32, f=900.0 * 32 / 1024,
                                log_scale_shift=math.log(32.0))


def fwdbwd_1m_1080p(seed: int = 0, n: int = 1_000_000, width: int = 1920, height: int = 1080,
                    f: float = 1100.0) -> Workload:
    rng = np.random.default_rng(seed)
    means = mixture_means(rng, n)
    scene = random_scene(rng, n, means, -4.5, 1.0, -1.0, 2.0)
    cam = camera_at_distance(12.0, width, height, f)
    target = target_image(np.random.default_rng(seed + 1), cam)
    return Workload(f"fwdbwd_{n}_{width}x{height}", [scene], [View(0, cam)], [target])


BATCH_RESOLUTIONS = [(256, 256), (640, 480), (1024, 768), (1280, 720)]


def batch_views_500k_64(seed: int = 0, n: int = 500_000, views: int = 64,
                        resolutions=None) -> Workload:
    rng = np.random.default_rng(seed)
    means = mixture_means(rng, n)
    scene = random_scene(rng, n, means, -4.5, 1.0, -1.0, 2.0)
    cams = sphere_cameras(rng, views, 10.0, resolutions or BATCH_RESOLUTIONS, focal_range=(300.0, 1200.0))
    trng = np.random.default_rng(seed + 1)
    return Workload(f"batch_views_{n}_{views}", [scene], [View(0, c) for c in cams],
                    [target_image(trng, c) for c in cams])


def batch_scenes_16x4(seed: int = 0, scenes: int = 16, views_per_scene: int = 4,
                      n_range=(10_000, 2_000_000), width: int = 960, height: int = 540,
                      f: float = 800.0) -> Workload:
    rng = np.random.default_rng(seed)
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    sc, vs = [], []
    for s in range(scenes):
        n = int(round(math.exp(rng.uniform(lo, hi))))
        means = rng.uniform(-2.0, 2.0, (n, 3))
        sc.append(random_scene(rng, n, means, -4.0, 0.7, 0.0, 1.5))
        for cam in sphere_cameras(rng, views_per_scene, 5.0, [(width, height)], focal=f):
            vs.append(View(s, cam))
    trng = np.random.default_rng(seed + 1)
    return Workload(f"batch_scenes_{scenes}x{views_per_scene}", sc, vs,
                    [target_image(trng, v.camera) for v in vs])


def small_case(seed: int, n: int, width: int, height: int, f: Optional[float] = None,
               distance: float = 4.0, log_scale_mu: float = -3.0, log_scale_sigma: float = 0.6,
               opacity_logit_mu: float = 0.0, opacity_logit_sigma: float = 1.5,
               extent: float = 1.5) -> Workload:
    """A small single-view scene for parity tests (sizes the oracle finishes
    in seconds); width/height need not be multiples of the 16-pixel tile."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, (n, 3))
    scene = random_scene(rng, n, means, log_scale_mu, log_scale_sigma, opacity_logit_mu, opacity_logit_sigma)
    cam = camera_at_distance(distance, width, height, f if f is not None else 1.1 * max(width, height))
    target = target_image(np.random.default_rng(seed + 1), cam)
    return Workload(f"small_{n}_{width}x{height}", [scene], [View(0, cam)], [target])


WORKLOADS: Dict[str, object] = {
    "forward_1k_128": forward_1k_128,
    "fwdbwd_100k_1024x768": fwdbwd_100k_1024x768,
    "gradcheck_64_32": gradcheck_64_32,
    "fwdbwd_1m_1080p": fwdbwd_1m_1080p,
    "batch_views_500k_64": batch_views_500k_64,
    "batch_scenes_16x4": batch_scenes_16x4,
}
