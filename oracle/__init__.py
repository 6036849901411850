"""FP64 CPU oracle for the differentiable Gaussian-splatting rasteriser of
"Mathematical Supplement for the gsplat Library" (arXiv 2312.02121).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It is the plain, slow definition the
CUDA library is checked against; it neither imports the CUDA library nor shares
any code with it.  The arithmetic lives in ``gs_oracle.c`` (plain C, double
precision, OpenMP over independent pixels/Gaussians), compiled here on first
use with the system C compiler and loaded through ctypes.

Cameras are duck-typed: any object with R [3,3], t [3], fx, fy, cx, cy, width,
height, near, far.  Inputs are upcast to float64.

Every function cites the passage it follows; the readings taken where the paper
is silent or garbled are listed at the top of ``gs_oracle.c`` (O1-O13).
Parity of the fixed thresholds (O7) and of the dilation eps2d (O11) rests on
that convention, not on the paper ("parity by convention").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgs_oracle.so")
_lib = None
_lock = threading.Lock()

TILE = 16
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into a shared library (gcc, -O2, OpenMP if available)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    cc = os.environ.get("CC", "gcc")
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = [cc, "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("near_plane", ctypes.c_double), ("far_plane", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "or_num_threads": (ctypes.c_int, []),
                "or_quat_to_rotmat": (None, [_P, _P]),
                "or_rotmat_jacobians": (None, [_P, _P, _P, _P, _P]),
                "or_covariance3d": (None, [_P, _P, _P, _P, _P]),
                "or_ewa_jacobian": (None, [_P, _P, _P]),
                "or_ewa_jacobian_dt": (None, [_P, _P, _P]),
                "or_pixel_trace": (_I64, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _I32, _I32, _I32, _P, _P, _P, _P]),
                "or_world_to_pixel": (None, [_P, _P, _P, _P]),
                "or_project": (None, [_P, _I64, _P, _P, _P, _D, _I32] + [_P] * 7),
                "or_rasterize": (None, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _I32, _I32, _I32, _P,
                                        _I64, _P, _P, _P, _P, _P, _P, _P]),
                "or_rasterize_bwd": (None, [_I64, _P, _P, _P, _P, _I32, _P, _P, _P, _I32, _I32, _I32, _P,
                                            _I64, _P, _P, _P, _P, _P, _P]),
                "or_project_bwd": (None, [_P, _I64, _P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P]),
                "or_bin": (_I64, [_I64, _P, _P, _P, _I32, _I32, _P, _P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def _d(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _colors(colors, n: int) -> np.ndarray:
    """[n, C] float64 colours (C = 3 when given as a flat array of 3n)."""
    a = np.asarray(colors, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(n, -1) if n else a.reshape(0, 3)
    return np.ascontiguousarray(a.reshape(n, -1) if n else a)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _cam(cam) -> _Cam:
    c = _Cam()
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float64).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane, c.far_plane = float(cam.near), float(cam.far)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def tiles(cam_or_w, h=None, tile: int = TILE):
    """(TX, TY) tile-grid size of an image."""
    if h is None:
        w, h = cam_or_w.width, cam_or_w.height
    else:
        w = cam_or_w
    return (w + tile - 1) // tile, (h + tile - 1) // tile


# --------------------------------------------------------------------------
# Sec. 2.1 building blocks
# --------------------------------------------------------------------------

def quat_to_rotmat(q) -> np.ndarray:
    """Eq. 5 (R_11 read as 1 - 2(x^2 + z^2)) for a unit quaternion (w,x,y,z)."""
    q = _d(q, (4,))
    R = np.zeros(9)
    _load().or_quat_to_rotmat(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def rotmat_jacobians(q) -> np.ndarray:
    """The printed dR/dw, dR/dx, dR/dy, dR/dz of Sec. 3.2.1, stacked [4,3,3]."""
    q = _d(q, (4,))
    out = [np.zeros(9) for _ in range(4)]
    _load().or_rotmat_jacobians(_ptr(q), *[_ptr(o) for o in out])
    return np.stack([o.reshape(3, 3) for o in out])


def covariance3d(q, s):
    """Eq. 6: Sigma = R S S^T R^T (q normalised first); returns (Sigma, R, M)."""
    q, s = _d(q, (4,)), _d(s, (3,))
    Sig, R, M = np.zeros(9), np.zeros(9), np.zeros(9)
    _load().or_covariance3d(_ptr(q), _ptr(s), _ptr(Sig), _ptr(R), _ptr(M))
    return Sig.reshape(3, 3), R.reshape(3, 3), M.reshape(3, 3)


def ewa_jacobian(cam, t) -> np.ndarray:
    """Eq. 3: J at camera-space point t."""
    c = _cam(cam)
    t = _d(t, (3,))
    J = np.zeros(6)
    _load().or_ewa_jacobian(ctypes.byref(c), _ptr(t), _ptr(J))
    return J.reshape(2, 3)


def ewa_jacobian_dt(cam, t) -> np.ndarray:
    """The printed dJ/dt_x, dJ/dt_y, dJ/dt_z of Sec. 3.2, stacked [3,2,3]."""
    c = _cam(cam)
    t = _d(t, (3,))
    out = np.zeros(18)
    _load().or_ewa_jacobian_dt(ctypes.byref(c), _ptr(t), _ptr(out))
    return out.reshape(3, 2, 3)


def world_to_pixel(cam, mu):
    """Eq. 2 (Reading O2): returns (t, mu')."""
    c = _cam(cam)
    mu = _d(mu, (3,))
    t, m2 = np.zeros(3), np.zeros(2)
    _load().or_world_to_pixel(ctypes.byref(c), _ptr(mu), _ptr(t), _ptr(m2))
    return t, m2


# --------------------------------------------------------------------------
# pipeline stages
# --------------------------------------------------------------------------

def project(cam, means, quats, scales, eps2d: float = 0.3, tile: int = TILE) -> dict:
    """Sec. 2.1 (Eq. 2-6) + 3-sigma tile rectangle (Sec. 2.2, Reading O9)."""
    means, quats, scales = _d(means), _d(quats), _d(scales)
    n = means.shape[0]
    out = dict(means2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conics=np.zeros((n, 3)),
               depths=np.zeros(n), rects=np.zeros((n, 4), np.int32), valid=np.zeros(n, np.int32),
               rect_margin=np.zeros(n))
    c = _cam(cam)
    _load().or_project(ctypes.byref(c), n, _ptr(means), _ptr(quats), _ptr(scales), float(eps2d), tile,
                       _ptr(out["means2d"]), _ptr(out["cov2d"]), _ptr(out["conics"]), _ptr(out["depths"]),
                       _ptr(out["rects"]), _ptr(out["valid"]), _ptr(out["rect_margin"]))
    return out


def _proj_arrays(proj):
    return (_d(proj["means2d"]), _d(proj["conics"]), _d(proj["depths"]),
            np.ascontiguousarray(proj["rects"], dtype=np.int32),
            np.ascontiguousarray(proj["valid"], dtype=np.int32))


def rasterize(proj: dict, opacities, colors, width: int, height: int, background=None,
              pixels=None, tile: int = TILE) -> dict:
    """Sec. 2.2, Eq. 7: front-to-back compositing over each pixel's tile list.

    ``proj`` needs means2d, conics, depths, rects, valid (oracle or any other
    source).  ``colors`` is [N, C] for any channel count C (default 3 when
    given flat); ``background`` has C values.  ``pixels``: optional int64
    array of linear pixel ids (y*W + x); outputs then follow that order.
    Returns rgb [.., C], T_final, last_id, n_contrib, margin (smallest
    relative margin of any alpha / T threshold test) and depth_gap (smallest
    relative depth difference between consecutive Gaussians that pass the
    alpha test, up to the one that stops the pixel; inf if fewer than two)."""
    m2, con, dep, rects, valid = _proj_arrays(proj)
    n = m2.shape[0]
    op, col = _d(opacities, (n,)), _colors(colors, n)
    nc = col.shape[1]
    bg = None if background is None else _d(background, (nc,))
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    npix = width * height if pix is None else pix.shape[0]
    out = dict(rgb=np.zeros((npix, nc)), T_final=np.zeros(npix), last_id=np.zeros(npix, np.int64),
               n_contrib=np.zeros(npix, np.int64), margin=np.zeros(npix), depth_gap=np.zeros(npix))
    _load().or_rasterize(n, _ptr(m2), _ptr(con), _ptr(op), _ptr(col), nc, _ptr(dep), _ptr(rects), _ptr(valid),
                         width, height, tile, _ptr(bg), npix, _ptr(pix),
                         _ptr(out["rgb"]), _ptr(out["T_final"]), _ptr(out["last_id"]), _ptr(out["n_contrib"]),
                         _ptr(out["margin"]), _ptr(out["depth_gap"]))
    if pix is None:
        out["rgb"] = out["rgb"].reshape(height, width, nc)
        for k in ("T_final", "last_id", "n_contrib", "margin", "depth_gap"):
            out[k] = out[k].reshape(height, width)
    return out


def pixel_trace(proj: dict, opacities, colors, px: int, py: int, tile: int = TILE) -> dict:
    """Eq. 7 record of one pixel: composited ids, alpha_n, T_n (running
    product, before n) and the final transmittance."""
    m2, con, dep, rects, valid = _proj_arrays(proj)
    n = m2.shape[0]
    op, col = _d(opacities, (n,)), _colors(colors, n)
    ids, al, T, Tf = np.zeros(max(n, 1), np.int64), np.zeros(max(n, 1)), np.zeros(max(n, 1)), np.zeros(1)
    c = _load().or_pixel_trace(n, _ptr(m2), _ptr(con), _ptr(op), _ptr(col), col.shape[1], _ptr(dep), _ptr(rects),
                               _ptr(valid), tile, px, py, _ptr(ids), _ptr(al), _ptr(T), _ptr(Tf))
    return dict(ids=ids[:c], alpha=al[:c], T=T[:c], T_final=float(Tf[0]))


def rasterize_bwd(proj: dict, opacities, colors, width: int, height: int, dL_drgb,
                  background=None, pixels=None, tile: int = TILE) -> dict:
    """Sec. 3.1: dL/dmu', dL/dconic (packed, O13), dL/do, dL/dc from dL/dC
    (C channels, as in ``rasterize``)."""
    m2, con, dep, rects, valid = _proj_arrays(proj)
    n = m2.shape[0]
    op, col = _d(opacities, (n,)), _colors(colors, n)
    nc = col.shape[1]
    bg = None if background is None else _d(background, (nc,))
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    npix = width * height if pix is None else pix.shape[0]
    g = _d(dL_drgb, (npix, nc))
    out = dict(means2d=np.zeros((n, 2)), conics=np.zeros((n, 3)), opacities=np.zeros(n),
               colors=np.zeros((n, nc)))
    _load().or_rasterize_bwd(n, _ptr(m2), _ptr(con), _ptr(op), _ptr(col), nc, _ptr(dep), _ptr(rects), _ptr(valid),
                             width, height, tile, _ptr(bg), npix, _ptr(pix), _ptr(g),
                             _ptr(out["means2d"]), _ptr(out["conics"]), _ptr(out["opacities"]),
                             _ptr(out["colors"]))
    return out


def project_bwd(cam, means, quats, scales, valid, dL_dmeans2d, dL_dconics, eps2d: float = 0.3) -> dict:
    """Sec. 3.2 / 3.2.1 (Eq. 16-20): dL/dmu, dL/dq (raw quaternion), dL/ds, and
    dL/dT_cw [4,4] (Eq. 20 plus the covariance route through R_cw, Reading
    O14; summed over the Gaussians)."""
    means, quats, scales = _d(means), _d(quats), _d(scales)
    n = means.shape[0]
    valid = np.ascontiguousarray(valid, dtype=np.int32)
    g2, gc = _d(dL_dmeans2d, (n, 2)), _d(dL_dconics, (n, 3))
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), scales=np.zeros((n, 3)), viewmat=np.zeros(16))
    c = _cam(cam)
    _load().or_project_bwd(ctypes.byref(c), n, _ptr(means), _ptr(quats), _ptr(scales), float(eps2d),
                           _ptr(valid), _ptr(g2), _ptr(gc), _ptr(out["means"]), _ptr(out["quats"]),
                           _ptr(out["scales"]), _ptr(out["viewmat"]))
    out["viewmat"] = out["viewmat"].reshape(4, 4)
    return out


def bin_tiles(rects, depths_f32, valid, TX: int, TY: int):
    """Sec. 2.2 binning by brute force over all (Gaussian, tile) pairs, ordered by
    (tile, float32 depth, index).  Returns (ids [K] int64, ranges [TX*TY, 2])."""
    rects = np.ascontiguousarray(rects, dtype=np.int32)
    dep = np.ascontiguousarray(depths_f32, dtype=np.float32)
    valid = np.ascontiguousarray(valid, dtype=np.int32)
    n = rects.shape[0]
    lib = _load()
    K = lib.or_bin(n, _ptr(rects), _ptr(dep), _ptr(valid), TX, TY, None, None)
    ids = np.zeros(max(K, 1), np.int64)
    ranges = np.zeros((TX * TY, 2), np.int64)
    lib.or_bin(n, _ptr(rects), _ptr(dep), _ptr(valid), TX, TY, _ptr(ids), _ptr(ranges))
    return ids[:K], ranges


# --------------------------------------------------------------------------
# whole path
# --------------------------------------------------------------------------

def render(cam, scene, eps2d: float = 0.3, background=None, pixels=None) -> dict:
    """Forward of Sec. 2: projection then compositing.  ``scene`` has means,
    quats, scales, opacities, colors."""
    proj = project(cam, scene.means, scene.quats, scene.scales, eps2d)
    out = rasterize(proj, scene.opacities, scene.colors, cam.width, cam.height, background, pixels)
    out["proj"] = proj
    return out


def backward(cam, scene, dL_drgb, eps2d: float = 0.3, background=None, pixels=None) -> dict:
    """Backward of Sec. 3: returns dL/d{means, quats, scales, opacities, colors},
    dL/dT_cw (``viewmat``, [4,4])
    plus the 2D intermediates (means2d, conics)."""
    proj = project(cam, scene.means, scene.quats, scene.scales, eps2d)
    g2d = rasterize_bwd(proj, scene.opacities, scene.colors, cam.width, cam.height, dL_drgb, background, pixels)
    g3d = project_bwd(cam, scene.means, scene.quats, scene.scales, proj["valid"], g2d["means2d"],
                      g2d["conics"], eps2d)
    return dict(means=g3d["means"], quats=g3d["quats"], scales=g3d["scales"], opacities=g2d["opacities"],
                colors=g2d["colors"], means2d=g2d["means2d"], conics=g2d["conics"], viewmat=g3d["viewmat"],
                proj=proj)


def finite_difference(cam, scene, dL_drgb, name: str, index, h: float = 1e-6, eps2d: float = 0.3,
                      background=None) -> float:
    """Central difference of L = <dL_drgb, C> w.r.t. one scalar parameter
    ``getattr(scene, name)[index]`` (step h relative to max(|x|, 1e-3))."""
    base = getattr(scene, name)
    x0 = float(np.asarray(base, np.float64)[index])
    step = h * max(abs(x0), 1e-3)

    class _S:  # a float64 copy of the scene with one entry moved
        pass

    def loss(v):
        s = _S()
        for k in ("means", "quats", "scales", "opacities", "colors"):
            setattr(s, k, np.array(getattr(scene, k), dtype=np.float64))
        getattr(s, name)[index] = v
        img = render(cam, s, eps2d, background)["rgb"]
        return float(np.sum(img * np.asarray(dL_drgb, np.float64).reshape(img.shape)))

    return (loss(x0 + step) - loss(x0 - step)) / (2 * step)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
