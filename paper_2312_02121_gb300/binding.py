"""Thin ctypes binding of ``libgsplat103.so`` (declared in ``include/gsplat103.h``).

Each ``gs_*`` function here has the name and argument order of the C entry
point and only marshals arguments: torch tensors become device pointers, the
stream defaults to torch's current stream, and a non-zero status raises
``GsError`` with ``gs_last_error()``.  All arithmetic runs in the library's
CUDA kernels; there is no CPU fallback -- importing this module on a machine
where the library cannot be loaded raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import build as _build
from . import debug as _debug

GS_OK = 0
GS_ERR_INVALID_ARG = 1
GS_ERR_CAPACITY = 2
GS_ERR_TIMEOUT = 3
GS_ERR_CUDA = 4
GS_FLAG_CAPACITY = 1
GS_TILE = 16
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


class GsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gsplat103 error {code}: {msg}")
        self.code = code


class GsCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("near_plane", ctypes.c_float), ("far_plane", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class GsView(ctypes.Structure):
    _fields_ = [("cam", GsCamera), ("g_begin", ctypes.c_int32), ("g_count", ctypes.c_int32),
                ("proj_offset", ctypes.c_int64), ("pixel_offset", ctypes.c_int64),
                ("tile_offset", ctypes.c_int32), ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GsRasterConfig(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tile_order", ctypes.c_void_p), ("queue", ctypes.c_void_p), ("warp_hits", ctypes.c_void_p),
                ("bwd_pixels", ctypes.c_int32), ("bwd_batch", ctypes.c_int32)]


class GsTuning(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("longest_first", ctypes.c_int32),
                ("bwd_pixels", ctypes.c_int32), ("bwd_batch", ctypes.c_int32), ("ms", ctypes.c_float)]


class GsAdamConfig(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 5), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


assert ctypes.sizeof(GsCamera) == 80 and ctypes.sizeof(GsView) == 120 and ctypes.sizeof(GsRasterConfig) == 40
assert ctypes.sizeof(GsAdamConfig) == 32 and ctypes.sizeof(GsTuning) == 24

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_F = ctypes.c_float
_D = ctypes.c_double
_SZ = ctypes.c_size_t

# C signatures, in header order
SIGNATURES = {
    "gs_version": (ctypes.c_int, []),
    "gs_last_error": (ctypes.c_char_p, []),
    "gs_kernel_launches": (ctypes.c_int64, []),
    "gs_views_layout": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "gs_project": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _F, _P, _P, _P, _P, _P, _P, _P]),
    "gs_bin_and_sort_workspace_size": (_SZ, [_I64, _I64, _I32]),
    "gs_bin_and_sort": (ctypes.c_int, [_P, _I32, _I64, _I32, _P, _P, _P, _I64, _P, _SZ, _P, _P, _P, _P, _P, _P, _P]),
    "gs_bin_and_sort_static": (ctypes.c_int, [_P, _I32, _I64, _I32, _P, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "gs_tile_order_workspace_size": (_SZ, [_I32]),
    "gs_tile_order": (ctypes.c_int, [_P, _I32, _P, _SZ, _P, _P]),
    "gs_rasterize_fwd": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gs_rasterize_fwd_l2": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _F, _P, _P, _P,
                                           _P]),
    "gs_rasterize_bwd_workspace_size": (_SZ, [_I64, _I32]),
    "gs_rasterize_bwd": (ctypes.c_int, [_P, _I32, _I64, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P,
                                        _P, _P, _I32, _P, _SZ, _P, _P, _P, _P, _P, _P]),
    "gs_project_bwd": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _F, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gs_project_bwd_exclusive": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _F, _P, _P, _P, _P, _P, _P, _P]),
    "gs_autotune_default_candidates": (ctypes.c_int, [_P, _I32, _P]),
    "gs_autotune_workspace_size": (_SZ, [_I64, _I64, _I32, _I64, _I64]),
    "gs_autotune": (ctypes.c_int, [_P, _I32, _I64, _I64, _I32, _I64, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _I32, _I32,
                                   _P, _SZ, _P, _P, _P]),
    "gs_rasterize_fwd_nc": (ctypes.c_int, [_P, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                           _P]),
    "gs_rasterize_bwd_nc": (ctypes.c_int, [_P, _I32, _I64, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                           _P, _P, _P, _P, _P]),
    "gs_l2_loss": (ctypes.c_int, [_P, _P, _I64, _F, _P, _P, _P]),
    "gs_l2_loss_f64": (ctypes.c_int, [_P, _P, _I64, _D, _P, _P, _P]),
    "gs_adam_state_size": (_SZ, [_I64, _I32]),
    "gs_adam_step": (ctypes.c_int, [_I64, _I32, _P, _P, _SZ] + [_P] * 14),
    "gs_activate": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P]),
    "gs_project_f64": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P]),
    "gs_rasterize_fwd_f64": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gs_rasterize_bwd_f64_workspace_size": (_SZ, [_I64, _I32]),
    "gs_rasterize_bwd_f64": (ctypes.c_int, [_P, _I32, _I64, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I64, _P,
                                            _P, _P, _P, _I32, _P, _SZ, _P, _P, _P, _P, _P, _P]),
    "gs_project_bwd_f64": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P, _P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    if _lib is None:
        path = _build.LIB_PATH
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgsplat103.so not found at {path}; build it with paper_2312_02121_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def last_error() -> str:
    return load().gs_last_error().decode()


def _check(code: int):
    if code != GS_OK:
        raise GsError(code, last_error())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("gsplat103 takes device tensors only (got a host tensor)")
    if not t.is_contiguous():
        raise ValueError("gsplat103 needs contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------------------
# views
# ---------------------------------------------------------------------------

def make_camera(cam) -> GsCamera:
    """GsCamera from any object with R, t, fx, fy, cx, cy, width, height, near, far."""
    c = GsCamera()
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float64).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane, c.far_plane = float(cam.near), float(cam.far)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


class Views:
    """A laid-out batch of views: host array, device copy and totals."""

    def __init__(self, cameras: Sequence, g_ranges: Sequence[Tuple[int, int]], device="cuda"):
        V = len(cameras)
        arr = (GsView * max(V, 1))()
        for i, (cam, (gb, gc)) in enumerate(zip(cameras, g_ranges)):
            arr[i].cam = make_camera(cam)
            arr[i].g_begin = int(gb)
            arr[i].g_count = int(gc)
        P, T, pix = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().gs_views_layout(ctypes.cast(arr, _P), V, ctypes.byref(P), ctypes.byref(T), ctypes.byref(pix)))
        self.V, self.P, self.T, self.pixels = V, P.value, T.value, pix.value
        self.host = arr
        raw = bytes(ctypes.string_at(ctypes.addressof(arr), ctypes.sizeof(GsView) * max(V, 1)))
        # an asynchronous copy on the current stream: the driver stages the (pageable) bytes
        # before the call returns, and building views does not wait for work already queued
        self.device = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device, non_blocking=True)
        self.cameras = list(cameras)

    def view(self, i: int) -> GsView:
        return self.host[i]

    def image_slice(self, i: int) -> Tuple[int, int, int, int]:
        """(pixel_offset, width, height, tile_offset) of view i."""
        v = self.host[i]
        return v.pixel_offset, v.cam.width, v.cam.height, v.tile_offset


# ---------------------------------------------------------------------------
# 1:1 wrappers of the C ABI
# ---------------------------------------------------------------------------

def gs_version() -> int:
    return int(load().gs_version())


def gs_kernel_launches() -> int:
    return int(load().gs_kernel_launches())


def _f64(t) -> bool:
    return t is not None and t.dtype == torch.float64


def gs_project(views: Views, means, quats, scales, eps2d: float, means2d, conics, depths, rects, touched,
               K_total=None, stream=None):
    """fp32 or fp64 (gs_project_f64) by the dtype of ``means``; depths are fp32 in both."""
    fn = load().gs_project_f64 if _f64(means) else load().gs_project
    _check(fn(_ptr(views.device), views.V, views.P, _ptr(means), _ptr(quats), _ptr(scales),
                             float(eps2d), _ptr(means2d), _ptr(conics), _ptr(depths), _ptr(rects), _ptr(touched),
                             _ptr(K_total), _stream(stream)))


def gs_bin_and_sort_workspace_size(P: int, K_capacity: int, T_total: int) -> int:
    return int(load().gs_bin_and_sort_workspace_size(P, K_capacity, T_total))


def gs_bin_and_sort(views: Views, rects, depths, touched, K_capacity: int, workspace, isect_ids, isect_pos,
                    emit_start, tile_ranges, K_out, flags, stream=None):
    _check(load().gs_bin_and_sort(_ptr(views.device), views.V, views.P, views.T, _ptr(rects), _ptr(depths),
                                  _ptr(touched), int(K_capacity), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _ptr(isect_ids), _ptr(isect_pos),
                                  _ptr(emit_start), _ptr(tile_ranges), _ptr(K_out), _ptr(flags), _stream(stream)))
    if _debug.enabled():
        _debug.check_binning(views.P, K_capacity, isect_ids, tile_ranges, K_out, flags)


def gs_bin_and_sort_static(views: Views, rects, depths, touched, K_capacity: int, isect_ids, isect_pos, emit_start,
                           tile_ranges, K_out, flags, stream=None):
    """gs_bin_and_sort with the library's fixed device scratch (no workspace)."""
    _check(load().gs_bin_and_sort_static(_ptr(views.device), views.V, views.P, views.T, _ptr(rects), _ptr(depths),
                                         _ptr(touched), int(K_capacity), _ptr(isect_ids), _ptr(isect_pos),
                                         _ptr(emit_start), _ptr(tile_ranges), _ptr(K_out), _ptr(flags),
                                         _stream(stream)))
    if _debug.enabled():
        _debug.check_binning(views.P, K_capacity, isect_ids, tile_ranges, K_out, flags)


class RasterConfig:
    """How the compositing kernels walk the tiles (GsRasterConfig); never
    changes results.  ``tile_order`` (device int32 [T]) and the queue counter
    are kept alive by this object."""

    def __init__(self, persistent: bool = False, ctas_per_sm: int = 0, tile_order=None, device="cuda",
                 warp_hits=None, bwd_pixels: int = 0, bwd_batch: int = 0):
        """``warp_hits``: optional device int32 [K_capacity] buffer through which the forward hands
        its per-pair warp-box cull (one 32-bit ballot per warp box and chunk of 32 pairs) to the
        backward of the same frame.  ``bwd_pixels`` / ``bwd_batch``: the backward's pixels per
        thread and staged batch (0 = defaults; see GsRasterConfig in gsplat103.h)."""
        if warp_hits is not None and (warp_hits.dtype != torch.int32 or warp_hits.device.type != "cuda"):
            raise TypeError("warp_hits must be a device int32 tensor of K_capacity words")
        self.persistent = bool(persistent)
        self.ctas_per_sm = int(ctas_per_sm)
        self.tile_order = tile_order
        self.warp_hits = warp_hits
        self.queue = torch.zeros(1, dtype=torch.int32, device=device) if persistent else None
        self.bwd_pixels, self.bwd_batch = int(bwd_pixels), int(bwd_batch)
        self.c = GsRasterConfig(int(self.persistent), self.ctas_per_sm,
                                None if tile_order is None else tile_order.data_ptr(),
                                None if self.queue is None else self.queue.data_ptr(),
                                None if warp_hits is None else warp_hits.data_ptr(),
                                self.bwd_pixels, self.bwd_batch)

    def ref(self):
        return ctypes.byref(self.c)

    def describe(self) -> dict:
        return {"persistent": self.persistent, "ctas_per_sm": self.ctas_per_sm,
                "tile_order": "longest-first" if self.tile_order is not None else "tile id",
                "warp_hits": self.warp_hits is not None, "bwd_pixels": self.bwd_pixels,
                "bwd_batch": self.bwd_batch}


def _cfg(config: Optional[RasterConfig]):
    return None if config is None else config.ref()


def gs_tile_order_workspace_size(T_total: int) -> int:
    return int(load().gs_tile_order_workspace_size(T_total))


def gs_tile_order(tile_ranges, T_total: int, workspace, order, stream=None):
    _check(load().gs_tile_order(_ptr(tile_ranges), int(T_total), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _ptr(order), _stream(stream)))


def gs_rasterize_fwd(views: Views, means2d, conics, opacities, colors, isect_ids, tile_ranges, background,
                     out_rgb, T_final, last_idx, n_contrib=None, config: Optional[RasterConfig] = None, stream=None):
    fn = load().gs_rasterize_fwd_f64 if _f64(means2d) else load().gs_rasterize_fwd
    _check(fn(_ptr(views.device), views.V, views.T, _ptr(means2d), _ptr(conics),
                                   _ptr(opacities), _ptr(colors), _ptr(isect_ids), _ptr(tile_ranges),
                                   _ptr(background), _ptr(out_rgb), _ptr(T_final), _ptr(last_idx),
                                   _ptr(n_contrib), _cfg(config), _stream(stream)))
    if _debug.enabled():
        _debug.check_forward(views, tile_ranges, out_rgb, T_final, last_idx)


def gs_rasterize_bwd_workspace_size(K_capacity: int, deterministic: bool = False, f64: bool = False) -> int:
    fn = load().gs_rasterize_bwd_f64_workspace_size if f64 else load().gs_rasterize_bwd_workspace_size
    return int(fn(K_capacity, int(bool(deterministic))))


def gs_rasterize_bwd(views: Views, means2d, conics, opacities, colors, isect_ids, isect_pos, emit_start, touched,
                     tile_ranges, K, K_capacity: int, background, T_final, last_idx, dL_drgb, deterministic: bool,
                     workspace, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors,
                     config: Optional[RasterConfig] = None, stream=None):
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    fn = load().gs_rasterize_bwd_f64 if _f64(means2d) else load().gs_rasterize_bwd
    _check(fn(_ptr(views.device), views.V, views.P, views.T, _ptr(means2d), _ptr(conics),
                                   _ptr(opacities), _ptr(colors), _ptr(isect_ids), _ptr(isect_pos),
                                   _ptr(emit_start), _ptr(touched), _ptr(tile_ranges), _ptr(K), int(K_capacity),
                                   _ptr(background), _ptr(T_final), _ptr(last_idx), _ptr(dL_drgb),
                                   int(bool(deterministic)), _ptr(workspace), nbytes, _ptr(dL_dmeans2d),
                                   _ptr(dL_dconics), _ptr(dL_dopacities), _ptr(dL_dcolors), _cfg(config),
                                   _stream(stream)))
    if _debug.enabled():
        _debug.check_gradients([("dL_dmeans2d", dL_dmeans2d), ("dL_dconics", dL_dconics),
                                ("dL_dopacities", dL_dopacities), ("dL_dcolors", dL_dcolors)])


TUNING_FIELDS = ("persistent", "ctas_per_sm", "longest_first", "bwd_pixels", "bwd_batch")


def gs_autotune_default_candidates() -> list:
    """The built-in candidates of gs_autotune, as dicts of the GsTuning fields."""
    return [{k: int(getattr(t, k)) for k in TUNING_FIELDS} for t in _default_candidates()]


def _default_candidates():
    n = ctypes.c_int32(0)
    _check(load().gs_autotune_default_candidates(None, 0, ctypes.byref(n)))
    arr = (GsTuning * n.value)()
    _check(load().gs_autotune_default_candidates(arr, n.value, ctypes.byref(n)))
    return arr


def gs_autotune_workspace_size(P: int, N: int, T_total: int, K_capacity: int, pixels: int) -> int:
    return int(load().gs_autotune_workspace_size(P, N, T_total, K_capacity, pixels))


def gs_autotune(views: Views, N: int, means2d, conics, opacities, colors, isect_ids, tile_ranges, K, K_capacity: int,
                workspace, candidates=None, repeats: int = 3, stream=None):
    """Times the compositing fwd + bwd of a projected and sorted frame for each
    candidate (dicts of the GsTuning fields; None = the built-in ones) and
    returns (best, all), each a dict with the fields and ``ms``.  Waits for
    the stream."""
    cands = None
    n = 0
    if candidates:
        n = len(candidates)
        cands = (GsTuning * n)(*[GsTuning(*[int(c[k]) for k in TUNING_FIELDS], 0.0) for c in candidates])
    else:
        n = len(_default_candidates())
    results = (GsTuning * n)()
    best = GsTuning()
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().gs_autotune(_ptr(views.device), views.V, views.P, int(N), views.T, views.pixels, _ptr(means2d),
                              _ptr(conics), _ptr(opacities), _ptr(colors), _ptr(isect_ids), _ptr(tile_ranges), _ptr(K),
                              int(K_capacity), cands, int(n if candidates else 0), int(repeats), _ptr(workspace),
                              nbytes, results, ctypes.byref(best), _stream(stream)))
    as_dict = lambda t: dict({k: int(getattr(t, k)) for k in TUNING_FIELDS}, ms=float(t.ms))
    return as_dict(best), [as_dict(t) for t in results]


def gs_project_bwd(views: Views, means, quats, scales, eps2d: float, touched, dL_dmeans2d, dL_dconics, dL_dmeans,
                   dL_dquats, dL_dscales, stream=None, dL_dviewmats=None):
    """``dL_dviewmats``: optional [V, 4, 4] buffer (zeroed by the caller) that
    receives dL/dT_cw of every view."""
    fn = load().gs_project_bwd_f64 if _f64(means) else load().gs_project_bwd
    _check(fn(_ptr(views.device), views.V, views.P, _ptr(means), _ptr(quats), _ptr(scales),
                                 float(eps2d), _ptr(touched), _ptr(dL_dmeans2d), _ptr(dL_dconics), _ptr(dL_dmeans),
                                 _ptr(dL_dquats), _ptr(dL_dscales), _ptr(dL_dviewmats), _stream(stream)))


def views_exclusive(views: Views) -> bool:
    """True when no Gaussian belongs to two views (gs_project_bwd_exclusive applies)."""
    ranges = sorted((views.host[i].g_begin, views.host[i].g_begin + views.host[i].g_count) for i in range(views.V)
                    if views.host[i].g_count > 0)
    return all(b[0] >= a[1] for a, b in zip(ranges, ranges[1:]))


def gs_project_bwd_exclusive(views: Views, means, quats, scales, eps2d: float, touched, dL_dmeans2d, dL_dconics,
                             dL_dmeans, dL_dquats, dL_dscales, stream=None):
    """gs_project_bwd when every Gaussian has exactly one projection (the views' Gaussian ranges do not
    overlap, checked here on the host copy of the views): the 3D gradients are written, not
    accumulated, so they need no zero fill.  fp32."""
    if not views_exclusive(views):
        raise GsError(GS_ERR_INVALID_ARG, "gs_project_bwd_exclusive: the views' Gaussian ranges overlap")
    _check(load().gs_project_bwd_exclusive(_ptr(views.device), views.V, views.P, _ptr(means), _ptr(quats),
                                           _ptr(scales), float(eps2d), _ptr(touched), _ptr(dL_dmeans2d),
                                           _ptr(dL_dconics), _ptr(dL_dmeans), _ptr(dL_dquats), _ptr(dL_dscales),
                                           _stream(stream)))


EXPORTED: List[str] = list(SIGNATURES)


def gs_rasterize_fwd_l2(views: Views, means2d, conics, opacities, colors, isect_ids, tile_ranges, background,
                        out_rgb, T_final, last_idx, target, inv_norm: float, dL_drgb=None, loss=None,
                        config: Optional[RasterConfig] = None, stream=None):
    """gs_rasterize_fwd with gs_l2_loss folded in (fp32, 3 channels); ``loss`` is accumulated."""
    _check(load().gs_rasterize_fwd_l2(_ptr(views.device), views.V, views.T, _ptr(means2d), _ptr(conics),
                                      _ptr(opacities), _ptr(colors), _ptr(isect_ids), _ptr(tile_ranges),
                                      _ptr(background), _ptr(out_rgb), _ptr(T_final), _ptr(last_idx), _ptr(target),
                                      float(inv_norm), _ptr(dL_drgb), _ptr(loss), _cfg(config), _stream(stream)))
    if _debug.enabled():
        _debug.check_forward(views, tile_ranges, out_rgb, T_final, last_idx)


def gs_l2_loss(rgb, target, inv_norm: float, dL_drgb=None, loss=None, stream=None):
    """fp32 or fp64 (gs_l2_loss_f64) by the dtype of ``rgb``; ``loss`` is accumulated."""
    fn = load().gs_l2_loss_f64 if _f64(rgb) else load().gs_l2_loss
    _check(fn(_ptr(rgb), _ptr(target), int(rgb.numel()), float(inv_norm), _ptr(dL_drgb), _ptr(loss),
              _stream(stream)))


def gs_adam_state_size(N: int, C: int = 3) -> int:
    return int(load().gs_adam_state_size(int(N), int(C)))


def adam_config(lr: Sequence[float], beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> GsAdamConfig:
    c = GsAdamConfig()
    c.lr[:] = [float(x) for x in lr]
    c.beta1, c.beta2, c.eps = float(beta1), float(beta2), float(eps)
    return c


def gs_adam_step(N: int, cfg: GsAdamConfig, state, means, quats, log_scales, opacity_logits, colors, dL_dmeans,
                 dL_dquats, dL_dscales, dL_dopacities, dL_dcolors, scales, opacities, skip_if_set=None,
                 stream=None):
    nbytes = state.numel() * state.element_size()
    C = int(colors.shape[1]) if colors.dim() == 2 else 3
    _check(load().gs_adam_step(int(N), C, ctypes.byref(cfg), _ptr(state), nbytes, _ptr(means), _ptr(quats),
                               _ptr(log_scales), _ptr(opacity_logits), _ptr(colors), _ptr(dL_dmeans),
                               _ptr(dL_dquats), _ptr(dL_dscales), _ptr(dL_dopacities), _ptr(dL_dcolors),
                               _ptr(scales), _ptr(opacities), _ptr(skip_if_set), _stream(stream)))


def gs_activate(N: int, log_scales, opacity_logits, scales, opacities, stream=None):
    _check(load().gs_activate(int(N), _ptr(log_scales), _ptr(opacity_logits), _ptr(scales), _ptr(opacities),
                              _stream(stream)))


def gs_rasterize_fwd_nc(views: Views, C: int, means2d, conics, opacities, colors, isect_ids, tile_ranges,
                        background, out, T_final, last_idx, n_contrib=None, config: Optional[RasterConfig] = None,
                        stream=None):
    _check(load().gs_rasterize_fwd_nc(_ptr(views.device), views.V, views.T, int(C), _ptr(means2d), _ptr(conics),
                                      _ptr(opacities), _ptr(colors), _ptr(isect_ids), _ptr(tile_ranges),
                                      _ptr(background), _ptr(out), _ptr(T_final), _ptr(last_idx), _ptr(n_contrib),
                                      _cfg(config), _stream(stream)))
    if _debug.enabled():
        _debug.check_forward(views, tile_ranges, out, T_final, last_idx)


def gs_rasterize_bwd_nc(views: Views, C: int, means2d, conics, opacities, colors, isect_ids, tile_ranges,
                        background, T_final, last_idx, dL_dout, dL_dmeans2d, dL_dconics, dL_dopacities, dL_dcolors,
                        config: Optional[RasterConfig] = None, stream=None):
    _check(load().gs_rasterize_bwd_nc(_ptr(views.device), views.V, views.P, views.T, int(C), _ptr(means2d),
                                      _ptr(conics), _ptr(opacities), _ptr(colors), _ptr(isect_ids),
                                      _ptr(tile_ranges), _ptr(background), _ptr(T_final), _ptr(last_idx),
                                      _ptr(dL_dout), _ptr(dL_dmeans2d), _ptr(dL_dconics), _ptr(dL_dopacities),
                                      _ptr(dL_dcolors), _cfg(config), _stream(stream)))
    if _debug.enabled():
        _debug.check_gradients([("dL_dmeans2d", dL_dmeans2d), ("dL_dconics", dL_dconics),
                                ("dL_dopacities", dL_dopacities), ("dL_dcolors", dL_dcolors)])
