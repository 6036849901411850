"""Batched rendering: many views (cameras) of one or several scenes per launch.

``BatchRenderer`` runs the whole training-style step -- projection, binning
and sort, compositing, the L2-loss gradient, compositing backward and
projection backward -- over every view with ONE launch per stage, into
preallocated buffers, so the step can be captured once into a CUDA graph and
replayed.  The intersection capacity is fixed at construction (graphs need
static sizes); ``overflowed()`` reports a step whose pairs did not fit.

``PerViewRenderer`` is the comparison point: the same kernels launched once
per view.  ``autotune`` picks how the compositing kernels walk the tiles
(one CTA per tile or a persistent grid over a global queue; tile-id or
longest-first order; CTAs per SM) and the backward's batch shape (pixels per
thread, staged batch) through the library's gs_autotune, which times each
candidate on the device; none of these choices changes any result.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from .pipeline import Params


class BatchRenderer:
    def __init__(self, params: Params, views: B.Views, K_capacity: int, targets: Optional[torch.Tensor] = None,
                 eps2d: float = 0.3, config: Optional[B.RasterConfig] = None, longest_first: bool = False,
                 deterministic: bool = False, background: Optional[torch.Tensor] = None,
                 shared_grads: Optional[Dict[str, torch.Tensor]] = None, loss_pixels: Optional[int] = None):
        """``shared_grads``: per-Gaussian gradient buffers (means, quats,
        scales, opacities, colors) owned and zeroed by the caller, into which
        this renderer accumulates; by default the renderer owns them.
        ``loss_pixels``: the pixel count the L2 loss is a mean over (default:
        this renderer's own pixels; a rank rendering part of a larger job
        passes the job's total)."""
        self.p, self.views, self.eps2d = params, views, eps2d
        self.cap = max(int(K_capacity), 1)
        self.config, self.longest_first, self.deterministic = config, longest_first, deterministic
        self.background = background
        dev = params.means.device
        P, T, pix, N = views.P, views.T, views.pixels, params.n
        C = self.C = params.channels
        if deterministic and C != 3:
            raise ValueError("the deterministic backward composites 3 channels")
        e = lambda *shape, dtype=torch.float32: torch.empty(*shape, dtype=dtype, device=dev)
        self.means2d, self.conics, self.depths = e(max(P, 1), 2), e(max(P, 1), 3), e(max(P, 1))
        self.rects = e(max(P, 1), 4, dtype=torch.int16)
        self.touched = e(max(P, 1), dtype=torch.int32)
        self.sort_ws = e(B.gs_bin_and_sort_workspace_size(P, self.cap, T), dtype=torch.uint8)
        self.isect_ids, self.isect_pos = e(self.cap, dtype=torch.int32), e(self.cap, dtype=torch.int32)
        self.emit_start = e(max(P, 1), dtype=torch.int32)
        self.tile_ranges = e(T, 2, dtype=torch.int32)
        self.K = e(1, dtype=torch.int32)
        self.order_ws = e(max(B.gs_tile_order_workspace_size(T), 1), dtype=torch.uint8)
        self.tile_order = e(T, dtype=torch.int32)
        self.rgb, self.T_final = e(pix, C), e(pix)
        self.last_idx = e(pix, dtype=torch.int32)
        self.targets = targets
        # three channels with a target: the forward kernel takes the L2 loss and dL/dC itself
        # (gs_rasterize_fwd_l2), so no second kernel reads the image back
        self.fuse_loss = targets is not None and C == 3
        self.inv_norm = 1.0 / (C * (loss_pixels if loss_pixels is not None else max(pix, 1)))
        self.dL = e(pix, C)
        nbw = B.gs_rasterize_bwd_workspace_size(self.cap, deterministic)
        self.bwd_ws = e(nbw, dtype=torch.uint8) if nbw else None
        # every buffer the step zeroes lives in one allocation, cleared by one fill at the start of the
        # step: the sort's flag word and the loss (the "state" words), then the gradient accumulators
        self.owns_grads = shared_grads is None
        Pm, Nm = max(P, 1), max(N, 1)
        shapes = [("state", (4,)), ("g2", (Pm, 2)), ("gc", (Pm, 3))]
        if self.owns_grads:
            shapes += [("g_op", (Nm,)), ("g_col", (Nm, C)), ("g_means", (Nm, 3)), ("g_quats", (Nm, 4)),
                       ("g_scales", (Nm, 3))]
        # each buffer starts on a 16-byte boundary (the quaternion gradients take 16-byte stores)
        offs, off = {}, 0
        for name, sh in shapes:
            offs[name] = off
            off += (int(np.prod(sh)) + 3) // 4 * 4
        self.grad_flat = torch.zeros(off, device=dev)  # the state words read zero before the first step
        for name, sh in shapes:
            n = int(np.prod(sh))
            setattr(self, name, self.grad_flat[offs[name]:offs[name] + n].view(*sh))
        # when every Gaussian belongs to exactly one view, the projection backward writes the 3D gradients
        # instead of adding to them (gs_project_bwd_exclusive), and the fill stops before them
        spans = sorted((views.host[i].g_begin, views.host[i].g_begin + views.host[i].g_count)
                       for i in range(views.V) if views.host[i].g_count > 0)
        covers_once = bool(spans) and spans[0][0] == 0 and spans[-1][1] == N and all(
            b[0] == a[1] for a, b in zip(spans, spans[1:]))
        self.exclusive = self.owns_grads and covers_once
        fill_end = offs["g_means"] if self.exclusive else off
        self.step_fill = self.grad_flat[:fill_end]  # zeroed by forward
        self.grad_fill = self.grad_flat[offs["g2"]:fill_end]  # the gradients alone, for a repeated backward
        self.flags = self.state[0:1].view(torch.int32)
        self.loss = self.state[1:2]
        self.grads_cleared = False  # set by forward's fill, used up by the next backward
        if not self.owns_grads:
            sg = shared_grads
            self.g_op, self.g_col = sg["opacities"], sg["colors"]
            self.g_means, self.g_quats, self.g_scales = sg["means"], sg["quats"], sg["scales"]
        # the forward hands its per-pair warp-box cull to the backward (kernels of up to 3 channels)
        self.warp_hits = e(self.cap, dtype=torch.int32) if C <= 3 else None
        cfg = config or B.RasterConfig(device=dev)
        self.config = B.RasterConfig(cfg.persistent, cfg.ctas_per_sm,
                                     self.tile_order if longest_first else cfg.tile_order, device=dev,
                                     warp_hits=self.warp_hits, bwd_pixels=cfg.bwd_pixels, bwd_batch=cfg.bwd_batch)
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self.host = None

    # -- inputs from host memory ---------------------------------------------
    def attach_host_inputs(self, params: Dict[str, torch.Tensor], targets: Optional[torch.Tensor] = None):
        """Makes every step start by copying its inputs from pinned host
        memory and end by copying the loss into the pinned host scalar
        ``loss_host``.  ``params`` maps means, quats, scales, opacities and
        colors to pinned host tensors shaped like the renderer's parameters;
        ``targets`` is the pinned host [pixels, C] target.  The projection's
        inputs (means, quats, scales) are copied first, on the step's stream;
        the copies of what compositing and the loss read (opacities, colours,
        target) follow on a second stream, so that they overlap projection and
        sorting instead of sharing the link with the projection's inputs, and
        the step waits for them only where they are needed.  Attach before
        ``capture``: the copies are then part of the graph, and each replay
        reads whatever the host tensors hold at that time."""
        for k in ("means", "quats", "scales", "opacities", "colors"):
            h, d = params[k], getattr(self.p, k)
            if not h.is_pinned() or h.shape != d.shape or h.dtype != d.dtype:
                raise ValueError(f"host {k} must be pinned and shaped {tuple(d.shape)} {d.dtype}")
        if targets is not None and (not targets.is_pinned() or targets.numel() != self.targets.numel()):
            raise ValueError("host targets must be pinned and hold as many values as the device targets")
        self.host = dict(params=params, targets=targets, stream=torch.cuda.Stream(),
                         early=torch.cuda.Event(), late=torch.cuda.Event(), tgt=torch.cuda.Event())
        self.loss_host = torch.zeros(1, dtype=self.loss.dtype, pin_memory=True)

    def _upload(self):
        """Issues this step's host -> device copies; returns after the ones
        the projection needs are enqueued on the current stream."""
        h, p = self.host, self.p
        main = torch.cuda.current_stream()
        # stream order makes the previous step done with every input buffer; the link is shared (about
        # 200 GB/s either way), so the projection's inputs go alone first
        for k in ("means", "quats", "scales"):
            getattr(p, k).copy_(h["params"][k], non_blocking=True)
        h["early"].record(main)
        side = h["stream"]
        side.wait_event(h["early"])
        with torch.cuda.stream(side):
            p.opacities.copy_(h["params"]["opacities"], non_blocking=True)
            p.colors.copy_(h["params"]["colors"], non_blocking=True)
            h["late"].record(side)
            if h["targets"] is not None:
                self.targets.view(-1).copy_(h["targets"].view(-1), non_blocking=True)
            h["tgt"].record(side)

    # -- one step, eagerly --------------------------------------------------
    def forward(self):
        v, p = self.views, self.p
        if self.host is not None:
            self._upload()
        self.step_fill.zero_()  # the flag word, the loss and the gradient accumulators of this step
        self.grads_cleared = True
        B.gs_project(v, p.means, p.quats, p.scales, self.eps2d, self.means2d, self.conics, self.depths, self.rects,
                     self.touched, None)  # the pair count comes from the sort (no per-block atomics here)
        B.gs_bin_and_sort(v, self.rects, self.depths, self.touched, self.cap, self.sort_ws, self.isect_ids,
                          self.isect_pos if self.deterministic else None,
                          self.emit_start if self.deterministic else None, self.tile_ranges, self.K,
                          self.flags)
        if self.longest_first:
            B.gs_tile_order(self.tile_ranges, v.T, self.order_ws, self.tile_order)
        if self.host is not None:
            torch.cuda.current_stream().wait_event(self.host["tgt" if self.fuse_loss else "late"])
        if self.fuse_loss:
            B.gs_rasterize_fwd_l2(v, self.means2d, self.conics, p.opacities, p.colors, self.isect_ids,
                                  self.tile_ranges, self.background, self.rgb, self.T_final, self.last_idx,
                                  self.targets, self.inv_norm, self.dL, self.loss, self.config)
        elif self.C == 3:
            B.gs_rasterize_fwd(v, self.means2d, self.conics, p.opacities, p.colors, self.isect_ids, self.tile_ranges,
                               self.background, self.rgb, self.T_final, self.last_idx, None, self.config)
        else:
            B.gs_rasterize_fwd_nc(v, self.C, self.means2d, self.conics, p.opacities, p.colors, self.isect_ids,
                                  self.tile_ranges, self.background, self.rgb, self.T_final, self.last_idx, None,
                                  self.config)

    def loss_grad(self):
        """L = mean((C - target)^2) over every pixel of every view (into
        ``self.loss``, on the device) and dL/dC, in one kernel; with three
        channels the forward has already done both."""
        if self.fuse_loss:
            return
        if self.host is not None:
            torch.cuda.current_stream().wait_event(self.host["tgt"])
        self.loss.zero_()
        B.gs_l2_loss(self.rgb, self.targets, self.inv_norm, self.dL, self.loss)

    def backward(self):
        v, p = self.views, self.p
        if not self.grads_cleared:  # a second backward after one forward starts from zero again
            self.grad_fill.zero_()
        self.grads_cleared = False
        if self.C == 3:
            B.gs_rasterize_bwd(v, self.means2d, self.conics, p.opacities, p.colors, self.isect_ids, self.isect_pos,
                               self.emit_start, self.touched, self.tile_ranges, self.K, self.cap, self.background,
                               self.T_final, self.last_idx, self.dL, self.deterministic, self.bwd_ws, self.g2,
                               self.gc, self.g_op, self.g_col, self.config)
        else:
            B.gs_rasterize_bwd_nc(v, self.C, self.means2d, self.conics, p.opacities, p.colors, self.isect_ids,
                                  self.tile_ranges, self.background, self.T_final, self.last_idx, self.dL, self.g2,
                                  self.gc, self.g_op, self.g_col, self.config)
        project_bwd = B.gs_project_bwd_exclusive if self.exclusive else B.gs_project_bwd
        project_bwd(v, p.means, p.quats, p.scales, self.eps2d, self.touched, self.g2, self.gc, self.g_means,
                    self.g_quats, self.g_scales)
        if self.host is not None:
            self.loss_host.copy_(self.loss, non_blocking=True)

    def step_eager(self):
        self.forward()
        self.loss_grad()
        self.backward()

    # -- CUDA graph ---------------------------------------------------------
    def capture(self):
        """Captures one whole step into a CUDA graph (after two eager warm-ups
        on a side stream, as graph capture requires)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(2):
                self.step_eager()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step_eager()
        self.graph = g

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.step_eager()

    def overflowed(self) -> bool:
        return bool(int(self.flags.item()) & B.GS_FLAG_CAPACITY)

    def grads(self) -> Dict[str, torch.Tensor]:
        N = self.p.n
        return dict(means=self.g_means[:N], quats=self.g_quats[:N], scales=self.g_scales[:N],
                    opacities=self.g_op[:N], colors=self.g_col[:N])

    def image(self, i: int) -> torch.Tensor:
        off, w, h, _ = self.views.image_slice(i)
        return self.rgb[off:off + w * h].view(h, w, -1)


class HostPipeline:
    """Steps fed from pinned host memory, two deep: two renderers (each with
    its own device buffers and host inputs attached, see
    ``BatchRenderer.attach_host_inputs``) replay their captured steps on two
    streams in turn, so that one step's host->device copies and compute
    overlap the previous step's.  Every step still copies its own inputs from
    the host and reads its own loss back; ``step`` returns the loss of the
    step before it (None for the first), ``finish`` the last one's."""

    def __init__(self, make):
        """``make()`` returns a BatchRenderer whose host inputs are attached."""
        self.r = [make(), make()]
        self.s = [torch.cuda.Stream(), torch.cuda.Stream()]
        self.done = [torch.cuda.Event(), torch.cuda.Event()]
        for r, st in zip(self.r, self.s):
            if r.host is None:
                raise ValueError("HostPipeline needs renderers with host inputs attached")
            st.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(st):
                r.capture()
        self.k = 0

    def step(self) -> Optional[float]:
        i = self.k % 2
        with torch.cuda.stream(self.s[i]):
            self.r[i].step()
            self.done[i].record()
        prev = None
        if self.k > 0:
            j = 1 - i
            self.done[j].synchronize()
            prev = float(self.r[j].loss_host[0])
        self.k += 1
        return prev

    def finish(self) -> Optional[float]:
        if self.k == 0:
            return None
        j = (self.k - 1) % 2
        self.done[j].synchronize()
        return float(self.r[j].loss_host[0])

    def overflowed(self) -> bool:
        return any(r.overflowed() for r in self.r)


class PerViewRenderer:
    """The same step with one set of launches per view (the per-view path the
    batched launch is measured against).  All views accumulate into one
    shared set of per-Gaussian gradient buffers, zeroed once per step."""

    def __init__(self, params: Params, cameras: Sequence, g_ranges, K_caps: Sequence[int],
                 targets: torch.Tensor, eps2d: float = 0.3, deterministic: bool = False):
        """``targets``: the packed [pixels, 3] targets of all views, in view order."""
        dev = params.means.device
        N = max(params.n, 1)
        self.C = params.channels
        self.shared = dict(means=torch.empty(N, 3, device=dev), quats=torch.empty(N, 4, device=dev),
                           scales=torch.empty(N, 3, device=dev), opacities=torch.empty(N, device=dev),
                           colors=torch.empty(N, self.C, device=dev))
        self.n = params.n
        self.r: List[BatchRenderer] = []
        off = 0
        # the same loss as the batch: a mean over every pixel of every view
        self.n_pix = sum(cam.width * cam.height for cam in cameras)
        for cam, gr, cap in zip(cameras, g_ranges, K_caps):
            pix = cam.width * cam.height
            tgt = targets[off:off + pix]
            off += pix
            v = B.Views([cam], [gr], device=dev)
            self.r.append(BatchRenderer(params, v, cap, tgt, eps2d, deterministic=deterministic,
                                        shared_grads=self.shared, loss_pixels=self.n_pix))

    def step(self):
        for t in self.shared.values():
            t.zero_()
        for r in self.r:
            r.forward()
            r.loss_grad()
            r.backward()

    def overflowed(self) -> bool:
        return any(r.overflowed() for r in self.r)

    def grads(self) -> Dict[str, torch.Tensor]:
        return {k: v[:self.n] for k, v in self.shared.items()}


def per_view_capacities(params: Params, cameras: Sequence, g_ranges, eps2d: float = 0.3) -> List[int]:
    return [exact_capacity(params, B.Views([c], [g], device=params.means.device), eps2d)
            for c, g in zip(cameras, g_ranges)]


def exact_capacity(params: Params, views: B.Views, eps2d: float = 0.3) -> int:
    """Intersections of the batch (one projection pass, one read-back)."""
    dev = params.means.device
    P = max(views.P, 1)
    tmp = [torch.empty(P, 2, device=dev), torch.empty(P, 3, device=dev), torch.empty(P, device=dev),
           torch.empty(P, 4, dtype=torch.int16, device=dev), torch.empty(P, dtype=torch.int32, device=dev)]
    K = torch.empty(1, dtype=torch.int64, device=dev)
    B.gs_project(views, params.means, params.quats, params.scales, eps2d, *tmp, K)
    return int(K.item())


def time_steps(step, n: int = 5, warmup: int = 2) -> float:
    """Mean device time of ``step`` in ms (CUDA events)."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n):
        step()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


# The tile walks the GPU tests exercise (the autotuner's candidates are gs_autotune's built-in ones:
# these walks times the backward batch shapes).
CANDIDATES = [
    dict(persistent=False, ctas_per_sm=0, longest_first=False),
    dict(persistent=False, ctas_per_sm=0, longest_first=True),
    dict(persistent=True, ctas_per_sm=0, longest_first=True),
    dict(persistent=True, ctas_per_sm=4, longest_first=True),
    dict(persistent=True, ctas_per_sm=3, longest_first=True),
]


def _cache_path() -> str:
    root = os.environ.get("GSPLAT103_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gsplat103"))
    return os.path.join(root, "tuning.json")


def autotune(renderer: "BatchRenderer", key: str, candidates=None, use_cache: bool = True, repeats: int = 5) -> dict:
    """Picks the tile walk and backward batch shape for ``renderer``'s frame
    with the library's gs_autotune (which times the compositing forward +
    backward of each candidate on the device) and returns the fastest as a
    dict (persistent, ctas_per_sm, longest_first, bwd_pixels, bwd_batch, ms,
    all = every candidate's time, cached).  The choice is cached per GPU name
    and ``key``; ``config(best)`` and ``best["longest_first"]`` build a
    renderer that walks that way."""
    gpu = torch.cuda.get_device_name()
    ck = f"{gpu}|{key}"
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if ck in cache:
        return dict(cache[ck], cached=True)
    r = renderer
    r.forward()  # the frame the candidates composite: projection and sorted lists in r's buffers
    ws = torch.empty(B.gs_autotune_workspace_size(r.views.P, r.p.n, r.views.T, r.cap, r.views.pixels),
                     dtype=torch.uint8, device=r.p.means.device)
    best, results = B.gs_autotune(r.views, r.p.n, r.means2d, r.conics, r.p.opacities, r.p.colors, r.isect_ids,
                                  r.tile_ranges, r.K, r.cap, ws, candidates, repeats)
    del ws
    best["all"] = results
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cache[ck] = best
            json.dump(cache, open(path, "w"))
        except OSError:
            pass
    return dict(best, cached=False)


def config(tuning: dict, device="cuda") -> B.RasterConfig:
    """The RasterConfig of a tuning dict (from ``autotune``); the longest-first
    order is the renderer's own (``longest_first``)."""
    return B.RasterConfig(bool(tuning["persistent"]), int(tuning["ctas_per_sm"]), device=device,
                          bwd_pixels=int(tuning.get("bwd_pixels", 0)), bwd_batch=int(tuning.get("bwd_batch", 0)))


def workload_views(w, device="cuda"):
    """Params, Views and packed targets of a workloads.Workload (all scenes
    concatenated; view i renders its scene's Gaussian range)."""
    offs = np.cumsum([0] + [s.n for s in w.scenes])
    cat = lambda k: torch.as_tensor(np.concatenate([getattr(s, k) for s in w.scenes]), dtype=torch.float32,
                                    device=device).contiguous()
    params = Params(cat("means"), cat("quats"), cat("scales"), cat("opacities"), cat("colors"))
    ranges = [(int(offs[v.scene]), w.scenes[v.scene].n) for v in w.views]
    views = B.Views([v.camera for v in w.views], ranges, device=device)
    targets = None
    if w.targets is not None:
        targets = torch.as_tensor(np.concatenate([t.reshape(-1, 3) for t in w.targets]), device=device)
    return params, views, ranges, targets
