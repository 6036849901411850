#!/usr/bin/env python3
"""Benchmark of the differentiable Gaussian-splatting hot path on GB300.

One step = one pass of the whole path over one synthetic frame: projection,
binning + tile/depth sort, compositing, the L2-loss gradient, compositing
backward and projection backward -- for the 1,000,000-Gaussian 1920x1080
workload (64-component mixture, log-scales N(-4.5, 1), opacity
sigmoid(N(-1, 2)), seed 0; see paper_2312_02121_gb300/workloads.py).

Prints ONE JSON line.  ``value`` is fwd+bwd Mpixel/s over all ranks with the
inputs resident in HBM (CUDA events on the launching stream, L2 flushed by a
256 MiB write before every timed step, outside the step's events); ``e2e`` is
the same metric through the public autograd API with the parameters and the
target copied host->device from pinned memory every step and the loss read
back.  ``--impl reference`` times the FP64 CPU oracle instead (the reference
arm of this comparison; it has no published GPU numbers).

Multi-GPU (torchrun, N > 1): the 64 views of the 500,000-Gaussian scene are
split over the ranks (shard.plan), each rank replays its captured share of the
step, and one NCCL all-reduce sums the per-Gaussian gradients; timings are
max-reduced over ranks (strong scaling: the batch is fixed).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpixel/s at 1M Gaussians 1080p; batched vs per-view launches"
UNIT = "Mpixel/s"
WORKLOAD = "fwdbwd_1m_1080p"
SMS = 152
FP32_LANES_PER_SM = 128
# MUFU results per SM and clock, measured on GB300 by a throughput loop of independent chains:
# ex2.approx 32, rcp.approx 16 (FP32 FMA: 128, i.e. 77.6 TFLOP/s at the clocks seen)
MUFU_EX2_PER_SM_CLK = 32
MUFU_RCP_PER_SM_CLK = 16


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target duration of the oracle sample")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-per-view measurement")
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--no-optim", action="store_true", help="skip the optimisation-loop measurement")
    ap.add_argument("--optim-steps", type=int, default=20)
    ap.add_argument("--profile", action="store_true",
                    help="run warmup + steps untimed and exit (a fixed command line for ncu)")
    ap.add_argument("--profile-batch", choices=["batch_views_500k_64", "batch_scenes_16x4"], default=None,
                    help="with --profile: run that batched workload's step (BatchRenderer, eager) instead")
    ap.add_argument("--tuning", default=None,
                    help="persistent,ctas_per_sm,longest_first,bwd_pixels,bwd_batch instead of gs_autotune's "
                         "choice (e.g. for an ncu launch list without the tuner's launches)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []
        self.windows = []  # (start, end) wall-clock seconds of the timed regions

    def __enter__(self):
        try:
            # line-buffered where coreutils' stdbuf exists, so no sample is held back in a pipe buffer
            line_buf = ["stdbuf", "-oL"] if shutil.which("stdbuf") else []
            self.proc = subprocess.Popen(line_buf + ["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.QUERY}",
                                                     "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)  # the reader has taken every line the sampler wrote

    def mark(self, t0: float, t1: float):
        """Declares [t0, t1] (time.time()) a timed region: the clock median is taken over the
        samples nvidia-smi stamped inside these regions, when it stamped any."""
        self.windows.append((t0, t1))

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None  # "[N/A]" and the like

        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9 or num(f[1]) is None or num(f[2]) is None:
                continue  # a clock sample needs both clocks; power may be unavailable
            ts = None
            if len(f) > 9:
                try:
                    ts = datetime.datetime.strptime(f[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
            rows.append(dict(sm=num(f[1]), max=num(f[2]), power=num(f[3]), hw=f[5], hwt=f[6], swt=f[7], cap=f[8],
                             ts=ts))
        if not rows:
            return None
        # samples stamped inside a timed region (20 ms of slack for the sampling period)
        timed = [r for r in rows if r["ts"] is not None
                 and any(a - 0.02 <= r["ts"] <= b + 0.02 for a, b in self.windows)]
        scope = "timed region" if timed else "whole run (warm-up, timed steps and the pauses between)"
        rows = timed or rows
        powers = [r["power"] for r in rows if r["power"] is not None]
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("cap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "scope": scope,
                "power_w_max": max(powers) if powers else None}


RASTER_SOURCES = ("gs_raster.cu", "gs_raster_bwd.cuh", "gs_raster_bwd2.cu", "gs_raster_common.cuh", "gs_common.cuh")


def tuning_table(best: dict) -> dict:
    """gs_autotune's time of every candidate, keyed g/p (one CTA per tile / persistent grid) + CTAs per
    SM + I/L (tile id / longest-first order) + the backward's pixels per thread and batch."""
    return {f"{'p' if x['persistent'] else 'g'}{x['ctas_per_sm']}"
            f"{'L' if x['longest_first'] else 'I'}_{x['bwd_pixels']}px{x['bwd_batch']}": round(x["ms"], 3)
            for x in best["all"]}


def raster_source_hash() -> str:
    """sha256 over the sources the 3-channel raster kernels are compiled from."""
    import hashlib
    h = hashlib.sha256()
    for f in RASTER_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2312_02121_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, if it
    was captured from the current source of the raster kernels (else None)."""
    import hashlib
    try:
        h = raster_source_hash()
        for line in open(os.path.join(ROOT, "profiles", "roofline_traffic.txt")):
            f = line.split()
            if len(f) == 3 and not line.startswith("#") and f[0] == kernel and f[1] == h:
                return int(f[2])
    except OSError:
        pass
    return None


def walked_pairs(f, cam, dev) -> int:
    """(pixel, Gaussian) pairs the backward of Sec. 3.1 evaluates: for every pixel the entries of its
    tile's sorted list from the first through the pixel's last composited one (none when nothing was
    composited), counted exactly from last_idx and the tile ranges."""
    import torch
    W, H = cam.width, cam.height
    tx = (W + 15) // 16
    tile = ((torch.arange(H, device=dev).view(H, 1) // 16) * tx + torch.arange(W, device=dev).view(1, W) // 16)
    start = f.tile_ranges[tile.reshape(-1), 0].long()
    return int((f.last_idx.reshape(-1).long() - start + 1).clamp_min(0).sum().item())


def forward_walked_pairs(f, cam, params, dev, chunk: int = 64) -> int:
    """(pixel, Gaussian) pairs the forward of Eq. 7 evaluates: for every pixel the entries of its tile's
    sorted list from the first until the pixel stops -- at the first Gaussian after its last composited
    one that passes the alpha test (it would take T below 1e-4), else at the list's end.  Counted from
    last_idx and the tile ranges, with the stop found by walking the entries after last_idx (fp32, the
    kernel's test up to rounding at the threshold)."""
    import torch
    W, H = cam.width, cam.height
    tx = (W + 15) // 16
    tile = ((torch.arange(H, device=dev).view(H, 1) // 16) * tx + torch.arange(W, device=dev).view(1, W) // 16)
    rng_ = f.tile_ranges[tile.reshape(-1)].long()
    start, end = rng_[:, 0], rng_[:, 1]
    last = f.last_idx.reshape(-1).long()
    px = torch.arange(W, device=dev).repeat(H).float() + 0.5
    py = torch.arange(H, device=dev).repeat_interleave(W).float() + 0.5
    stop = end - 1  # pixels that never stop walk the whole list
    active = torch.nonzero(last + 1 < end).squeeze(1)
    pos = last + 1
    op = params.opacities
    while active.numel():
        offs = torch.arange(chunk, device=dev)
        idx = pos[active].view(-1, 1) + offs.view(1, -1)
        valid = idx < end[active].view(-1, 1)
        ids = f.isect_ids[idx.clamp_max(f.isect_ids.numel() - 1)].long()
        m2, cf = f.means2d[ids], f.conics[ids]
        dx = m2[..., 0] - px[active].view(-1, 1)
        dy = m2[..., 1] - py[active].view(-1, 1)
        u = dx + cf[..., 1] * dy
        sig = 0.5 * (cf[..., 0] * u * u + cf[..., 2] * dy * dy)
        taker = valid & (sig >= 0) & (op[ids] * torch.exp(-sig) >= 1.0 / 255.0)
        has = taker.any(dim=1)
        first = torch.argmax(taker.int(), dim=1)
        done = has | ~valid[:, -1]
        stop[active[has]] = pos[active[has]] + first[has]
        pos[active] += chunk
        active = active[~done]
    return int((stop - start + 1).clamp_min(0).sum().item())


def stage_rooflines(stage_ms: dict, P: int, K: int, pix: int, walked_fwd: int, walked_bwd: int, hbm: float,
                    fp32_peak: float, sm_mhz: float) -> dict:
    """Every stage of the step against the roofline that bounds it.  HBM stages: the bytes the method
    must move per unit over the stage's CUDA-event time, against the measured copy
    bandwidth.  Compositing: FP32 flops per evaluated pair (16 forward, 40 backward) against the FP32
    FMA peak at the maximum SM clock, with the SFU rate beside it."""
    out = {}

    def hbm_entry(stage, nbytes, work):
        t = stage_ms[stage] / 1e3
        a = nbytes / t / 1e9
        out[stage] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm, "work": work,
                      "ms": stage_ms[stage]}

    hbm_entry("project", P * 80.0, f"{P} projections x 80 B (44 B read, 36 B written)")
    hbm_entry("bin_and_sort", P * 80.0 + K * 60.0,
              f"{P} projections x 80 B (depth keys, 3 depth passes, scan) + {K} pairs x 60 B (emission, "
              f"2 tile passes, ranges)")
    hbm_entry("loss_grad", pix * 3 * 12.0, f"{pix} pixels x 3 channels x 12 B (image and target read, dL/dC written)")
    hbm_entry("project_bwd", P * 104.0, f"{P} projections x 104 B (64 B read, 40 B written)")
    for stage, pairs, flops in (("rasterize_fwd", walked_fwd, 16), ("rasterize_bwd", walked_bwd, 40)):
        t = stage_ms[stage] / 1e3
        a = pairs * flops / t / 1e12
        e = {"bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "TFLOP/s", "frac": a / fp32_peak,
             "work": f"{pairs} evaluated (pixel, Gaussian) pairs x {flops} FP32 flops", "ms": stage_ms[stage]}
        if stage == "rasterize_bwd":
            e["sfu"] = sfu_roof(pairs, t, sm_mhz)
        else:
            peak_ex2 = SMS * MUFU_EX2_PER_SM_CLK * sm_mhz * 1e6 / 1e9
            e["sfu"] = {"achieved": pairs / t / 1e9, "peak": peak_ex2, "unit": "Gpair/s",
                        "frac": pairs / t / 1e9 / peak_ex2, "note": "one ex2 (32 per SM clock) per evaluated pair"}
        out[stage] = e
    return out


def sfu_roof(pairs: int, seconds: float, sm_mhz: float) -> dict:
    """One ex2 and one reciprocal per evaluated pair against the measured MUFU rates."""
    clk_per_pair = 1.0 / MUFU_EX2_PER_SM_CLK + 1.0 / MUFU_RCP_PER_SM_CLK  # SM clocks per pair
    peak = SMS * sm_mhz * 1e6 / clk_per_pair / 1e9
    achieved = pairs / seconds / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "Gpair/s", "frac": achieved / peak,
            "note": "ex2 (32 per SM clock) + rcp (16 per SM clock) per evaluated pair"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def tile_sample(cam, n_tiles: int, seed: int = 0):
    """Every pixel of n_tiles seeded random 16x16 tiles (linear pixel ids)."""
    TX, TY = (cam.width + 15) // 16, (cam.height + 15) // 16
    rng = np.random.default_rng(seed)
    tiles = rng.choice(TX * TY, min(n_tiles, TX * TY), replace=False)
    pix = []
    for t in tiles:
        ty, tx = divmod(int(t), TX)
        ys = np.arange(ty * 16, min(ty * 16 + 16, cam.height))
        xs = np.arange(tx * 16, min(tx * 16 + 16, cam.width))
        pix.append((ys[:, None] * cam.width + xs[None, :]).ravel())
    return np.sort(np.concatenate(pix))


def oracle_step(oracle, w, pix):
    """The oracle's fwd+bwd of one view restricted to the sampled pixels."""
    cam, sc = w.views[0].camera, w.scenes[0]
    proj = oracle.project(cam, sc.means, sc.quats, sc.scales, w.eps2d)
    fwd = oracle.rasterize(proj, sc.opacities, sc.colors, cam.width, cam.height, pixels=pix)
    tgt = w.targets[0].reshape(-1, 3)[pix]
    G = 2.0 * (fwd["rgb"] - tgt) / (cam.pixels * 3)
    g2 = oracle.rasterize_bwd(proj, sc.opacities, sc.colors, cam.width, cam.height, G, pixels=pix)
    oracle.project_bwd(cam, sc.means, sc.quats, sc.scales, proj["valid"], g2["means2d"], g2["conics"], w.eps2d)


def sized_sample(oracle, w, seconds: float):
    """Tile count whose oracle step takes about ``seconds`` on this host: grows
    a seeded tile sample (x4 per probe) until a step takes at least half the
    target, then scales linearly; the whole frame at most."""
    cam = w.views[0].camera
    TX, TY = (cam.width + 15) // 16, (cam.height + 15) // 16
    n, dt = 16, 0.0
    while True:
        pix = tile_sample(cam, n)
        t0 = time.perf_counter()
        oracle_step(oracle, w, pix)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds or n >= TX * TY:
            break
        n = min(TX * TY, n * 4)
    return int(min(TX * TY, max(16, n * seconds / max(dt, 1e-3))))


def cpu_baseline(w, seconds: float):
    """Times the oracle as it stands on this host's cores over a tile sample
    sized to take about ``seconds``."""
    import oracle
    oracle.build()
    cam = w.views[0].camera
    n_tiles = sized_sample(oracle, w, seconds)
    pix = tile_sample(cam, n_tiles)
    t0 = time.perf_counter()
    oracle_step(oracle, w, pix)
    dt = time.perf_counter() - t0
    return {"value": len(pix) / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n_tiles} seeded random 16x16 tiles ({len(pix)} pixels, "
                      f"{100.0 * len(pix) / cam.pixels:.1f}% of the frame): full projection and projection "
                      f"backward of all {w.scenes[0].n} Gaussians, compositing fwd+bwd of the sampled pixels",
            "seconds": dt}


# ---------------------------------------------------------------------------
# the oracle leg (rank 0, one GPU): the oracle timed on the host cores, and the
# GPU results' error against it on the same pixels
# ---------------------------------------------------------------------------

def _proj_of(r, i, compare):
    """The CUDA projection of view i of a BatchRenderer, as an oracle projection dict."""
    hv = r.views.host[i]
    s_, e = hv.proj_offset, hv.proj_offset + hv.g_count
    n = lambda t: t[s_:e].detach().cpu().numpy()
    return dict(means2d=n(r.means2d).astype(np.float64), conics=compare.conic_from_factors(n(r.conics)),
                depths=n(r.depths).astype(np.float64), rects=n(r.rects).astype(np.int32),
                valid=(n(r.touched) > 0).astype(np.int32))


def oracle_accuracy(dev, w, frac: float, seed: int, tuning=None) -> dict:
    """The timed step (forward and fast backward of a BatchRenderer with the bench's walk) against the
    FP64 oracle on a seeded ``frac`` pixel subsample of every view (frac = 1: every pixel).  dL/dC is
    the L2 loss gradient of the oracle's image on those pixels, zero elsewhere and on pixels where
    fp32 and fp64 may composite differently end to end (threshold margin 1e-3, depth gap 1e-6, tile-box
    edges).  Reports the image max-abs error given the CUDA projection and end to end, and the
    relative L2 error of every per-Gaussian gradient summed over the views."""
    import torch
    import oracle
    from oracle import compare
    from paper_2312_02121_gb300 import batch as GB
    keys = ("means", "quats", "scales", "opacities", "colors")
    params, views, ranges, targets = GB.workload_views(w, dev)
    cap = GB.exact_capacity(params, views, w.eps2d)
    cfg = GB.config(tuning, dev) if tuning else None
    r = GB.BatchRenderer(params, views, cap, targets, w.eps2d, cfg, bool(tuning and tuning["longest_first"]))
    r.forward()
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    offs = np.cumsum([0] + [sc.n for sc in w.scenes])
    tot = {k: np.zeros((int(offs[-1]),) + np.shape(getattr(w.scenes[0], k))[1:]) for k in keys}
    G = torch.zeros(views.pixels, 3, device=dev)
    err_gp = err_e2e = 0.0
    excluded = sampled = 0
    t0 = time.perf_counter()
    for i, v in enumerate(w.views):
        cam, sc = v.camera, w.scenes[v.scene]
        pix = (np.arange(cam.pixels) if frac >= 1 else
               np.sort(rng.choice(cam.pixels, max(1, int(round(frac * cam.pixels))), replace=False)))
        off = views.host[i].pixel_offset
        img = r.rgb[off:off + cam.pixels].detach().cpu().numpy()[pix]
        ogp = oracle.rasterize(_proj_of(r, i, compare), sc.opacities, sc.colors, cam.width, cam.height, pixels=pix)
        ok = ogp["margin"] >= 1e-4
        err_gp = max(err_gp, float(np.abs(img - ogp["rgb"])[ok].max(initial=0.0)))
        fwd = oracle.render(cam, sc, w.eps2d, pixels=pix)
        bad = compare.uncertain_pixels(fwd["margin"], fwd["proj"], cam.width, cam.height, sc.opacities, pixels=pix,
                                       margin_rel=1e-3, depth_gap=fwd["depth_gap"])
        err_e2e = max(err_e2e, float(np.abs(img - fwd["rgb"])[~bad].max(initial=0.0)))
        tgt = np.asarray(w.targets[i], np.float64).reshape(-1, 3)[pix]
        Gv = np.where(bad[:, None], 0.0, 2.0 * (fwd["rgb"] - tgt) / (3 * w.pixels))
        ob = oracle.backward(cam, sc, Gv, w.eps2d, pixels=pix)
        for k in keys:
            tot[k][int(offs[v.scene]):int(offs[v.scene]) + sc.n] += ob[k]
        G[off + torch.as_tensor(pix, device=dev)] = torch.as_tensor(Gv, dtype=torch.float32, device=dev)
        excluded += int(bad.sum())
        sampled += len(pix)
    oracle_s = time.perf_counter() - t0
    r.dL.copy_(G)
    r.backward()
    torch.cuda.synchronize()
    got = r.grads()
    out = {"pixels": int(sampled), "fraction": frac, "excluded": excluded / max(sampled, 1),
           "image_max_abs_given_projection": err_gp, "image_max_abs_end_to_end": err_e2e,
           "grad_rel_l2": {k: compare.rel_l2(got[k].detach().cpu().numpy(), tot[k]) for k in keys},
           "oracle_seconds": oracle_s, "cores": oracle.num_threads(),
           "tolerances": {"image_given_projection": 1e-5, "image_end_to_end": 5e-4, "grad_rel_l2": 1e-4}}
    del r
    torch.cuda.empty_cache()
    return out


def small_configs(dev, steps: int = 50) -> dict:
    """The two small workloads, each timed on the GPU (one CUDA graph per step) and by the oracle in
    full on the host cores, with the GPU's error against the oracle: 1,000 Gaussians at 128x128
    (forward only) and 100,000 at 1024x768 (forward and backward of the L2 loss)."""
    import torch
    import oracle
    from oracle import compare
    from paper_2312_02121_gb300 import batch as GB
    from paper_2312_02121_gb300 import workloads as wl
    out = {}
    for name, make, backward in (("forward_1k_128", wl.forward_1k_128, False),
                                 ("fwdbwd_100k_1024x768", wl.fwdbwd_100k_1024x768, True)):
        w = make()
        cam, sc = w.views[0].camera, w.scenes[0]
        params, views, ranges, targets = GB.workload_views(w, dev)
        if targets is None:
            targets = torch.zeros(views.pixels, 3, device=dev)
        cap = GB.exact_capacity(params, views, w.eps2d)
        r = GB.BatchRenderer(params, views, cap, targets, w.eps2d)
        step = r.step_eager if backward else r.forward
        # one CUDA graph per step (forward alone for the forward-only workload)
        s_ = torch.cuda.Stream()
        s_.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s_):
            for _ in range(2):
                step()
        torch.cuda.current_stream().wait_stream(s_)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        assert not r.overflowed()
        # the oracle, whole image, timed
        t0 = time.perf_counter()
        fwd = oracle.render(cam, sc, w.eps2d)
        G = None
        if backward:
            tgt = np.asarray(w.targets[0], np.float64)
            G = 2.0 * (fwd["rgb"] - tgt) / fwd["rgb"].size
            ob = oracle.backward(cam, sc, G, w.eps2d)
        o_s = time.perf_counter() - t0
        e = {"gaussians": sc.n, "width": cam.width, "height": cam.height, "intersections": cap,
             "gpu": {"ms_per_step": ms, "mpix_s": views.pixels / ms / 1e3, "intersections_per_s": cap / (ms / 1e3),
                     "step": "fwd+bwd (L2 loss)" if backward else "forward", "cuda_graph": True},
             "oracle": {"seconds": o_s, "mpix_s": views.pixels / o_s / 1e6, "cores": oracle.num_threads(),
                        "sample": "the whole image"}}
        img = r.rgb.detach().cpu().numpy().reshape(cam.height, cam.width, 3)
        bad = compare.uncertain_pixels(fwd["margin"], fwd["proj"], cam.width, cam.height, sc.opacities,
                                       margin_rel=1e-3, depth_gap=fwd["depth_gap"])
        acc = {"image_max_abs_end_to_end": float(np.abs(img - fwd["rgb"])[~bad].max(initial=0.0)),
               "excluded": float(bad.mean())}
        if backward:
            Gm = np.where(bad[..., None], 0.0, G)
            ob = oracle.backward(cam, sc, Gm, w.eps2d)
            r.dL.copy_(torch.as_tensor(Gm.reshape(-1, 3), dtype=torch.float32, device=dev))
            r.backward()
            torch.cuda.synchronize()
            got = r.grads()
            acc["grad_rel_l2"] = {k: compare.rel_l2(got[k].detach().cpu().numpy(), ob[k]) for k in got}
        e["accuracy"] = acc
        out[name] = e
        del r, g
        torch.cuda.empty_cache()
    return out


def batched_comparison(dev, steps: int):
    """The two multi-view workloads: one autotuned, graph-captured batched step
    (one launch per stage over all views) against the same kernels launched
    once per view; same loss, same results (gradients compared below)."""
    import torch
    from paper_2312_02121_gb300 import batch as GB
    from paper_2312_02121_gb300 import binding as B
    from paper_2312_02121_gb300 import workloads as wl
    out = {}
    for name, make in (("batch_views_500k_64", wl.batch_views_500k_64), ("batch_scenes_16x4", wl.batch_scenes_16x4)):
        w = make()
        params, views, ranges, targets = GB.workload_views(w, dev)
        cap = GB.exact_capacity(params, views, w.eps2d)

        def mk(c):
            return GB.BatchRenderer(params, views, cap, targets, w.eps2d, GB.config(c, dev), bool(c["longest_first"]))

        # the library's autotuner (gs_autotune) picks the tile walk and the backward batch shape
        best = GB.autotune(GB.BatchRenderer(params, views, cap, targets, w.eps2d),
                           key=f"{name}|P{views.P}|T{views.T}|K{cap}", use_cache=False)
        r = mk(best)
        r.capture()
        l0 = B.gs_kernel_launches()
        r.step_eager()
        launches_b = B.gs_kernel_launches() - l0
        ms_b = GB.time_steps(r.step, n=steps)
        assert not r.overflowed()
        caps = GB.per_view_capacities(params, [v.camera for v in w.views], ranges, w.eps2d)
        pv = GB.PerViewRenderer(params, [v.camera for v in w.views], ranges, caps, targets, w.eps2d)
        l0 = B.gs_kernel_launches()
        pv.step()
        launches_v = B.gs_kernel_launches() - l0
        ms_v = GB.time_steps(pv.step, n=steps)
        r.step()
        torch.cuda.synchronize()
        same_images = bool(torch.equal(r.rgb, torch.cat([x.rgb for x in pv.r])))
        rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b).clamp_min(1e-30))
        # per-projection 2D gradients (well conditioned) in the timed, atomic mode
        agree_2d = max(rel(r.g2, torch.cat([x.g2 for x in pv.r])), rel(r.gc, torch.cat([x.gc for x in pv.r])))
        del pv
        torch.cuda.empty_cache()
        # every gradient with the summation order fixed (deterministic mode): must be identical
        rd = GB.BatchRenderer(params, views, cap, targets, w.eps2d, deterministic=True)
        rd.step_eager()
        pvd = GB.PerViewRenderer(params, [v.camera for v in w.views], ranges, caps, targets, w.eps2d,
                                 deterministic=True)
        pvd.step()
        torch.cuda.synchronize()
        gb, gv = rd.grads(), pvd.grads()
        agree_det = max(rel(gb[k], gv[k]) for k in gb)
        del rd, pvd
        out[name] = {"views": views.V, "scenes": len(w.scenes), "gaussians": params.n, "pixels": views.pixels,
                     "intersections": cap, "batched_mpix_s": views.pixels / ms_b / 1e3,
                     "batched_intersections_per_s": cap / (ms_b / 1e3),
                     "per_view_mpix_s": views.pixels / ms_v / 1e3, "speedup": ms_v / ms_b,
                     "batched_ms_per_step": ms_b, "per_view_ms_per_step": ms_v,
                     "batched_launches_per_step": int(launches_b), "per_view_launches_per_step": int(launches_v),
                     "batched_cuda_graph": True,
                     "tuning": {k: best[k] for k in B.TUNING_FIELDS},
                     "tuning_ms": tuning_table(best),
                     "tuning_note": "compositing fwd+bwd ms per candidate (gs_autotune): g/p = one CTA per tile / "
                                    "persistent grid (CTAs per SM, 0 = as many as fit), I/L = tile id / longest-first "
                                    "order, then the backward's pixels per thread and staged batch",
                     "images_identical": same_images, "grad2d_rel_l2_batched_vs_per_view": agree_2d,
                     "grad_rel_l2_batched_vs_per_view_deterministic": agree_det,
                     "l2": "inputs larger than L2"}
        del r, params, views, targets
        torch.cuda.empty_cache()
    return out


def optimisation_loop(dev, w, steps: int):
    """The graph-captured training step (forward, fused L2 loss, backward, fused
    Adam on the raw parameters) on the headline workload, from its scene toward
    its target image."""
    import numpy as np
    import torch
    from paper_2312_02121_gb300 import binding as B
    from paper_2312_02121_gb300.train import Trainer
    cam, sc = w.views[0].camera, w.scenes[0]
    o = np.clip(np.asarray(sc.opacities, np.float64), 1e-6, 1 - 1e-6)
    raw = {"means": sc.means, "quats": sc.quats, "log_scales": np.log(sc.scales),
           "opacity_logits": np.log(o / (1 - o)), "colors": sc.colors}
    raw = {k: torch.as_tensor(np.asarray(v, np.float32), device=dev).contiguous() for k, v in raw.items()}
    views = B.Views([cam], [(0, sc.n)], device=dev)
    tgt = torch.as_tensor(w.targets[0].reshape(-1, 3), device=dev)
    t = Trainer(raw, views, tgt)
    t.capture()
    t.step()
    torch.cuda.synchronize()
    loss0 = t.loss()
    l0 = B.gs_kernel_launches()
    t.step_eager()
    launches = B.gs_kernel_launches() - l0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        t.step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out = {"ms_per_step": ms, "mpix_s": views.pixels / ms / 1e3, "steps": steps, "cuda_graph": True,
           "gpu_launches_per_step": int(launches), "loss_first": loss0, "loss_last": t.loss(),
           "adam_steps_applied": t.steps_taken(), "overflowed": t.overflowed(), "capacity": t.capacity,
           "l2": "inputs larger than L2 (params, moments, target: > 129 MB)"}
    del t
    torch.cuda.empty_cache()
    return out


def channel_cost(dev, views, params, pr, frame_ids, tile_ranges, K, cap, eps2d: float,
                 channels=(1, 3, 4, 8, 12, 16, 32),
                 steps: int = 10):
    """Device time of compositing forward + backward on the headline frame for
    several channel counts (same projection and sorted lists)."""
    import torch
    from paper_2312_02121_gb300 import binding as B
    N, pix = params.n, views.pixels
    out = {}
    for C in channels:
        col = torch.rand(N, C, device=dev)
        rgb, Tf = torch.empty(pix, C, device=dev), torch.empty(pix, device=dev)
        last = torch.empty(pix, dtype=torch.int32, device=dev)
        G = torch.randn(pix, C, device=dev)
        g2, gc = torch.zeros(views.P, 2, device=dev), torch.zeros(views.P, 3, device=dev)
        go, gcol = torch.zeros(N, device=dev), torch.zeros(N, C, device=dev)

        def once():
            B.gs_rasterize_fwd_nc(views, C, pr["means2d"], pr["conics"], params.opacities, col, frame_ids,
                                  tile_ranges, None, rgb, Tf, last)
            B.gs_rasterize_bwd_nc(views, C, pr["means2d"], pr["conics"], params.opacities, col, frame_ids,
                                  tile_ranges, None, Tf, last, G, g2, gc, go, gcol)
        for _ in range(2):
            once()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            once()
        b.record()
        torch.cuda.synchronize()
        out[str(C)] = {"fwd_bwd_ms": a.elapsed_time(b) / steps}
        del col, rgb, Tf, last, G, g2, gc, go, gcol
    return out


def view_gradient_cost(dev, views, params, pr, g2, gc, eps2d: float, steps: int = 20):
    """Device time of the projection backward with and without the per-view
    dL/dT_cw output."""
    import torch
    from paper_2312_02121_gb300 import binding as B
    N = params.n
    z = lambda *shape: torch.zeros(*shape, device=dev)
    gm, gq, gs, gv = z(N, 3), z(N, 4), z(N, 3), z(views.V, 4, 4)
    res = {}
    for name, vm in (("plain", None), ("with_viewmats", gv)):
        for _ in range(3):
            B.gs_project_bwd(views, params.means, params.quats, params.scales, eps2d, pr["touched"], g2, gc, gm, gq,
                             gs, None, vm)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            B.gs_project_bwd(views, params.means, params.quats, params.scales, eps2d, pr["touched"], g2, gc, gm, gq,
                             gs, None, vm)
        b.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = a.elapsed_time(b) / steps
    return res


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_2312_02121_gb300 import workloads as wl
    oracle.build()
    w = wl.fwdbwd_1m_1080p(seed=0)
    cam = w.views[0].camera
    # size each step so the whole run stays within a few minutes
    per_step = max(2.0, min(8.0, 150.0 / max(args.steps + args.warmup, 1)))
    n_tiles = sized_sample(oracle, w, per_step)
    pix = tile_sample(cam, n_tiles)
    for _ in range(args.warmup):
        oracle_step(oracle, w, pix)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(oracle, w, pix)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = len(pix) / (ms / 1e3) / 1e6
    sample = (f"{n_tiles} seeded random 16x16 tiles ({len(pix)} pixels) of the 1920x1080 frame per step; "
              f"projection and its backward over all {w.scenes[0].n} Gaussians")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": w.scenes[0].n, "width": cam.width, "height": cam.height,
                   "pixels_per_step": int(len(pix))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_profile_batch(args):
    """--profile --profile-batch W: warm-up + steps of the batched workload W's step (the batch renderer,
    eagerly, every stage in its own launches), untimed: a fixed command line for ncu."""
    import torch
    from paper_2312_02121_gb300 import batch as GB
    from paper_2312_02121_gb300 import binding as B
    from paper_2312_02121_gb300 import workloads as wl
    B.load()
    w = getattr(wl, args.profile_batch)()
    params, views, ranges, targets = GB.workload_views(w, "cuda")
    cap = GB.exact_capacity(params, views, w.eps2d)
    t = (dict(zip(B.TUNING_FIELDS, (int(x) for x in args.tuning.split(",")))) if args.tuning else
         dict(persistent=0, ctas_per_sm=0, longest_first=0, bwd_pixels=2, bwd_batch=64))
    r = GB.BatchRenderer(params, views, cap, targets, w.eps2d, GB.config(t, "cuda"), bool(t["longest_first"]))
    for _ in range(args.warmup + args.steps):
        r.step_eager()
    torch.cuda.synchronize()
    assert not r.overflowed()


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2312_02121_gb300 import autograd as ga
    from paper_2312_02121_gb300 import binding as B
    from paper_2312_02121_gb300 import pipeline
    from paper_2312_02121_gb300 import workloads as wl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B.load()
    w = wl.fwdbwd_1m_1080p(seed=0)
    cam, sc = w.views[0].camera, w.scenes[0]
    params = pipeline.Params.from_scene(sc, dev)
    target = torch.as_tensor(w.targets[0].reshape(-1, 3), device=dev)
    views = B.Views([cam], [(0, sc.n)], device=dev)
    pixels = views.pixels
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # exact intersection capacity (the workload is fixed), so steps never sync
    f0 = pipeline.forward(views, params, w.eps2d, count_contrib=True)
    K = int(f0.K_total.item())
    contrib = int(f0.n_contrib.sum().item())
    walked = walked_pairs(f0, cam, dev)
    walked_fwd = forward_walked_pairs(f0, cam, params, dev)
    cap = K
    del f0
    from paper_2312_02121_gb300 import batch as GB
    # the library's autotuner (gs_autotune) picks the tile walk and the backward's batch shape for this frame;
    # every timed path below uses its choice
    if args.tuning:
        tuning = dict(zip(B.TUNING_FIELDS, (int(x) for x in args.tuning.split(","))), ms=float("nan"))
    else:
        tuning = GB.autotune(GB.BatchRenderer(params, views, cap, target, w.eps2d),
                             key=f"{WORKLOAD}|P{views.P}|T{views.T}|K{cap}", use_cache=False)
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    stages = ["project", "bin_and_sort", "rasterize_fwd", "loss_grad", "zero_grads", "rasterize_bwd", "project_bwd"]
    last_state = {}
    # the forward hands its per-pair warp-box cull to the backward through this buffer
    order_buf = torch.empty(views.T, dtype=torch.int32, device=dev) if tuning["longest_first"] else None
    order_ws = (torch.empty(max(B.gs_tile_order_workspace_size(views.T), 1), dtype=torch.uint8, device=dev)
                if tuning["longest_first"] else None)
    hits_cfg = B.RasterConfig(bool(tuning["persistent"]), int(tuning["ctas_per_sm"]), order_buf, device=dev,
                              warp_hits=torch.empty(cap, dtype=torch.int32, device=dev),
                              bwd_pixels=int(tuning["bwd_pixels"]), bwd_batch=int(tuning["bwd_batch"]))

    def step(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        pr = pipeline.project(views, params, w.eps2d)
        mark(1)
        P, T = views.P, views.T
        ws = torch.empty(B.gs_bin_and_sort_workspace_size(P, cap, T), dtype=torch.uint8, device=dev)
        ids = torch.empty(cap, dtype=torch.int32, device=dev)
        tr = torch.empty(T, 2, dtype=torch.int32, device=dev)
        Kd = torch.empty(1, dtype=torch.int32, device=dev)
        fl = torch.zeros(1, dtype=torch.int32, device=dev)
        B.gs_bin_and_sort(views, pr["rects"], pr["depths"], pr["touched"], cap, ws, ids, None, None, tr, Kd, fl)
        mark(2)
        rgb = torch.empty(pixels, 3, device=dev)
        Tf = torch.empty(pixels, device=dev)
        last = torch.empty(pixels, dtype=torch.int32, device=dev)
        if order_buf is not None:
            B.gs_tile_order(tr, views.T, order_ws, order_buf)
        B.gs_rasterize_fwd(views, pr["means2d"], pr["conics"], params.opacities, params.colors, ids, tr, None, rgb,
                           Tf, last, None, hits_cfg)
        mark(3)
        dL = torch.empty(pixels, 3, device=dev)
        B.gs_l2_loss(rgb, target, 1.0 / rgb.numel(), dL, None)
        mark(4)
        # the accumulated gradients in one allocation, zeroed by one fill; one view, so the projection
        # backward writes the 3D gradients (gs_project_bwd_exclusive) and they need no fill
        N = sc.n
        gz = torch.zeros(5 * P + 4 * N, device=dev)
        g2, gc = gz[:2 * P].view(P, 2), gz[2 * P:5 * P].view(P, 3)
        go, gcol = gz[5 * P:5 * P + N], gz[5 * P + N:5 * P + 4 * N].view(N, 3)
        gm, gq, gs = (torch.empty(N, k, device=dev) for k in (3, 4, 3))
        mark(5)
        B.gs_rasterize_bwd(views, pr["means2d"], pr["conics"], params.opacities, params.colors, ids, None, None,
                           pr["touched"], tr, Kd, cap, None, Tf, last, dL, False, None, g2, gc, go, gcol, hits_cfg)
        mark(6)
        B.gs_project_bwd_exclusive(views, params.means, params.quats, params.scales, w.eps2d, pr["touched"], g2, gc,
                                   gm, gq, gs)
        mark(7)
        last_state.update(pr=pr, g2=g2, gc=gc, ids=ids, tr=tr, Kd=Kd)
        return fl

    if args.profile:
        for _ in range(args.warmup + args.steps):
            step()
        torch.cuda.synchronize()
        return
    def barrier():
        if world > 1:
            torch.distributed.barrier()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)  # let the sampler start; it covers warm-up and the timed steps
        for _ in range(max(args.warmup, 3)):
            fl = step()
        torch.cuda.synchronize()
        assert int(fl.item()) == 0, "intersection capacity overflow"
        launches0 = B.gs_kernel_launches()
        barrier()
        torch.cuda.synchronize()
        wall0, tw0 = time.perf_counter(), time.time()
        for k in range(args.steps):
            flush.zero_()
            step(evs[k])
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark(tw0, time.time())
        # kernels per instrumented eager step (the captured step below counts its own)
        launches = (B.gs_kernel_launches() - launches0) // max(args.steps, 1)
        barrier()
        # the same step captured once into a CUDA graph (BatchRenderer), as a training loop runs it:
        # this is the timed headline; the instrumented eager steps above give the per-stage split
        rgraph = GB.BatchRenderer(params, views, cap, target, w.eps2d, GB.config(tuning, dev),
                                  bool(tuning["longest_first"]))
        # the kernels one replay launches: those of one eager step of the same renderer
        l_g0 = B.gs_kernel_launches()
        rgraph.step_eager()
        launches = B.gs_kernel_launches() - l_g0
        rgraph.capture()
        for _ in range(max(args.warmup, 3)):
            rgraph.step()
        torch.cuda.synchronize()
        assert not rgraph.overflowed()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        tw0 = time.time()
        for a, b in gev:
            flush.zero_()
            a.record(stream)
            rgraph.step()
            b.record(stream)
        torch.cuda.synchronize()
        clk.mark(tw0, time.time())
        barrier()
        graph_ms = sum(a.elapsed_time(b) for a, b in gev) / args.steps
        del rgraph
    stage_ms = {s: 0.0 for s in stages}
    total_ms = 0.0
    for ev in evs:
        for i, s in enumerate(stages):
            stage_ms[s] += ev[i].elapsed_time(ev[i + 1])
        total_ms += ev[0].elapsed_time(ev[-1])
    eager_ms = total_ms / args.steps
    stage_ms = {s: v / args.steps for s, v in stage_ms.items()}
    ms_step = graph_ms
    if world > 1:
        t = torch.tensor([ms_step, eager_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step, eager_ms = float(t[0].item()), float(t[1].item())
    value = world * pixels / (ms_step / 1e3) / 1e6

    # --- end to end from host buffers: every step copies the Gaussian parameters and the target image
    # from pinned host memory, runs the whole step and reads the loss back into pinned host memory.
    # Headline path: a BatchRenderer with attached host inputs, captured once into a CUDA graph (the
    # copies of what compositing and the loss read overlap projection and sorting on a second stream).
    # Also reported: the same step through the autograd API (render + l2_loss + backward).
    from paper_2312_02121_gb300 import batch as GB
    keys = ("means", "quats", "scales", "opacities", "colors")
    host = {k: torch.as_tensor(getattr(sc, k)).pin_memory() for k in keys}
    host_tgt = torch.as_tensor(w.targets[0]).reshape(-1, 3).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + host_tgt.numel() * host_tgt.element_size()
    dev_params = pipeline.Params(*[torch.empty_like(host[k], device=dev) for k in keys])
    rg = GB.BatchRenderer(dev_params, views, cap, torch.empty_like(host_tgt, device=dev), w.eps2d,
                          GB.config(tuning, dev), bool(tuning["longest_first"]))
    rg.attach_host_inputs(host, host_tgt)
    rg.capture()

    def e2e_graph_step():
        rg.step()
        torch.cuda.current_stream().synchronize()
        return float(rg.loss_host[0])

    dev_bufs = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    dev_tgt = torch.empty_like(host_tgt, device=dev)

    def e2e_autograd_step():
        for k, v in host.items():
            dev_bufs[k].copy_(v, non_blocking=True)
        dev_tgt.copy_(host_tgt, non_blocking=True)
        v = B.Views([cam], [(0, sc.n)], device=dev)
        leaves = {k: t.detach().requires_grad_(True) for k, t in dev_bufs.items()}
        img = ga.render(leaves["means"], leaves["quats"], leaves["scales"], leaves["opacities"], leaves["colors"],
                        None, eps2d=w.eps2d, K_capacity=cap, views=v)[0]
        loss = ga.l2_loss(img, dev_tgt.view(img.shape))
        loss.backward()
        return float(loss.item())

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fn()
        dt = (time.perf_counter() - t0) / args.e2e_steps
        if world > 1:
            t = torch.tensor([dt], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        return dt

    e2e_serial_s = timed(e2e_graph_step)
    e2e_ag_s = timed(e2e_autograd_step)
    assert not rg.overflowed()
    del rg
    torch.cuda.empty_cache()

    # the headline end-to-end path: the same captured step, two deep (batch.HostPipeline): step k's copies
    # and compute overlap step k-1's on a second stream; every step copies its own inputs and reads back
    # its own loss
    def make_host_renderer():
        dp = pipeline.Params(*[torch.empty_like(host[k], device=dev) for k in keys])
        r = GB.BatchRenderer(dp, views, cap, torch.empty_like(host_tgt, device=dev), w.eps2d, GB.config(tuning, dev),
                             bool(tuning["longest_first"]))
        r.attach_host_inputs(host, host_tgt)
        return r

    pipe = GB.HostPipeline(make_host_renderer)
    for _ in range(3):
        pipe.step()
    pipe.finish()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        pipe.step()
    pipe.finish()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert not pipe.overflowed()
    del pipe
    torch.cuda.empty_cache()
    e2e = {"value": world * pixels / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": 4, "ms_per_step": 1e3 * e2e_s,
           "inputs": "per step: Gaussian parameters and target image (pinned host -> device); result: the loss "
                     "(device -> pinned host)",
           "api": "batch.HostPipeline: BatchRenderer.attach_host_inputs + capture, two steps in flight on two "
                  "streams (each step's copies and compute overlap the previous step's)",
           "serial": {"value": world * pixels / e2e_serial_s / 1e6, "ms_per_step": 1e3 * e2e_serial_s,
                      "api": "one captured step at a time: copies, step, loss read back, then the next"},
           "autograd_api": {"value": world * pixels / e2e_ag_s / 1e6, "ms_per_step": 1e3 * e2e_ag_s,
                            "api": "autograd.render + autograd.l2_loss + backward, views laid out per step"}}

    if rank != 0:
        return
    # --- roofline of the dominant kernel
    peaks, src = measured_peaks()
    clocks = clk.summary()
    dom = max(("rasterize_fwd", "rasterize_bwd", "bin_and_sort", "project", "project_bwd"), key=lambda s: stage_ms[s])
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2 flops
    # every stage against its roofline; the dominant one is the line's `roofline`
    stages_roof = stage_rooflines(stage_ms, views.P, K, pixels, walked_fwd, walked, peaks["hbm_gbs"], fp32_peak,
                                  sm_mhz)
    roof = dict(stages_roof[dom], kernel=dom)
    roof["peak_source"] = (f"FP32 FMA lanes: {SMS} SMs x {FP32_LANES_PER_SM} x 2 x {sm_mhz:.0f} MHz (max SM clock, "
                           f"{src})" if roof["bound"] == "alu" else f"hbm_gbs ({src})")
    roof["launch_ms"] = stage_ms[dom]
    roof["traffic"] = recorded_traffic({"rasterize_bwd": "k_raster_bwd", "rasterize_fwd": "k_raster_fwd"}.get(dom, ""))
    if dom in ("rasterize_fwd", "rasterize_bwd"):
        # the stricter count over composited pairs only (20 / 49 flops each) rides along
        fl = {"rasterize_fwd": 20, "rasterize_bwd": 49}[dom]
        strict = contrib * fl / 1e12 / (stage_ms[dom] / 1e3)
        roof["composited_only"] = {"achieved": strict, "frac": strict / fp32_peak,
                                   "work": f"{contrib} composited pairs x {fl} flops"}
    roof["stages"] = stages_roof

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": sc.n, "width": cam.width, "height": cam.height,
                   "views": 1, "intersections": K, "intersections_per_s": K / (ms_step / 1e3),
                   "composited_pairs": contrib, "evaluated_pairs_bwd": walked, "evaluated_pairs_fwd": walked_fwd,
                   "tuning": {k: tuning[k] for k in B.TUNING_FIELDS}, "tuning_ms": tuning["ms"],
                   "tuning_candidates_ms": tuning_table(tuning) if "all" in tuning else None,
                   "l2": "flushed (256 MiB write) before every timed step, outside its events",
                   "multi_gpu": "under torchrun the 64-view batch is split over the ranks instead (run_sharded)"},
        "stage_ms": stage_ms, "eager_ms_per_step": eager_ms,
        "timing": "ms_per_step: the step captured once into a CUDA graph and replayed (BatchRenderer, whose "
                  "forward kernel also takes the L2 loss and dL/dC: gs_rasterize_fwd_l2); stage_ms and "
                  "eager_ms_per_step: the same stages launched eagerly with an event between them, the loss as "
                  "its own kernel (gs_l2_loss)", "wall_s": wall,
        # kernels of ours launched in the timed region: each of the replayed steps launches the step's kernels
        "gpu_launches": int(launches) * args.steps, "gpu_launches_per_step": int(launches),
        "e2e": e2e, "roofline": roof, "clocks": clocks,
    }
    line["project_bwd_view_gradient"] = view_gradient_cost(dev, views, params, last_state["pr"], last_state["g2"],
                                                           last_state["gc"], w.eps2d)
    line["channels"] = channel_cost(dev, views, params, last_state["pr"], last_state["ids"], last_state["tr"],
                                    last_state["Kd"], cap, w.eps2d)
    if not args.no_optim:
        line["optimisation_loop"] = optimisation_loop(dev, w, args.optim_steps)
    if not args.no_batched:
        line["batched"] = batched_comparison(dev, args.batched_steps)
    if not args.no_cpu_baseline and world == 1:
        # the oracle leg: the oracle timed on the host cores, and the GPU results' error against it
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        acc = {"fwdbwd_1m_1080p": oracle_accuracy(dev, w, 1.0, 21, tuning)}
        if not args.no_batched:
            t16 = line["batched"]["batch_scenes_16x4"]["tuning"]
            acc["batch_scenes_16x4"] = oracle_accuracy(dev, wl.batch_scenes_16x4(), 0.01, 22, t16)
        line["accuracy"] = acc
        line["small_configs"] = small_configs(dev)
    print(json.dumps(line), flush=True)


def sharded_plan(world: int):
    """The view split of the multi-GPU mode: the 64 views of the 500,000-Gaussian scene (their pixel
    counts as costs) over ``world`` ranks by shard.plan (longest processing time first)."""
    from paper_2312_02121_gb300 import shard
    from paper_2312_02121_gb300 import workloads as wl
    w = wl.batch_views_500k_64()
    return w, shard.plan([v.scene for v in w.views], [v.camera.pixels for v in w.views], world)


def timed_sharded_steps(step, allreduce, steps: int, warmup: int, world: int, flush=None, dev=None):
    """Device time of ``steps`` sharded steps (the local step, then the gradient all-reduce when the split
    needs it), max over ranks, in ms per step.  ``step`` and ``allreduce`` are callables; events bracket
    each step on the current stream."""
    import torch
    for _ in range(max(warmup, 3)):
        step()
        allreduce()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        allreduce()
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    ms = total / steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms


def run_sharded(args, rank, world, local_rank):
    """--gpus N > 1: the multi-view workload split over the ranks as the sharding design has it.  The 64
    views of one 500,000-Gaussian scene go to the ranks by shard.plan; each rank renders its views with
    one captured BatchRenderer step into a flat per-Gaussian gradient buffer, and one NCCL all-reduce sums
    the buffers (the views share the scene, so its gradients are summed over views: Sec. 3.2).  The total
    work is fixed (strong scaling); value = all 64 views' pixels per second of the slowest rank."""
    import torch
    from paper_2312_02121_gb300 import batch as GB
    from paper_2312_02121_gb300 import binding as B
    from paper_2312_02121_gb300 import shard
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B.load()
    w, plan = sharded_plan(world)
    params, views_all, ranges, targets = GB.workload_views(w, dev)
    cams = [v.camera for v in w.views]
    sr = shard.ShardedRenderer(params, cams, ranges, [v.scene for v in w.views], targets, world, rank)
    sr.capture()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    allreduce = (lambda: sr.buf.allreduce()) if sr.plan.needs_allreduce else (lambda: None)
    l0 = B.gs_kernel_launches()
    sr.local_step()
    launches = B.gs_kernel_launches() - l0  # the local step's eager launch count (the graph replays them)
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        t0 = time.time()
        ms = timed_sharded_steps(sr.local_step, allreduce, args.steps, args.warmup, world, flush, dev)
        clk.mark(t0, time.time())
    assert not sr.overflowed()
    # end to end: the parameters and this rank's targets from pinned host memory every step, the loss back
    keys = ("means", "quats", "scales", "opacities", "colors")
    host = {k: getattr(params, k).cpu().pin_memory() for k in keys}
    mine_t = sr.r.targets.cpu().pin_memory() if sr.r is not None else None
    if sr.r is not None:
        sr.r.attach_host_inputs(host, mine_t)
        sr.r.graph = None
        sr.capture()

    def e2e_step():
        sr.local_step()
        allreduce()
        torch.cuda.current_stream().synchronize()
        return float(sr.r.loss_host[0]) if sr.r is not None else 0.0

    for _ in range(3):
        e2e_step()
    torch.distributed.barrier()
    t1 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    dt = torch.tensor([(time.perf_counter() - t1) / args.e2e_steps], device=dev)
    torch.distributed.all_reduce(dt, op=torch.distributed.ReduceOp.MAX)
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + (mine_t.numel() * 4 if mine_t is not None else 0)
    pixels = views_all.pixels
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": pixels / ms / 1e3, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch_views_500k_64", "views": len(w.views), "gaussians": params.n, "pixels": pixels,
                   "split": "views over ranks by shard.plan (LPT on pixels), every rank holds the whole scene",
                   "views_per_rank": [len(v) for v in plan.views_of_rank],
                   "allreduce_bytes": int(sr.buf.flat.numel() * 4) if plan.needs_allreduce else 0,
                   "l2": "flushed (256 MiB write) before every timed step, outside its events"},
        "gpu_launches": int(launches) * args.steps, "gpu_launches_per_step": int(launches),
        "timing": "each rank replays its captured local step, then the NCCL all-reduce of the gradient buffer; "
                  "max over ranks",
        "e2e": {"value": pixels / float(dt.item()) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": 4, "ms_per_step": 1e3 * float(dt.item()),
                "inputs": "per rank and step: the scene's parameters and the rank's targets (pinned host -> "
                          "device); result: the rank's loss (device -> pinned host)"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.profile and args.profile_batch:
            run_profile_batch(args)
        elif world > 1:
            run_sharded(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
