"""A synthetic optimisation loop: Adam on the raw Gaussian parameters toward
target images.

Every part of a step runs in the library's kernels, on the device, with
fixed-size buffers: projection, binning and sort, compositing, the L2 loss and
its gradient, compositing and projection backward, and the fused Adam update.
The update works on the raw parameters (log-scales, opacity logits) and
rewrites the activated scales and opacities the next forward reads.  So the
whole step can be captured once into a CUDA graph and replayed.

The intersection capacity is fixed when the buffers are made, while
optimisation moves the Gaussians.  A step whose pairs overflow the capacity
raises the binning flag, and the Adam kernel then skips that step, so no
update is ever made from incomplete gradients.  ``run`` checks the flag every
``check_every`` steps and rebuilds with more room when it was raised.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import torch

from . import binding as B
from .batch import BatchRenderer, exact_capacity
from .pipeline import Params

RAW = ("means", "quats", "log_scales", "opacity_logits", "colors")


class Trainer:
    def __init__(self, raw: Dict[str, torch.Tensor], views: B.Views, targets: torch.Tensor,
                 lr: Sequence[float] = (1.6e-4, 1e-3, 5e-3, 5e-2, 2.5e-3), betas=(0.9, 0.999), eps: float = 1e-15,
                 eps2d: float = 0.3, K_capacity: Optional[int] = None, headroom: float = 1.5,
                 config: Optional[B.RasterConfig] = None):
        """``raw``: device fp32 tensors means [N,3], quats [N,4], log_scales [N,3],
        opacity_logits [N], colors [N,C]; they are updated in place.
        ``targets``: packed [pixels, C] target images of ``views``.
        ``lr``: learning rates of the five groups, in that order."""
        for k in RAW:
            t = raw[k]
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"{k} must be a contiguous float32 CUDA tensor")
        self.raw = raw
        self.views, self.targets, self.eps2d, self.config = views, targets, eps2d, config
        self.N = int(raw["means"].shape[0])
        dev = raw["means"].device
        self.scales = torch.empty(max(self.N, 1), 3, device=dev)
        self.opacities = torch.empty(max(self.N, 1), device=dev)
        B.gs_activate(self.N, raw["log_scales"], raw["opacity_logits"], self.scales, self.opacities)
        self.params = Params(raw["means"], raw["quats"], self.scales[:self.N], self.opacities[:self.N], raw["colors"])
        self.adam = B.adam_config(lr, betas[0], betas[1], eps)
        self.state = torch.zeros(B.gs_adam_state_size(self.N, self.params.channels), dtype=torch.uint8, device=dev)
        self.headroom = headroom
        if K_capacity is None:
            K_capacity = int(headroom * exact_capacity(self.params, views, eps2d)) + 1024
        self._make(K_capacity)

    def _make(self, cap: int):
        self.r = BatchRenderer(self.params, self.views, cap, self.targets, self.eps2d, self.config)
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    @property
    def capacity(self) -> int:
        return self.r.cap

    def step_eager(self):
        r = self.r
        r.step_eager()
        B.gs_adam_step(self.N, self.adam, self.state, self.raw["means"], self.raw["quats"], self.raw["log_scales"],
                       self.raw["opacity_logits"], self.raw["colors"], r.g_means, r.g_quats, r.g_scales, r.g_op,
                       r.g_col, self.scales, self.opacities, r.flags)

    def capture(self):
        """Captures one step into a CUDA graph.  Graph capture needs warm-up
        launches first: the two eager steps taken here are real optimisation
        steps."""
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
        return self.r.overflowed()

    def loss(self) -> float:
        """The loss of the last step's forward (one device read)."""
        return float(self.r.loss.item())

    def state_dict(self) -> Dict[str, torch.Tensor]:
        """Host copies of everything a later run resumes from: the raw
        parameters, the Adam state (both moments and the count of applied
        steps) and the Adam constants (five learning rates, beta1, beta2, eps)."""
        out = {k: self.raw[k].detach().cpu().clone() for k in RAW}
        out["adam_state"] = self.state.detach().cpu().clone()
        a = self.adam
        out["adam_config"] = torch.tensor([*a.lr, a.beta1, a.beta2, a.eps], dtype=torch.float64)
        return out

    def load_state_dict(self, sd: Dict[str, torch.Tensor]) -> None:
        """Resumes from ``state_dict()`` of a trainer over as many Gaussians
        and channels.  The values go into this trainer's own buffers and the
        activated scales and opacities are rebuilt; the step graph is captured
        again at the next ``run`` (it holds the Adam constants)."""
        for k in RAW:
            if tuple(sd[k].shape) != tuple(self.raw[k].shape):
                raise ValueError(f"{k}: shape {tuple(sd[k].shape)} in the checkpoint, {tuple(self.raw[k].shape)} here")
        if sd["adam_state"].numel() != self.state.numel():
            raise ValueError("the checkpoint's Adam state has another size (Gaussian or channel count)")
        for k in RAW:
            self.raw[k].copy_(sd[k])
        self.state.copy_(sd["adam_state"])
        c = [float(x) for x in sd["adam_config"]]
        self.adam = B.adam_config(c[:5], c[5], c[6], c[7])
        B.gs_activate(self.N, self.raw["log_scales"], self.raw["opacity_logits"], self.scales, self.opacities)
        self.graph = None

    def steps_taken(self) -> int:
        """Adam steps applied so far (skipped steps excluded; one device read)."""
        return int(self.state[:4].view(torch.int32).item())

    def run(self, n: int, check_every: int = 50, graph: bool = True) -> None:
        """``n`` steps.  Every ``check_every`` steps the overflow flag is read;
        after an overflow the buffers grow by ``headroom`` over the current
        intersection count and the graph is captured again."""
        if graph and self.graph is None:
            self.capture()
        for i in range(n):
            self.step()
            if (i + 1) % check_every == 0 or i + 1 == n:
                if self.overflowed():
                    K = exact_capacity(self.params, self.views, self.eps2d)
                    self._make(int(self.headroom * K) + 1024)
                    if graph:
                        self.capture()
