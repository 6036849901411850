"""Splitting a multi-view step over ranks (one process per GPU).

Each view's projection, binning, compositing and their backward passes read
only that view's camera and its scene's Gaussians (Sec. 2 and 3 treat one
camera at a time).  Views are coupled in one place only: a per-Gaussian
gradient of a scene sums over every view of that scene.  A rank that renders
some of a scene's views therefore holds a partial sum.  So the views are split
across ranks with no exchange in the data path.  One all-reduce (sum) of the
flat per-Gaussian gradient buffer then completes the step, and it is issued
only when some scene's views landed on more than one rank.  With
``whole_scenes`` every scene goes to a single rank, and no collective is
needed at all.

The loss is the mean over every pixel of every view of the whole job.  So each
rank scales dL/dC by the job's pixel count, not by its own.

Nothing here touches pixels or Gaussians: ``plan`` and ``GradBuffer`` are
host logic, shared by the GPU path (``ShardedRenderer``) and by CPU tests that
run the ranks as ``gloo`` processes.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import torch

# per-Gaussian gradient fields and their widths: 14 numbers per Gaussian for
# 3 colour channels (11 + C for C channels)
GRAD_FIELDS = (("means", 3), ("quats", 4), ("scales", 3), ("opacities", 1), ("colors", 3))
GRAD_WIDTH = sum(k for _, k in GRAD_FIELDS)


def grad_fields(channels: int = 3):
    return GRAD_FIELDS[:-1] + (("colors", int(channels)),)


def lpt_assign(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time-first list scheduling.  Units are taken in
    decreasing cost (ties by index).  Each goes to the rank with the least cost
    so far (ties to the lowest rank).  The result is deterministic, so every
    rank computes the same assignment with no communication.  The makespan is
    at most total/world + max(cost).  Returns each rank's units in
    increasing order."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for u in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world), key=lambda j: (load[j], j))
        out[r].append(u)
        load[r] += float(costs[u])
    return [sorted(o) for o in out]


@dataclasses.dataclass
class Plan:
    world: int
    views_of_rank: List[List[int]]
    split_scenes: List[int]  # scenes whose views are spread over more than one rank

    @property
    def needs_allreduce(self) -> bool:
        return bool(self.split_scenes)

    def owner_of_scene(self, scene_of_view: Sequence[int]) -> Dict[int, List[int]]:
        """Ranks that render at least one view of each scene."""
        own: Dict[int, List[int]] = {}
        for r, vs in enumerate(self.views_of_rank):
            for v in vs:
                lst = own.setdefault(int(scene_of_view[v]), [])
                if r not in lst:
                    lst.append(r)
        return own


def plan(scene_of_view: Sequence[int], view_cost: Sequence[float], world: int,
         whole_scenes: bool = False) -> Plan:
    """Assigns views to ranks.  By default the unit is a view, with cost
    ``view_cost`` (its pixel count, or its intersection count when known).
    With ``whole_scenes`` the unit is a scene with the summed cost of its
    views, so that no scene is split."""
    if len(scene_of_view) != len(view_cost):
        raise ValueError("scene_of_view and view_cost differ in length")
    if whole_scenes:
        scenes = sorted(set(int(s) for s in scene_of_view))
        cost = [sum(float(c) for s2, c in zip(scene_of_view, view_cost) if int(s2) == s) for s in scenes]
        by_rank = lpt_assign(cost, world)
        views = [sorted(v for v, s in enumerate(scene_of_view) if scenes.index(int(s)) in units)
                 for units in by_rank]
    else:
        views = lpt_assign(view_cost, world)
    p = Plan(world, views, [])
    p.split_scenes = sorted(s for s, ranks in p.owner_of_scene(scene_of_view).items() if len(ranks) > 1)
    return p


class GradBuffer:
    """All per-Gaussian gradients in one flat buffer, so that one collective
    sums them.  Each field is a contiguous [N, k] view into the buffer (field
    after field), which can be handed directly to the gradient outputs of the
    compositing and projection backward calls."""

    def __init__(self, n: int, dtype=torch.float32, device="cpu", channels: int = 3):
        self.n = int(n)
        rows = max(self.n, 1)
        fields = grad_fields(channels)
        self.flat = torch.zeros(rows * sum(k for _, k in fields), dtype=dtype, device=device)
        self.fields: Dict[str, torch.Tensor] = {}
        off = 0
        for name, k in fields:
            v = self.flat[off:off + rows * k]
            self.fields[name] = v.view(rows) if k == 1 else v.view(rows, k)
            off += rows * k

    def zero_(self):
        self.flat.zero_()

    def allreduce(self, group=None):
        """Sums the buffer over the ranks of ``group`` in place (one call)."""
        import torch.distributed as dist
        dist.all_reduce(self.flat, op=dist.ReduceOp.SUM, group=group)

    def grads(self) -> Dict[str, torch.Tensor]:
        return {k: v[:self.n] for k, v in self.fields.items()}


class ShardedRenderer:
    """One rank's share of a multi-view step on its GPU: a ``BatchRenderer``
    over the views that ``plan`` gave this rank, accumulating into a
    ``GradBuffer`` that is summed over ranks after the backward when a scene
    is split.

    ``params``, ``cameras``, ``g_ranges`` (each view's Gaussian range) and
    ``targets`` (packed [pixels, 3] of ALL views, in view order) describe the
    whole job and are the same on every rank."""

    def __init__(self, params, cameras: Sequence, g_ranges: Sequence, scene_of_view: Sequence[int],
                 targets: torch.Tensor, world: int, rank: int, group=None, whole_scenes: bool = False,
                 view_cost: Optional[Sequence[float]] = None, eps2d: float = 0.3, K_capacity: Optional[int] = None,
                 config=None, deterministic: bool = False):
        from . import batch as GB
        from . import binding as B
        dev = params.means.device
        pix = [c.width * c.height for c in cameras]
        self.plan = plan(scene_of_view, view_cost if view_cost is not None else pix, world, whole_scenes)
        self.rank, self.group = rank, group
        self.mine = self.plan.views_of_rank[rank]
        self.buf = GradBuffer(params.n, params.means.dtype, dev, params.channels)
        starts = [0]
        for p_ in pix:
            starts.append(starts[-1] + p_)
        self.views = None
        self.r = None
        if self.mine:
            tg = torch.cat([targets[starts[v]:starts[v + 1]] for v in self.mine])
            self.views = B.Views([cameras[v] for v in self.mine], [g_ranges[v] for v in self.mine], device=dev)
            cap = K_capacity if K_capacity is not None else GB.exact_capacity(params, self.views, eps2d)
            self.r = GB.BatchRenderer(params, self.views, cap, tg, eps2d, config, deterministic=deterministic,
                                      shared_grads=self.buf.fields, loss_pixels=sum(pix))

    def capture(self):
        if self.r is not None:
            self.r.capture()

    def local_step(self):
        """This rank's views only: the gradient buffer then holds this
        rank's partial sums."""
        self.buf.zero_()
        if self.r is not None:
            self.r.step()

    def step(self):
        self.local_step()
        if self.plan.needs_allreduce:
            self.buf.allreduce(self.group)

    def overflowed(self) -> bool:
        return self.r is not None and self.r.overflowed()

    def grads(self) -> Dict[str, torch.Tensor]:
        return self.buf.grads()
