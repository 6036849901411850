"""The multi-GPU bench mode's host logic on the CPU, with two and three gloo
ranks: bench.sharded_plan splits the 64 views of the one-scene batch over the
ranks (every view once, the pixel load balanced within one view's pixels), and
the step's one all-reduce of the flat per-Gaussian gradient buffer leaves on
every rank the sum over all views -- here with per-view stand-in gradients
(view v adds v + 1 to its own slice), since the kernels need a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2312_02121_gb300 import shard


def test_sharded_plan_covers_every_view_once_and_balances_pixels():
    for world in (1, 2, 3, 8):
        w, p = bench.sharded_plan(world)
        assert len(p.views_of_rank) == world
        assert sorted(v for r in p.views_of_rank for v in r) == list(range(len(w.views))) and len(w.views) == 64
        loads = [sum(w.views[v].camera.pixels for v in r) for r in p.views_of_rank]
        assert max(loads) <= sum(loads) / world + max(v.camera.pixels for v in w.views)
        assert p.needs_allreduce == (world > 1)  # one scene: split over ranks as soon as there are two


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, p = bench.sharded_plan(world)
        n = 1000  # a stand-in scene size: the buffer's shape, not the workload's
        buf = shard.GradBuffer(n, torch.float64)
        for v in p.views_of_rank[rank]:
            for name, _ in shard.GRAD_FIELDS:
                buf.fields[name][(v * 13) % n:(v * 13) % n + 10] += v + 1
        if p.needs_allreduce:
            buf.allreduce()
        np.save(out.format(rank=rank), buf.flat.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_one_allreduce_leaves_the_sum_over_all_views_on_every_rank(world, tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "r{rank}.npy")
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    ref = shard.GradBuffer(1000, torch.float64)
    for v in range(64):
        for name, _ in shard.GRAD_FIELDS:
            ref.fields[name][(v * 13) % 1000:(v * 13) % 1000 + 10] += v + 1
    for r in range(world):
        np.testing.assert_array_equal(np.load(out.format(rank=r)), ref.flat.numpy())
