"""Splitting a multi-view step over ranks, checked on the CPU.

Ranks run as ``gloo`` processes (world size 2 and 3).  Each rank computes the
FP64 oracle's gradients for the views that ``shard.plan`` gives it, into a
``shard.GradBuffer``, and then sums the buffers with the buffer's one
all-reduce.  The summed gradients must equal the gradients of the whole batch
computed in one process.  With whole scenes per rank, no collective is issued,
and each rank's own scenes must already be complete."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2312_02121_gb300 import shard
from paper_2312_02121_gb300 import workloads as wl


# -- host logic ---------------------------------------------------------------

def test_lpt_assigns_every_unit_once_and_bounds_the_makespan():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        for n in (0, 1, 5, 64):
            costs = rng.integers(1, 1000, n).tolist()
            a = shard.lpt_assign(costs, world)
            assert len(a) == world
            flat = sorted(u for r in a for u in r)
            assert flat == list(range(n))
            if n:
                loads = [sum(costs[u] for u in r) for r in a]
                assert max(loads) <= sum(costs) / world + max(costs)
    # deterministic and tie-broken by index
    assert shard.lpt_assign([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert shard.lpt_assign([1, 9, 4, 4], 2) == [[1], [0, 2, 3]]
    with pytest.raises(ValueError):
        shard.lpt_assign([1], 0)


def test_plan_split_scenes_and_whole_scenes():
    scene_of_view = [0, 0, 0, 1, 1, 2]
    cost = [10, 10, 10, 1, 1, 30]
    p = shard.plan(scene_of_view, cost, 2)
    assert sorted(v for r in p.views_of_rank for v in r) == list(range(6))
    # LPT: view 5 (30) -> rank 0; views 0, 1, 2 (10 each) -> rank 1; the two 1s split
    assert p.views_of_rank == [[3, 5], [0, 1, 2, 4]]
    assert p.needs_allreduce and p.split_scenes == [1]
    q = shard.plan(scene_of_view, cost, 2, whole_scenes=True)
    assert not q.needs_allreduce
    own = q.owner_of_scene(scene_of_view)
    assert all(len(r) == 1 for r in own.values())
    # scene costs 30, 2, 30: the two 30s go to different ranks
    assert own[0] != own[2]
    one = shard.plan(scene_of_view, cost, 1)
    assert one.views_of_rank == [list(range(6))] and not one.needs_allreduce


def test_grad_buffer_fields_are_contiguous_views_of_one_buffer():
    b = shard.GradBuffer(7, torch.float64)
    assert b.flat.numel() == 7 * shard.GRAD_WIDTH
    for name, k in shard.GRAD_FIELDS:
        f = b.fields[name]
        assert f.is_contiguous() and f.shape[0] == 7 and (f.dim() == 1 if k == 1 else f.shape[1] == k)
        f.fill_(1.0)
    assert float(b.flat.sum()) == 7 * shard.GRAD_WIDTH
    b.zero_()
    assert float(b.flat.abs().sum()) == 0.0


# -- ranks as processes -------------------------------------------------------

def _views_workload():
    return wl.batch_views_500k_64(seed=4, n=1500, views=5, resolutions=[(48, 32), (40, 40), (64, 24)])


def _scenes_workload():
    return wl.batch_scenes_16x4(seed=5, scenes=3, views_per_scene=2, n_range=(200, 1200), width=40, height=30)


def _view_grads(oracle, w, v, total_pix):
    """FP64 oracle gradients of L = mean over all pixels of all views of
    (C - target)^2, restricted to view v's share (its own pixels)."""
    cam, sc = w.views[v].camera, w.scenes[w.views[v].scene]
    out = oracle.render(cam, sc, w.eps2d)
    dL = 2.0 * (out["rgb"] - np.asarray(w.targets[v], np.float64)) / (3 * total_pix)
    return oracle.backward(cam, sc, dL, w.eps2d)


def _accumulate(oracle, w, views, buf, offs, total_pix):
    for v in views:
        g = _view_grads(oracle, w, v, total_pix)
        o, n = offs[w.views[v].scene], w.scenes[w.views[v].scene].n
        for name, _ in shard.GRAD_FIELDS:
            buf.fields[name][o:o + n] += torch.from_numpy(np.asarray(g[name], np.float64).reshape(
                buf.fields[name][o:o + n].shape))


def _rank_main(rank, world, port, which, whole, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        w = _views_workload() if which == "views" else _scenes_workload()
        offs = np.cumsum([0] + [s.n for s in w.scenes])
        total_pix = w.pixels
        scene_of_view = [v.scene for v in w.views]
        cost = [v.camera.pixels for v in w.views]
        p = shard.plan(scene_of_view, cost, world, whole_scenes=whole)
        buf = shard.GradBuffer(w.gaussians, torch.float64)
        _accumulate(oracle, w, p.views_of_rank[rank], buf, offs, total_pix)
        if p.needs_allreduce:
            buf.allreduce()
        np.save(result_path.format(rank=rank), buf.flat.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, which, whole, tmp_path, oracle_lib):
    path = str(tmp_path / "rank{rank}.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), which, whole, path), nprocs=world, join=True,
                       start_method="spawn")
    w = _views_workload() if which == "views" else _scenes_workload()
    offs = np.cumsum([0] + [s.n for s in w.scenes])
    full = shard.GradBuffer(w.gaussians, torch.float64)
    _accumulate(oracle_lib, w, range(len(w.views)), full, offs, w.pixels)
    got = [np.load(path.format(rank=r)) for r in range(world)]
    p = shard.plan([v.scene for v in w.views], [v.camera.pixels for v in w.views], world, whole_scenes=whole)
    return w, p, full, got, offs


@pytest.mark.parametrize("world", [2, 3])
def test_view_sharded_gradients_sum_to_the_whole_batch(world, tmp_path, oracle_lib):
    w, p, full, got, _ = _run(world, "views", False, tmp_path, oracle_lib)
    assert p.needs_allreduce  # one scene, several ranks
    ref = full.flat.numpy()
    assert np.abs(ref).max() > 0
    for g in got:  # every rank holds the full sum after the all-reduce
        np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_scene_sharded_ranks_need_no_collective(tmp_path, oracle_lib):
    w, p, full, got, offs = _run(2, "scenes", True, tmp_path, oracle_lib)
    assert not p.needs_allreduce
    own = p.owner_of_scene([v.scene for v in w.views])
    N = w.gaussians
    ref = {name: f.numpy() for name, f in full.fields.items()}
    for s, (r,) in own.items():
        buf = shard.GradBuffer(N, torch.float64)
        buf.flat.copy_(torch.from_numpy(got[r]))
        o, n = offs[s], w.scenes[s].n
        for name, _ in shard.GRAD_FIELDS:
            a, b = buf.fields[name].numpy()[o:o + n], ref[name][o:o + n]
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)
        for other in range(2):  # ranks that do not own the scene left its rows at zero
            if other != r:
                z = shard.GradBuffer(N, torch.float64)
                z.flat.copy_(torch.from_numpy(got[other]))
                assert all(float(np.abs(z.fields[name].numpy()[o:o + n]).max()) == 0.0
                           for name, _ in shard.GRAD_FIELDS)
