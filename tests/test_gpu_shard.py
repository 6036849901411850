"""Splitting a multi-view step over ranks, with the CUDA kernels on one GPU.

The ranks' shares run one after the other on the same device (no collective,
and no kernel waits on another).  The images of each rank's views must equal
the whole batch's bit for bit.  The ranks' partial gradients must sum to the
whole batch's gradients.  Both sides use the deterministic backward, so only
the order of the final per-scene sum differs."""
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import batch as GB
from paper_2312_02121_gb300 import shard
from paper_2312_02121_gb300 import workloads as wl
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu


def _whole(w):
    params, views, ranges, targets = GB.workload_views(w)
    cap = GB.exact_capacity(params, views, w.eps2d)
    r = GB.BatchRenderer(params, views, cap, targets, w.eps2d, deterministic=True)
    r.step()
    return r, params, ranges, targets


@pytest.mark.parametrize("whole_scenes", [False, True])
@pytest.mark.parametrize("world", [2, 3])
def test_rank_shares_sum_to_the_whole_batch(world, whole_scenes):
    w = wl.batch_scenes_16x4(seed=6, scenes=3, views_per_scene=3, n_range=(2000, 20000), width=120, height=90)
    full, params, ranges, targets = _whole(w)
    scene_of_view = [v.scene for v in w.views]
    cams = [v.camera for v in w.views]
    total = {k: torch.zeros_like(v) for k, v in full.grads().items()}
    seen = []
    for rank in range(world):
        s = shard.ShardedRenderer(params, cams, ranges, scene_of_view, targets, world, rank,
                                  whole_scenes=whole_scenes, eps2d=w.eps2d, deterministic=True)
        s.local_step()
        assert not s.overflowed()
        for k, v in s.grads().items():
            total[k] += v
        for j, v in enumerate(s.mine):
            assert torch.equal(s.r.image(j), full.image(v)), (rank, v)
            seen.append(v)
    torch.cuda.synchronize()
    assert sorted(seen) == list(range(len(w.views)))
    for k, ref in full.grads().items():
        assert rel_l2(total[k].cpu(), ref.cpu()) < 1e-6, k


def test_one_rank_is_the_whole_batch():
    w = wl.batch_views_500k_64(seed=2, n=20000, views=4, resolutions=[(100, 80), (64, 64)])
    full, params, ranges, targets = _whole(w)
    s = shard.ShardedRenderer(params, [v.camera for v in w.views], ranges, [0] * len(w.views), targets, 1, 0,
                              eps2d=w.eps2d, deterministic=True)
    assert not s.plan.needs_allreduce
    s.step()
    torch.cuda.synchronize()
    for k, ref in full.grads().items():  # views of one scene meet in atomics: order only
        assert rel_l2(s.grads()[k].cpu(), ref.cpu()) < 1e-6, k
    for j in range(len(w.views)):
        assert torch.equal(s.r.image(j), full.image(j))
