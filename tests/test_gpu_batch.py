"""Batched rendering (many views and scenes per launch): the batch equals the
per-view launches; tile-walking configurations (persistent queue, longest-first
order) and CUDA-graph replay change no result; the batched workloads match the
FP64 oracle on sampled pixels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import compare
from paper_2312_02121_gb300 import batch as GB
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import pipeline
from paper_2312_02121_gb300 import workloads as wl
from gpu_helpers import np_, rel_l2

pytestmark = pytest.mark.gpu


def _mixed_workload():
    a = wl.small_case(31, 900, 70, 45, log_scale_mu=-2.6)
    b = wl.small_case(32, 1500, 96, 64, log_scale_mu=-2.8)
    rng = np.random.default_rng(7)
    cams = wl.sphere_cameras(rng, 3, 4.0, [(64, 48), (50, 37), (80, 80)], focal_range=(60.0, 120.0))
    views = [wl.View(0, a.views[0].camera), wl.View(1, b.views[0].camera)] + [wl.View(i % 2, c) for i, c in
                                                                          enumerate(cams)]
    trng = np.random.default_rng(8)
    return wl.Workload("mixed", [a.scenes[0], b.scenes[0]], views,
                       [wl.target_image(trng, v.camera) for v in views])


def _renderer(w, deterministic=True, **cfg):
    params, views, ranges, targets = GB.workload_views(w)
    cap = GB.exact_capacity(params, views, w.eps2d)
    rc = B.RasterConfig(cfg.get("persistent", False), cfg.get("ctas_per_sm", 0)) if cfg else None
    return GB.BatchRenderer(params, views, cap, targets, w.eps2d, rc, cfg.get("longest_first", False),
                            deterministic), params, views, ranges, targets


def test_batch_matches_per_view_launches():
    w = _mixed_workload()
    r, params, views, ranges, targets = _renderer(w)
    r.step()
    caps = GB.per_view_capacities(params, [v.camera for v in w.views], ranges, w.eps2d)
    pv = GB.PerViewRenderer(params, [v.camera for v in w.views], ranges, caps, targets, w.eps2d, deterministic=True)
    pv.step()
    torch.cuda.synchronize()
    assert not r.overflowed() and not pv.overflowed()
    for i, sub in enumerate(pv.r):
        assert torch.equal(r.image(i), sub.image(0))
    # deterministic mode fixes every summation order except the per-Gaussian sum
    # over the views of a scene (atomics); per-projection gradients are identical
    assert torch.equal(r.g2, torch.cat([x.g2 for x in pv.r])) and torch.equal(r.gc, torch.cat([x.gc for x in pv.r]))
    gb, gp = r.grads(), pv.grads()
    for k in gb:
        assert rel_l2(np_(gb[k]), np_(gp[k])) <= 1e-5, k


@pytest.mark.parametrize("cfg", GB.CANDIDATES)
def test_tile_walking_configs_change_nothing(cfg):
    w = _mixed_workload()
    r0, *_ = _renderer(w)
    r0.step()
    r1, *_ = _renderer(w, **cfg)
    r1.step()
    torch.cuda.synchronize()
    assert torch.equal(r0.rgb, r1.rgb) and torch.equal(r0.last_idx, r1.last_idx)
    # deterministic mode: per-projection gradients are bit-identical; per-Gaussian
    # ones are summed over the views of a scene with atomics (order varies)
    assert torch.equal(r0.g2, r1.g2) and torch.equal(r0.gc, r1.gc)
    for k, v in r0.grads().items():
        assert rel_l2(np_(v), np_(r1.grads()[k])) <= 1e-5, k


def test_graph_replay_equals_eager():
    w = _mixed_workload()
    r, *_ = _renderer(w, deterministic=True, persistent=True, longest_first=True)
    r.step_eager()
    torch.cuda.synchronize()
    ref_img, ref_g2, ref_gc = r.rgb.clone(), r.g2.clone(), r.gc.clone()
    ref = {k: v.clone() for k, v in r.grads().items()}
    r.capture()
    for _ in range(3):
        r.step()
    torch.cuda.synchronize()
    assert torch.equal(ref_img, r.rgb)
    assert torch.equal(ref_g2, r.g2) and torch.equal(ref_gc, r.gc)
    for k, v in r.grads().items():  # summed over the views of a scene with atomics
        assert rel_l2(np_(v), np_(ref[k])) <= 1e-5, k


def test_batch_overflow_flagged():
    w = _mixed_workload()
    params, views, ranges, targets = GB.workload_views(w)
    r = GB.BatchRenderer(params, views, 50, targets, w.eps2d)
    r.step()
    assert r.overflowed()


def _sampled_view_parity(w, view_ids, n_pix=400, seed=0):
    """Batched fwd+bwd of the whole workload; the oracle on sampled pixels of a
    few views, with dL/dC nonzero only there (gradient comparison per view)."""
    params, views, ranges, targets = GB.workload_views(w)
    cap = GB.exact_capacity(params, views, w.eps2d)
    r = GB.BatchRenderer(params, views, cap, targets, w.eps2d, B.RasterConfig(True, 0), True, False)
    r.forward()
    torch.cuda.synchronize()
    assert not r.overflowed()
    rng = np.random.default_rng(seed)
    for vi in view_ids:
        v = w.views[vi]
        cam, sc = v.camera, w.scenes[v.scene]
        hv = views.host[vi]
        s, e = hv.proj_offset, hv.proj_offset + hv.g_count
        gp = dict(means2d=np_(r.means2d[s:e]).astype(float),
                  conics=compare.conic_from_factors(np_(r.conics[s:e])),
                  depths=np_(r.depths[s:e]).astype(float), rects=np_(r.rects[s:e]).astype(np.int32),
                  valid=(np_(r.touched[s:e]) > 0).astype(np.int32))
        pix = np.sort(rng.choice(cam.pixels, n_pix, replace=False))
        o = oracle.rasterize(gp, sc.opacities, sc.colors, cam.width, cam.height, pixels=pix)
        img = np_(r.image(vi)).reshape(-1, 3)[pix]
        ok = o["margin"] >= 1e-4
        assert ok.mean() > 0.97
        assert np.abs(img - o["rgb"])[ok].max() <= 1e-5, vi
        # gradients of this view alone, masked to the sampled pixels
        G = torch.zeros(views.pixels, 3, device="cuda")
        Gs = rng.standard_normal((n_pix, 3)) * ok[:, None]
        off = hv.pixel_offset
        G[off + torch.as_tensor(pix, device="cuda")] = torch.as_tensor(Gs, dtype=torch.float32, device="cuda")
        r.dL.copy_(G)
        r.backward()
        torch.cuda.synchronize()
        ob = compare.with_factored_conic_grad(
            oracle.rasterize_bwd(gp, sc.opacities, sc.colors, cam.width, cam.height, Gs, pixels=pix), gp["conics"])
        g0 = ranges[vi][0]
        for k, gk in (("opacities", r.g_op), ("colors", r.g_col)):
            got = np_(gk[g0:g0 + sc.n])
            assert rel_l2(got, ob[k]) <= 1e-4, (vi, k)
        for k, gk in (("means2d", r.g2), ("conics", r.gc)):
            assert rel_l2(np_(gk[s:e]), ob[k]) <= 1e-4, (vi, k)


def test_batch_views_500k_64_sampled_parity():
    w = wl.batch_views_500k_64()
    _sampled_view_parity(w, [0, 17, 63])


def test_batch_scenes_16x4_sampled_parity():
    w = wl.batch_scenes_16x4()
    _sampled_view_parity(w, [0, 21, 62])


def test_host_inputs_are_uploaded_by_every_replay():
    # a captured step that copies its inputs from pinned host memory, with the late copies on a
    # second stream, renders exactly what the same step renders from device inputs; a change of the
    # host tensors between replays reaches the next replay
    w = _mixed_workload()
    params, views, ranges, targets = GB.workload_views(w)
    cap = GB.exact_capacity(params, views, w.eps2d) + 1000
    ref = GB.BatchRenderer(params, views, cap, targets, w.eps2d, deterministic=True)
    keys = ("means", "quats", "scales", "opacities", "colors")
    dev = pipeline.Params(*[torch.full_like(getattr(params, k), 0.5) for k in keys])
    r = GB.BatchRenderer(dev, views, cap, torch.zeros_like(targets), w.eps2d, deterministic=True)
    host = {k: getattr(params, k).cpu().pin_memory() for k in keys}
    r.attach_host_inputs(host, targets.cpu().pin_memory())
    r.capture()
    for trial in range(2):
        if trial == 1:
            host["colors"].mul_(0.5)
            host["means"].add_(0.01)
            params.colors.mul_(0.5)
            params.means.add_(0.01)
        ref.step_eager()
        r.step()
        torch.cuda.synchronize()
        assert torch.equal(r.rgb, ref.rgb)
        # the loss is summed with one atomic per block: equal up to the order of those sums
        assert float(r.loss_host[0]) == pytest.approx(float(ref.loss.item()), rel=1e-6)
        for k, g in ref.grads().items():
            assert rel_l2(np_(r.grads()[k]), np_(g)) <= 1e-6, k


def test_host_pipeline_two_deep_gives_each_step_its_own_inputs_and_loss():
    # batch.HostPipeline keeps two captured steps in flight on two streams; each step copies the host
    # inputs and reads back its own loss, which must equal the loss of a plain step on the same inputs.
    # Host inputs may change only while no step is in flight (after finish), as for any async copy.
    w = _mixed_workload()
    params, views, ranges, targets = GB.workload_views(w)
    cap = GB.exact_capacity(params, views, w.eps2d) + 1000
    keys = ("means", "quats", "scales", "opacities", "colors")
    host = {k: getattr(params, k).cpu().pin_memory() for k in keys}
    host_t = targets.cpu().pin_memory()

    def make():
        dev_p = pipeline.Params(*[torch.empty_like(getattr(params, k)) for k in keys])
        r = GB.BatchRenderer(dev_p, views, cap, torch.empty_like(targets), w.eps2d)
        r.attach_host_inputs(host, host_t)
        return r

    pipe = GB.HostPipeline(make)
    ref = GB.BatchRenderer(params, views, cap, targets, w.eps2d)
    for trial in range(2):
        if trial == 1:  # nothing in flight: change the inputs on the host and in the reference
            host["colors"].mul_(0.5)
            params.colors.mul_(0.5)
        ref.step_eager()
        want = float(ref.loss.item())
        first = pipe.step()
        assert (first is None) == (trial == 0)
        got = [pipe.step() for _ in range(3)] + [pipe.finish()]
        assert got == pytest.approx([want] * 4, rel=1e-6), trial
    assert not pipe.overflowed()
