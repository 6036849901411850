"""The training-step kernels (L2 loss, fused Adam with activations) against the
FP64 reference of ``oracle.optim``, and the graph-captured optimisation loop
against the oracle's loop."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import optim as ref
from paper_2312_02121_gb300 import binding as B
from paper_2312_02121_gb300 import workloads as wl
from paper_2312_02121_gb300.train import RAW, Trainer
from gpu_helpers import np_, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,offset", [(3 * 64 * 64, 0), (4097, 0), (4097, 1), (5, 0)])
def test_l2_loss_matches_oracle(n, offset):
    rng = np.random.default_rng(n + offset)
    a, b = rng.uniform(size=n + offset).astype(np.float32), rng.uniform(size=n + offset).astype(np.float32)
    ta, tb = torch.tensor(a, device="cuda")[offset:], torch.tensor(b, device="cuda")[offset:]
    dL = torch.empty_like(ta)
    loss = torch.zeros(1, device="cuda")
    B.gs_l2_loss(ta, tb, 1.0 / n, dL, loss)
    L, g = ref.l2_loss(a[offset:], b[offset:], 1.0 / n)
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    np.testing.assert_allclose(np_(dL), g, rtol=1e-6, atol=1e-12)


def _raw_host(rng, n):
    return dict(means=rng.standard_normal((n, 3)).astype(np.float32),
                quats=rng.standard_normal((n, 4)).astype(np.float32),
                log_scales=rng.normal(-3, 0.5, (n, 3)).astype(np.float32),
                opacity_logits=rng.standard_normal(n).astype(np.float32),
                colors=rng.uniform(size=(n, 3)).astype(np.float32))


def _dev(raw):
    return {k: torch.tensor(v, device="cuda") for k, v in raw.items()}


LR = (1e-3, 2e-3, 5e-3, 5e-2, 2.5e-3)


def test_adam_kernel_matches_oracle():
    rng = np.random.default_rng(0)
    N = 1000
    raw = _raw_host(rng, N)
    d = _dev(raw)
    sc, op = torch.empty(N, 3, device="cuda"), torch.empty(N, device="cuda")
    B.gs_activate(N, d["log_scales"], d["opacity_logits"], sc, op)
    s_ref, o_ref = ref.activate(raw)
    np.testing.assert_allclose(np_(sc), s_ref, rtol=1e-6)
    np.testing.assert_allclose(np_(op), o_ref, rtol=1e-6)
    cfg = B.adam_config(LR, 0.9, 0.999, 1e-8)
    state = torch.zeros(B.gs_adam_state_size(N), dtype=torch.uint8, device="cuda")
    adam = ref.Adam(raw, LR, 0.9, 0.999, 1e-8)
    cur = {k: v.astype(np.float64) for k, v in raw.items()}
    for step in range(5):
        g = dict(means=rng.standard_normal((N, 3)), quats=rng.standard_normal((N, 4)),
                 scales=rng.standard_normal((N, 3)), opacities=rng.standard_normal(N),
                 colors=rng.standard_normal((N, 3)))
        g32 = {k: torch.tensor(v.astype(np.float32), device="cuda") for k, v in g.items()}
        B.gs_adam_step(N, cfg, state, d["means"], d["quats"], d["log_scales"], d["opacity_logits"], d["colors"],
                       g32["means"], g32["quats"], g32["scales"], g32["opacities"], g32["colors"], sc, op)
        cur = adam.step(cur, ref.raw_gradients(cur, {k: v.astype(np.float32) for k, v in g.items()}))
    torch.cuda.synchronize()
    for k in RAW:
        np.testing.assert_allclose(np_(d[k]), cur[k], rtol=2e-5, atol=2e-6, err_msg=k)
    s_ref, o_ref = ref.activate(cur)
    np.testing.assert_allclose(np_(sc), s_ref, rtol=2e-5)
    np.testing.assert_allclose(np_(op), o_ref, rtol=2e-5, atol=1e-6)
    assert int(state[:4].view(torch.int32).item()) == 5


def test_adam_step_is_skipped_when_the_flag_is_set():
    rng = np.random.default_rng(1)
    N = 100
    d = _dev(_raw_host(rng, N))
    before = {k: v.clone() for k, v in d.items()}
    sc, op = torch.empty(N, 3, device="cuda"), torch.empty(N, device="cuda")
    B.gs_activate(N, d["log_scales"], d["opacity_logits"], sc, op)
    g = [torch.ones(N, 3, device="cuda"), torch.ones(N, 4, device="cuda"), torch.ones(N, 3, device="cuda"),
         torch.ones(N, device="cuda"), torch.ones(N, 3, device="cuda")]
    state = torch.zeros(B.gs_adam_state_size(N), dtype=torch.uint8, device="cuda")
    flag = torch.ones(1, dtype=torch.int32, device="cuda")
    B.gs_adam_step(N, B.adam_config(LR), state, d["means"], d["quats"], d["log_scales"], d["opacity_logits"],
                   d["colors"], *g, sc, op, flag)
    torch.cuda.synchronize()
    for k in RAW:
        assert torch.equal(d[k], before[k]), k
    assert int(state[:4].view(torch.int32).item()) == 0
    flag.zero_()
    B.gs_adam_step(N, B.adam_config(LR), state, d["means"], d["quats"], d["log_scales"], d["opacity_logits"],
                   d["colors"], *g, sc, op, flag)
    assert int(state[:4].view(torch.int32).item()) == 1
    assert not torch.equal(d["means"], before["means"])


def _scene_raw(sc):
    o = np.clip(np.asarray(sc.opacities, np.float64), 1e-6, 1 - 1e-6)
    return dict(means=np.array(sc.means, np.float32), quats=np.array(sc.quats, np.float32),
                log_scales=np.log(np.asarray(sc.scales, np.float64)).astype(np.float32),
                opacity_logits=np.log(o / (1 - o)).astype(np.float32), colors=np.array(sc.colors, np.float32))


def _oracle_loop(cam, raw, target, steps, eps2d):
    """The same optimisation in FP64: oracle forward and backward, oracle Adam."""
    adam = ref.Adam(raw, LR, 0.9, 0.999, 1e-15)
    cur = {k: v.astype(np.float64) for k, v in raw.items()}
    losses = []
    for _ in range(steps):
        s, o = ref.activate(cur)

        class Sc:
            pass

        scn = Sc()
        scn.means, scn.quats, scn.scales, scn.opacities, scn.colors = cur["means"], cur["quats"], s, o, cur["colors"]
        img = oracle.render(cam, scn, eps2d)["rgb"]
        L, dL = ref.l2_loss(img, target, 1.0 / img.size)
        losses.append(L)
        g = oracle.backward(cam, scn, dL, eps2d)
        cur = adam.step(cur, ref.raw_gradients(cur, g))
    return cur, losses


def test_optimisation_loop_matches_oracle_loop():
    w = wl.small_case(41, 600, 64, 48, log_scale_mu=-2.4)
    cam, sc = w.views[0].camera, w.scenes[0]
    raw = _scene_raw(sc)
    target = w.targets[0]
    views = B.Views([cam], [(0, sc.n)], device="cuda")
    t = Trainer(_dev(raw), views, torch.tensor(target.reshape(-1, 3), device="cuda"), lr=LR, eps=1e-15,
                eps2d=w.eps2d)
    steps = 3
    losses = []
    for _ in range(steps):
        t.step()
        losses.append(t.loss())
    assert not t.overflowed() and t.steps_taken() == steps
    cur, ref_losses = _oracle_loop(cam, raw, target, steps, w.eps2d)
    np.testing.assert_allclose(losses, ref_losses, rtol=1e-4)
    # Adam moves each parameter by about lr per step whatever the gradient's size, so a
    # gradient within rounding of zero can move either way: compare the motion as a whole
    for k in RAW:
        moved_gpu = np_(t.raw[k]).astype(np.float64) - raw[k]
        moved_ref = cur[k] - raw[k]
        assert rel_l2(moved_gpu, moved_ref) <= 2e-2, k


def test_graph_replay_follows_the_eager_loop():
    w = wl.small_case(42, 1500, 96, 80, log_scale_mu=-2.6)
    cam, sc = w.views[0].camera, w.scenes[0]
    raw = _scene_raw(sc)
    tgt = torch.tensor(w.targets[0].reshape(-1, 3), device="cuda")
    views = B.Views([cam], [(0, sc.n)], device="cuda")
    a = Trainer(_dev(raw), views, tgt, lr=LR)
    b = Trainer(_dev(raw), views, tgt, lr=LR, K_capacity=a.capacity)
    la, lb = [], []
    for _ in range(10):
        a.step_eager()
        la.append(a.loss())
    b.capture()  # two eager steps
    lb += [float("nan")] * 2
    for _ in range(8):
        b.step()
        lb.append(b.loss())
    assert b.steps_taken() == 10 and a.steps_taken() == 10
    np.testing.assert_allclose(la[2:], lb[2:], rtol=1e-3)
    assert la[-1] < la[0]
    for k in RAW:
        assert rel_l2(np_(b.raw[k]) - raw[k], np_(a.raw[k]) - raw[k]) <= 2e-2, k


def test_overflow_skips_updates_and_run_grows_the_capacity():
    w = wl.small_case(43, 800, 64, 64, log_scale_mu=-2.4)
    cam, sc = w.views[0].camera, w.scenes[0]
    raw = _scene_raw(sc)
    views = B.Views([cam], [(0, sc.n)], device="cuda")
    t = Trainer(_dev(raw), views, torch.tensor(w.targets[0].reshape(-1, 3), device="cuda"), lr=LR, K_capacity=50)
    t.step_eager()
    assert t.overflowed() and t.steps_taken() == 0
    np.testing.assert_array_equal(np_(t.raw["means"]), raw["means"])
    t.run(6, check_every=1)
    assert t.capacity > 50 and not t.overflowed()
    assert t.steps_taken() >= 1


def test_checkpoint_resume_continues_the_same_loop(tmp_path):
    # 4 steps, a checkpoint through torch.save, a fresh trainer that loads it and takes 4 more:
    # the same loop as 8 steps in one trainer (up to the backward's fp32 summation order)
    w = wl.small_case(44, 1500, 96, 80, log_scale_mu=-2.6)
    cam, sc = w.views[0].camera, w.scenes[0]
    raw = _scene_raw(sc)
    tgt = torch.tensor(w.targets[0].reshape(-1, 3), device="cuda")
    views = B.Views([cam], [(0, sc.n)], device="cuda")
    a = Trainer(_dev(raw), views, tgt, lr=LR)
    for _ in range(8):
        a.step_eager()
    b = Trainer(_dev(raw), views, tgt, lr=LR, K_capacity=a.capacity)
    for _ in range(4):
        b.step_eager()
    path = tmp_path / "ckpt.pt"
    torch.save(b.state_dict(), path)
    other = {k: v + 1.0 for k, v in _dev(raw).items()}  # different starting values, overwritten by the load
    c = Trainer(other, views, tgt, lr=(0.1,) * 5, K_capacity=a.capacity)
    c.load_state_dict(torch.load(path))
    assert c.steps_taken() == 4
    for _ in range(4):
        c.step_eager()
    assert c.steps_taken() == 8 == a.steps_taken()
    for k in RAW:
        assert rel_l2(np_(c.raw[k]) - raw[k], np_(a.raw[k]) - raw[k]) <= 2e-2, k
    assert c.loss() == pytest.approx(a.loss(), rel=1e-3)
    with pytest.raises(ValueError):
        d = Trainer(_dev({k: v[:-1] for k, v in raw.items()}), B.Views([cam], [(0, sc.n - 1)], device="cuda"), tgt,
                    lr=LR)
        d.load_state_dict(torch.load(path))
