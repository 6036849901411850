"""The fp64 instantiation of the CUDA path: equal to the FP64 oracle to
round-off, and its analytic backward (behind the torch.autograd.Function)
passes torch.autograd.gradcheck against finite differences on the
64-Gaussian 32x32 case (seed 1: every threshold test at least 5e-4 from its
threshold, so the finite-difference step never crosses one)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2312_02121_gb300 import autograd as ga
from paper_2312_02121_gb300 import workloads as wl
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

KEYS = ("means", "quats", "scales", "opacities", "colors")


def _leaves(sc, requires_grad=True):
    return [torch.tensor(np.asarray(getattr(sc, k), np.float64), device="cuda", requires_grad=requires_grad)
            for k in KEYS]


def test_fp64_path_equals_oracle_to_roundoff():
    w = wl.gradcheck_64_32()
    cam, sc = w.views[0].camera, w.scenes[0]
    leaves = _leaves(sc)
    img = ga.render(*leaves, [cam], eps2d=w.eps2d)[0]
    G = np.random.default_rng(0).standard_normal((32, 32, 3))
    (img * torch.tensor(G, device="cuda")).sum().backward()
    o = oracle.render(cam, sc, w.eps2d)
    assert np.abs(img.detach().cpu().numpy() - o["rgb"]).max() <= 1e-12
    ob = oracle.backward(cam, sc, G, w.eps2d)
    for k, leaf in zip(KEYS, leaves):
        assert rel_l2(leaf.grad.cpu().numpy(), ob[k]) <= 1e-10, k


def test_autograd_gradcheck_fp64():
    w = wl.gradcheck_64_32()
    cam, sc = w.views[0].camera, w.scenes[0]
    leaves = _leaves(sc)
    W = torch.tensor(np.random.default_rng(1).standard_normal((32, 32, 3)), device="cuda")

    def loss(*p):
        return (ga.render(*p, [cam], eps2d=w.eps2d)[0] * W).sum()

    # per-Gaussian sums use atomics, so repeated backwards differ at round-off
    assert torch.autograd.gradcheck(loss, tuple(leaves), eps=1e-6, atol=1e-8, rtol=1e-5, nondet_tol=1e-12)


def test_fp64_view_matrix_gradient_equals_oracle():
    # dL/dT_cw through autograd (viewmats leaf) on a rotated camera; the camera reaches the GPU in fp32,
    # so the oracle is given the same fp32-rounded pose
    w = wl.gradcheck_64_32()
    sc = w.scenes[0]
    cam = wl.sphere_cameras(np.random.default_rng(2), 1, 3.0, [(32, 32)], focal=30.0)[0]
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)
    vm = torch.tensor(T[None], device="cuda", requires_grad=True)
    leaves = _leaves(sc)
    img = ga.render(*leaves, [cam], eps2d=w.eps2d, viewmats=vm)[0]
    G = np.random.default_rng(3).standard_normal((32, 32, 3))
    (img * torch.tensor(G, device="cuda")).sum().backward()
    ob = oracle.backward(cam, sc, G, w.eps2d)
    o = oracle.render(cam, sc, w.eps2d)
    assert np.abs(img.detach().cpu().numpy() - o["rgb"]).max() <= 1e-12
    assert rel_l2(vm.grad[0].cpu().numpy(), ob["viewmat"]) <= 1e-10
    for k, leaf in zip(KEYS, leaves):
        assert rel_l2(leaf.grad.cpu().numpy(), ob[k]) <= 1e-10, k
