"""Pins of the FP64 training-step reference (``oracle.optim``): the L2 loss by
closed form and finite differences, the activations by closed form and
their chain rule by finite differences, and Adam against torch.optim.Adam on the CPU (the library
routine the textbook algorithm reduces to)."""
import numpy as np
import pytest

from oracle import optim


def test_l2_loss_closed_form_and_gradient():
    rgb, tgt = np.full((4, 5, 3), 0.5), np.full((4, 5, 3), 0.25)
    L, g = optim.l2_loss(rgb, tgt, 1.0 / rgb.size)
    assert L == pytest.approx(0.0625, rel=1e-15)
    np.testing.assert_allclose(g, 2 * 0.25 / rgb.size)
    rng = np.random.default_rng(0)
    a, b = rng.uniform(size=7), rng.uniform(size=7)
    L, g = optim.l2_loss(a, b, 0.3)
    h = 1e-7
    for i in range(7):
        e = np.zeros(7)
        e[i] = h
        fd = (optim.l2_loss(a + e, b, 0.3)[0] - optim.l2_loss(a - e, b, 0.3)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-7)


def _raw(rng, n):
    return dict(means=rng.standard_normal((n, 3)), quats=rng.standard_normal((n, 4)),
                log_scales=rng.normal(-3, 0.5, (n, 3)), opacity_logits=rng.standard_normal(n),
                colors=rng.uniform(size=(n, 3)))


def test_activations_closed_form():
    # exp of the log-scales; the logistic sigmoid: sigmoid(0) = 1/2, sigmoid(ln 3) = 3/4,
    # sigmoid(-x) = 1 - sigmoid(x).  (1 / (1 - e^-x) also has derivative o (1 - o), so
    # the chain-rule check below alone would not tell it from the sigmoid.)
    x = np.array([0.0, np.log(3.0), -np.log(3.0), 2.0])
    s, o = optim.activate(dict(log_scales=np.log([[0.5, 2.0, 1e-3]]), opacity_logits=x))
    np.testing.assert_allclose(s, [[0.5, 2.0, 1e-3]], rtol=1e-15)
    np.testing.assert_allclose(o[:3], [0.5, 0.75, 0.25], rtol=1e-15)
    assert o[3] == pytest.approx(1.0 - optim.activate(dict(log_scales=np.zeros(1), opacity_logits=-x[3:]))[1][0],
                                 rel=1e-15)


def test_activation_chain_rule_matches_finite_differences():
    rng = np.random.default_rng(1)
    raw = _raw(rng, 5)
    A, B = rng.standard_normal((5, 3)), rng.standard_normal(5)

    def L(r):  # a loss of the activated values
        s, o = optim.activate(r)
        return np.sum(A * s) + np.sum(B * o)

    s, o = optim.activate(raw)
    g = optim.raw_gradients(raw, dict(means=np.zeros((5, 3)), quats=np.zeros((5, 4)), scales=A, opacities=B,
                                      colors=np.zeros((5, 3))))
    h = 1e-6
    for key in ("log_scales", "opacity_logits"):
        for idx in np.ndindex(raw[key].shape):
            p, m = {k: v.copy() for k, v in raw.items()}, {k: v.copy() for k, v in raw.items()}
            p[key][idx] += h
            m[key][idx] -= h
            # L is O(1), so the difference quotient carries ~1e-10 of rounding
            assert g[key][idx] == pytest.approx((L(p) - L(m)) / (2 * h), rel=1e-6, abs=1e-9)


def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    raw = _raw(rng, 6)
    lr = (1e-3, 2e-3, 5e-3, 5e-2, 2.5e-3)
    ref = optim.Adam(raw, lr, beta1=0.9, beta2=0.99, eps=1e-10)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in raw.items()}
    topt = torch.optim.Adam([{"params": [tp[k]], "lr": l} for k, l in zip(optim.GROUPS, lr)], betas=(0.9, 0.99),
                            eps=1e-10)
    cur = {k: v.copy() for k, v in raw.items()}
    for step in range(5):
        g = {k: rng.standard_normal(v.shape) for k, v in raw.items()}
        cur = ref.step(cur, g)
        topt.zero_grad()
        for k in optim.GROUPS:
            tp[k].grad = torch.tensor(g[k], dtype=torch.float64)
        topt.step()
        for k in optim.GROUPS:
            np.testing.assert_allclose(cur[k], tp[k].detach().numpy(), rtol=1e-13, atol=1e-15)
