"""FP64 reference of the training-step helpers: the L2 image loss and one Adam
step on the raw Gaussian parameters with their activations.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the tests and the
benchmark's CPU leg may use it; the CUDA library never does.  The paper
derives gradients only.  The loss is the plain mean of squared differences.
Adam follows Kingma & Ba (2015, Algorithm 1): bias-corrected first and second
moments.  The activations are scale = exp(log-scale) and opacity =
sigmoid(logit).
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

GROUPS = ("means", "quats", "log_scales", "opacity_logits", "colors")


def l2_loss(rgb, target, inv_norm: float) -> Tuple[float, np.ndarray]:
    """L = inv_norm * sum (rgb - target)^2 and dL/drgb = 2 inv_norm (rgb - target)."""
    d = np.asarray(rgb, np.float64) - np.asarray(target, np.float64)
    return float(inv_norm * np.sum(d * d)), 2.0 * inv_norm * d


def activate(raw: Dict[str, np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """(scales, opacities) = (exp(log_scales), sigmoid(opacity_logits))."""
    return np.exp(np.asarray(raw["log_scales"], np.float64)), \
        1.0 / (1.0 + np.exp(-np.asarray(raw["opacity_logits"], np.float64)))


def raw_gradients(raw: Dict[str, np.ndarray], grads: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Gradients with respect to the raw parameters, given those with respect
    to the activated values the renderer consumed (means, quats, scales,
    opacities, colors): d/dlog s = s d/ds, d/dlogit = o (1 - o) d/do."""
    s, o = activate(raw)
    return dict(means=np.asarray(grads["means"], np.float64), quats=np.asarray(grads["quats"], np.float64),
                log_scales=s * np.asarray(grads["scales"], np.float64),
                opacity_logits=o * (1.0 - o) * np.asarray(grads["opacities"], np.float64),
                colors=np.asarray(grads["colors"], np.float64))


class Adam:
    """Adam of Kingma & Ba on the five raw parameter groups, one learning rate
    per group (means, quats, log_scales, opacity_logits, colors)."""

    def __init__(self, raw: Dict[str, np.ndarray], lr, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        self.lr = dict(zip(GROUPS, lr))
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.m = {k: np.zeros_like(np.asarray(raw[k], np.float64)) for k in GROUPS}
        self.v = {k: np.zeros_like(np.asarray(raw[k], np.float64)) for k in GROUPS}
        self.t = 0

    def step(self, raw: Dict[str, np.ndarray], g_raw: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
        """Returns the updated raw parameters (new arrays)."""
        self.t += 1
        b1, b2 = self.beta1, self.beta2
        out = {}
        for k in GROUPS:
            g = np.asarray(g_raw[k], np.float64)
            self.m[k] = b1 * self.m[k] + (1 - b1) * g
            self.v[k] = b2 * self.v[k] + (1 - b2) * g * g
            m_hat = self.m[k] / (1 - b1 ** self.t)
            v_hat = self.v[k] / (1 - b2 ** self.t)
            out[k] = np.asarray(raw[k], np.float64) - self.lr[k] * m_hat / (np.sqrt(v_hat) + self.eps)
        return out
