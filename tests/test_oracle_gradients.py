"""Pins of the oracle's analytic backward (Sec. 3) against central finite
differences of the oracle's forward (Sec. 2), stage by stage and end to end,
plus the matrix-calculus rule of Sec. 3 the derivation rests on."""
import numpy as np
import pytest

import oracle
from paper_2312_02121_gb300 import workloads as wl


def test_frobenius_chain_rule():
    # Sec. 3: for X = A Y and f = <G, X>, df/dA = G Y^T and df/dY = A^T G.
    rng = np.random.default_rng(0)
    A, Y, G = rng.standard_normal((3, 4)), rng.standard_normal((4, 2)), rng.standard_normal((3, 2))
    f = lambda A_, Y_: np.sum(G * (A_ @ Y_))
    h = 1e-6
    dA = np.zeros_like(A)
    for i in np.ndindex(A.shape):
        E = np.zeros_like(A)
        E[i] = h
        dA[i] = (f(A + E, Y) - f(A - E, Y)) / (2 * h)
    dY = np.zeros_like(Y)
    for i in np.ndindex(Y.shape):
        E = np.zeros_like(Y)
        E[i] = h
        dY[i] = (f(A, Y + E) - f(A, Y - E)) / (2 * h)
    np.testing.assert_allclose(dA, G @ Y.T, atol=1e-8)
    np.testing.assert_allclose(dY, A.T @ G, atol=1e-8)


def _rel_err(a, b):
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_projection_gradients_match_finite_differences():
    # Sec. 3.2 / 3.2.1: L = <A, mu'> + <B, conic> through Eq. 2-6; every input of every Gaussian.
    w = wl.small_case(11, 12, 48, 40, log_scale_mu=-2.0)
    cam, sc = w.views[0].camera, w.scenes[0]
    rng = np.random.default_rng(1)
    A = rng.standard_normal((sc.n, 2))
    B = rng.standard_normal((sc.n, 3))
    means, quats, scales = (np.array(getattr(sc, k), float) for k in ("means", "quats", "scales"))
    quats = quats * rng.uniform(0.5, 2.0, (sc.n, 1))  # unnormalised quaternions (O5)

    def L(m, q, s):
        p = oracle.project(cam, m, q, s, eps2d=0.3)
        return np.sum(A * p["means2d"]) + np.sum(B * p["conics"])

    p = oracle.project(cam, means, quats, scales)
    assert p["valid"].all()
    g = oracle.project_bwd(cam, means, quats, scales, p["valid"], A, B, eps2d=0.3)
    for name, arr, got in (("means", means, g["means"]), ("quats", quats, g["quats"]), ("scales", scales, g["scales"])):
        fd = np.zeros_like(arr)
        for i in np.ndindex(arr.shape):
            h = 1e-6 * max(abs(arr[i]), 1e-2)
            plus, minus = arr.copy(), arr.copy()
            plus[i] += h
            minus[i] -= h
            args = {"means": means, "quats": quats, "scales": scales}
            args[name] = plus
            lp = L(args["means"], args["quats"], args["scales"])
            args[name] = minus
            lm = L(args["means"], args["quats"], args["scales"])
            fd[i] = (lp - lm) / (2 * h)
        assert _rel_err(got, fd) < 1e-7, name


def test_compositing_gradients_match_finite_differences():
    # Sec. 3.1: gradients w.r.t. the 2D parameters (mu', packed conic, o, c) with a background.
    w = wl.small_case(21, 40, 32, 32, log_scale_mu=-2.0, opacity_logit_mu=0.5)
    cam, sc = w.views[0].camera, w.scenes[0]
    proj = oracle.project(cam, sc.means, sc.quats, sc.scales)
    op, col = sc.opacities.astype(float), sc.colors.astype(float)
    bg = np.array([0.3, 0.2, 0.1])
    G = np.random.default_rng(2).standard_normal((32, 32, 3))
    base = oracle.rasterize(proj, op, col, 32, 32, background=bg)
    assert base["margin"].min() > 1e-4 and base["n_contrib"].max() >= 3
    g = oracle.rasterize_bwd(proj, op, col, 32, 32, G, background=bg)

    def L(proj_, op_, col_):
        return np.sum(G * oracle.rasterize(proj_, op_, col_, 32, 32, background=bg)["rgb"])

    checks = {"means2d": proj["means2d"], "conics": proj["conics"], "opacities": op, "colors": col}
    for name, arr in checks.items():
        fd = np.zeros_like(arr)
        for i in np.ndindex(arr.shape):
            h = 1e-7 * max(abs(arr[i]), 1e-2)
            vals = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2[i] += sgn * h
                pj, o2, c2 = dict(proj), op, col
                if name in ("means2d", "conics"):
                    pj[name] = a2
                elif name == "opacities":
                    o2 = a2
                else:
                    c2 = a2
                vals.append(L(pj, o2, c2))
            fd[i] = (vals[0] - vals[1]) / (2 * h)
        assert _rel_err(g[name], fd) < 1e-6, name


def test_end_to_end_gradients_match_finite_differences():
    # The whole path of Sec. 2 differentiated as in Sec. 3, on the 64-Gaussian 32x32 case.
    w = wl.gradcheck_64_32()
    cam, sc = w.views[0].camera, w.scenes[0]
    fwd = oracle.render(cam, sc)
    assert fwd["margin"].min() > 1e-4 and fwd["proj"]["rect_margin"].min() > 1e-3
    G = np.random.default_rng(7).standard_normal((32, 32, 3))
    g = oracle.backward(cam, sc, G)
    rng = np.random.default_rng(8)
    visible = np.nonzero(fwd["proj"]["valid"])[0]
    for name, shape in (("means", 3), ("quats", 4), ("scales", 3), ("opacities", None), ("colors", 3)):
        idx = rng.choice(visible, 12, replace=False)
        got, fd = [], []
        for n in idx:
            for j in (range(shape) if shape else [None]):
                ix = (n,) if j is None else (n, j)
                fd.append(oracle.finite_difference(cam, sc, G, name, ix, h=1e-6))
                got.append(g[name][ix])
        assert _rel_err(got, fd) < 1e-6, name


def test_culled_gaussians_get_zero_gradient():
    w = wl.small_case(13, 20, 32, 32)
    cam, sc = w.views[0].camera, w.scenes[0]
    means = np.array(sc.means, float)
    means[0] = [0, 0, -10.0]  # behind the camera
    p = oracle.project(cam, means, sc.quats, sc.scales)
    assert p["valid"][0] == 0
    g = oracle.project_bwd(cam, means, sc.quats, sc.scales, p["valid"], np.ones((20, 2)), np.ones((20, 3)))
    assert not g["means"][0].any() and not g["quats"][0].any() and not g["scales"][0].any()
