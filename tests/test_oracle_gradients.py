"""Pins of the oracle's analytic backward (Sec. 3) against central finite
differences of the oracle's forward (Sec. 2), stage by stage and end to end,
plus the matrix-calculus rule of Sec. 3 the derivation rests on."""
import numpy as np

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


# -- dL/dT_cw (Eq. 20, Reading O14) -------------------------------------------

def _camera_with(cam, R=None, t=None):
    import dataclasses
    return dataclasses.replace(cam, R=np.array(cam.R if R is None else R, np.float64),
                               t=np.array(cam.t if t is None else t, np.float64))


def _viewmat_fd(cam, loss, h=1e-6):
    """Central differences of ``loss(camera)`` over the 12 entries of [R_cw t_cw]."""
    R0, t0 = np.array(cam.R, np.float64), np.array(cam.t, np.float64)
    fd = np.zeros((4, 4))
    for i in range(3):
        for j in range(4):
            vals = []
            for sgn in (1, -1):
                R, t = R0.copy(), t0.copy()
                if j < 3:
                    R[i, j] += sgn * h
                else:
                    t[i] += sgn * h * max(abs(t0[i]), 1.0)
                vals.append(loss(_camera_with(cam, R, t)))
            fd[i, j] = (vals[0] - vals[1]) / (2 * h * (1.0 if j < 3 else max(abs(t0[i]), 1.0)))
    return fd


def test_view_matrix_gradient_of_projection_matches_finite_differences():
    # L = <A, mu'> + <B, conic> through Eq. 2-6; the camera is rotated and moved so no entry is trivial.
    w = wl.small_case(11, 12, 48, 40, log_scale_mu=-2.0)
    sc = w.scenes[0]
    cam = wl.sphere_cameras(np.random.default_rng(3), 1, 4.0, [(48, 40)], focal=50.0)[0]
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((sc.n, 2)), rng.standard_normal((sc.n, 3))

    def L(c):
        p = oracle.project(c, sc.means, sc.quats, sc.scales, eps2d=0.3)
        return np.sum(A * p["means2d"]) + np.sum(B * p["conics"])

    cam64 = _camera_with(cam)
    p = oracle.project(cam64, sc.means, sc.quats, sc.scales)
    assert p["valid"].all()
    g = oracle.project_bwd(cam64, sc.means, sc.quats, sc.scales, p["valid"], A, B)["viewmat"]
    fd = _viewmat_fd(cam64, L)
    assert not g[3].any()
    assert _rel_err(g, fd) < 1e-6
    # Eq. 20 alone, sum_n (dL/dt_n) [mu_n; 1]^T, gets the translation column but misses the
    # covariance route through R_cw in the rotation block (Reading O14)
    gm = oracle.project_bwd(cam64, sc.means, sc.quats, sc.scales, p["valid"], A, B)["means"]
    gt = gm @ np.array(cam64.R).T  # per-Gaussian dL/dt = R_cw dL/dmu
    assert _rel_err(gt.T @ np.array(sc.means, np.float64), fd[:3, :3]) > 1e-3
    np.testing.assert_allclose(gt.sum(0), fd[:3, 3], rtol=1e-6, atol=1e-9)


def test_view_matrix_gradient_end_to_end_matches_finite_differences():
    w = wl.gradcheck_64_32()
    cam, sc = _camera_with(w.views[0].camera), w.scenes[0]
    G = np.random.default_rng(7).standard_normal((32, 32, 3))
    g = oracle.backward(cam, sc, G)["viewmat"]

    def L(c):
        return float(np.sum(oracle.render(c, sc)["rgb"] * G))

    assert _rel_err(g, _viewmat_fd(cam, L)) < 1e-6


def _quat_mul(a, b):
    """Hamilton product of (w, x, y, z) quaternions."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def test_view_matrix_gradient_satisfies_rigid_motion_invariance():
    # Moving the scene and the camera by the same rigid motion leaves every t, Sigma' and pixel unchanged,
    # so the gradients must cancel along it.  Translation by d: mu -> mu + d, t_cw -> t_cw - R_cw d gives
    # sum_n dL/dmu_n = R_cw^T dL/dt_cw.  Rotation by Q = I + eps [k]x: mu -> Q mu, q -> q_Q (x) q,
    # R_cw -> R_cw Q^T gives sum_n <dL/dmu_n, [k]x mu_n> + <dL/dq_n, (0, k/2) (x) q_n> - <dL/dR_cw, R_cw [k]x> = 0.
    rng = np.random.default_rng(4)
    for _ in range(3):  # the product rule of the helper: R(a (x) b) = R(a) R(b)
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        a, b = a / np.linalg.norm(a), b / np.linalg.norm(b)
        np.testing.assert_allclose(oracle.quat_to_rotmat(_quat_mul(a, b)),
                                   oracle.quat_to_rotmat(a) @ oracle.quat_to_rotmat(b), atol=1e-14)
    w = wl.small_case(17, 150, 64, 48, log_scale_mu=-2.3)
    sc = w.scenes[0]
    cam = _camera_with(wl.sphere_cameras(np.random.default_rng(5), 1, 4.0, [(64, 48)], focal=60.0)[0])
    G = np.random.default_rng(6).standard_normal((48, 64, 3))
    g = oracle.backward(cam, sc, G)
    R = np.array(cam.R, np.float64)
    gV = g["viewmat"]
    scale = np.abs(g["means"]).sum() * 10
    np.testing.assert_allclose(g["means"].sum(0), R.T @ gV[:3, 3], atol=1e-10 * scale)
    mu, q = np.array(sc.means, np.float64), np.array(sc.quats, np.float64)
    for k in np.eye(3):
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        d_means = np.sum(g["means"] * (mu @ Kx.T))
        d_quats = sum(np.dot(g["quats"][n], _quat_mul(np.r_[0.0, 0.5 * k], q[n])) for n in range(sc.n))
        d_cam = -np.sum(gV[:3, :3] * (R @ Kx))
        terms = abs(d_means) + abs(d_quats) + abs(d_cam)
        assert terms > 0
        assert abs(d_means + d_quats + d_cam) < 1e-9 * terms
        # with Eq. 20's rotation block alone (no covariance route, O14) the balance fails
        paper_R = (g["means"] @ R.T).T @ mu
        assert abs(d_means + d_quats - np.sum(paper_R * (R @ Kx))) > 1e-6 * terms
