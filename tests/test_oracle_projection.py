"""Pins of the oracle's projection (Sec. 2.1, Eq. 2-6) against facts that do not
come from the oracle itself: textbook rotations, orthonormality, eigenvalues,
the printed Jacobians of Sec. 3.2 / 3.2.1 checked by finite differences, and
closed forms of special cases."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_02121_gb300 import workloads as wl


def _unit(rng, n=4):
    q = rng.standard_normal(n)
    return q / np.linalg.norm(q)


def test_rotation_is_orthonormal_with_unit_determinant():
    # Eq. 5 as printed (R_11 = 1 - 2(x^2 - z^2)) fails this; the reading O4 passes.
    rng = np.random.default_rng(0)
    for _ in range(50):
        R = oracle.quat_to_rotmat(_unit(rng))
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rotation_about_coordinate_axis_is_textbook(axis):
    # q = (cos(th/2), sin(th/2) e_axis) is the right-handed rotation by th about e_axis.
    th = 0.7345
    q = np.zeros(4)
    q[0] = math.cos(th / 2)
    q[1 + axis] = math.sin(th / 2)
    c, s = math.cos(th), math.sin(th)
    if axis == 0:
        ref = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    elif axis == 1:
        ref = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    else:
        ref = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    np.testing.assert_allclose(oracle.quat_to_rotmat(q), ref, atol=1e-14)


def test_printed_rotation_jacobians_match_finite_differences():
    # The four matrices printed in Sec. 3.2.1 are the derivatives of the
    # polynomial map R(q); this pins R(q) (including the R_11 sign, O4) and the
    # Jacobians against each other.
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        q = _unit(rng)
        jac = oracle.rotmat_jacobians(q)
        for i in range(4):
            dq = np.zeros(4)
            dq[i] = h
            fd = (oracle.quat_to_rotmat(q + dq) - oracle.quat_to_rotmat(q - dq)) / (2 * h)
            np.testing.assert_allclose(jac[i], fd, atol=1e-8)


def test_identity_quaternion_gives_diagonal_covariance():
    s = np.array([0.3, 0.05, 1.7])
    Sig, R, M = oracle.covariance3d([1, 0, 0, 0], s)
    np.testing.assert_allclose(Sig, np.diag(s ** 2), atol=1e-15)
    np.testing.assert_allclose(R, np.eye(3), atol=0)


def test_covariance_eigenvalues_are_squared_scales():
    rng = np.random.default_rng(2)
    for _ in range(20):
        s = np.exp(rng.normal(-1, 1, 3))
        q = rng.standard_normal(4) * 2.5  # unnormalised on purpose (O5)
        Sig, R, M = oracle.covariance3d(q, s)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Sig)), np.sort(s ** 2), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Sig, Sig.T, atol=1e-15)
        # the columns of R are the principal axes: Sigma R e_i = s_i^2 R e_i
        np.testing.assert_allclose(Sig @ R, R * s ** 2, rtol=1e-11, atol=1e-14)


def test_covariance_ignores_quaternion_norm():
    rng = np.random.default_rng(3)
    q, s = rng.standard_normal(4), np.array([0.2, 0.4, 0.1])
    np.testing.assert_allclose(oracle.covariance3d(q, s)[0], oracle.covariance3d(7.3 * q, s)[0], atol=1e-15)


def _cam(w=64, h=48, f=50.0, R=None, t=(0, 0, 4.0)):
    c = wl.camera_at_distance(4.0, w, h, f)
    if R is not None:
        c.R = np.asarray(R, np.float64)
    c.t = np.asarray(t, np.float64)
    c.cx, c.cy = 31.0, 22.5
    return c


def test_pinhole_projection_closed_form():
    cam = _cam()
    t, m2 = oracle.world_to_pixel(cam, [0.0, 0.0, 0.0])
    np.testing.assert_allclose(t, [0, 0, 4.0])
    np.testing.assert_allclose(m2, [cam.cx, cam.cy])
    t, m2 = oracle.world_to_pixel(cam, [0.4, -0.2, 1.0])
    np.testing.assert_allclose(m2, [50.0 * 0.4 / 5.0 + 31.0, 50.0 * -0.2 / 5.0 + 22.5])


def test_ewa_jacobian_is_derivative_of_the_projection():
    # Eq. 3 versus a finite difference of the pinhole map of Eq. 2 (reading O2).
    rng = np.random.default_rng(4)
    R = oracle.quat_to_rotmat(_unit(rng))
    cam = _cam(R=R, t=(0.1, -0.3, 5.0))
    h = 1e-6
    for _ in range(10):
        mu = rng.uniform(-1, 1, 3)
        t, _ = oracle.world_to_pixel(cam, mu)
        J = oracle.ewa_jacobian(cam, t)
        # d mu' / d mu = J R_cw; the finite difference is taken in world space
        fd = np.zeros((2, 3))
        for i in range(3):
            d = np.zeros(3)
            d[i] = h
            fd[:, i] = (oracle.world_to_pixel(cam, mu + d)[1] - oracle.world_to_pixel(cam, mu - d)[1]) / (2 * h)
        np.testing.assert_allclose(J @ R, fd, rtol=1e-7, atol=1e-7)


def test_printed_jacobian_derivatives_match_finite_differences():
    # dJ/dt_x, dJ/dt_y, dJ/dt_z as printed in Sec. 3.2 versus finite differences of Eq. 3.
    cam = _cam(f=60.0)
    cam.fy = 45.0
    h = 1e-6
    for t in ([0.3, -0.2, 2.0], [-1.0, 0.5, 7.0]):
        t = np.array(t)
        dJ = oracle.ewa_jacobian_dt(cam, t)
        for i in range(3):
            d = np.zeros(3)
            d[i] = h
            fd = (oracle.ewa_jacobian(cam, t + d) - oracle.ewa_jacobian(cam, t - d)) / (2 * h)
            np.testing.assert_allclose(dJ[i], fd, rtol=1e-7, atol=1e-9)


def test_projected_covariance_of_isotropic_gaussian_on_axis():
    # On the optical axis J = diag(f/d) (plus zero column) so Sigma' = (f s / d)^2 I (+ eps).
    cam = _cam(f=80.0, t=(0, 0, 0))
    d, s = 4.0, 0.05
    for eps in (0.0, 0.3):
        p = oracle.project(cam, [[0, 0, d]], [[1, 0, 0, 0]], [[s, s, s]], eps2d=eps)
        ref = (80.0 * s / d) ** 2 + eps
        np.testing.assert_allclose(p["cov2d"][0], [ref, 0.0, ref], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(p["conics"][0], [1 / ref, 0.0, 1 / ref], rtol=1e-13)


def test_projected_covariance_is_linearised_pushforward():
    # Sigma' = D Sigma D^T with D = d mu'/d mu, taken here by finite differences
    # of the pinhole map -- an independent route to J R_cw of Eq. 4.
    rng = np.random.default_rng(5)
    R = oracle.quat_to_rotmat(_unit(rng))
    cam = _cam(R=R, t=(0.2, 0.1, 6.0))
    h = 1e-6
    for _ in range(8):
        mu = rng.uniform(-1, 1, 3)
        q = rng.standard_normal(4)
        s = np.exp(rng.normal(-2, 0.5, 3))
        D = np.zeros((2, 3))
        for i in range(3):
            dd = np.zeros(3)
            dd[i] = h
            D[:, i] = (oracle.world_to_pixel(cam, mu + dd)[1] - oracle.world_to_pixel(cam, mu - dd)[1]) / (2 * h)
        Sig = oracle.covariance3d(q, s)[0]
        ref = D @ Sig @ D.T
        p = oracle.project(cam, [mu], [q], [s], eps2d=0.0)
        got = np.array([[p["cov2d"][0, 0], p["cov2d"][0, 1]], [p["cov2d"][0, 1], p["cov2d"][0, 2]]])
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
        Y = np.array([[p["conics"][0, 0], p["conics"][0, 1]], [p["conics"][0, 1], p["conics"][0, 2]]])
        np.testing.assert_allclose(Y @ got, np.eye(2), atol=1e-10)


def test_tile_rectangle_of_known_gaussian():
    # Sigma' = (4 px)^2 I at mu' = (64.5, 40.5): the 3-sigma box is [52.5, 76.5] x [28.5, 52.5],
    # i.e. tiles x in {3, 4}, y in {1, 2, 3} of a 16-pixel grid.
    cam = wl.camera_at_distance(0.0, 160, 96, 80.0)
    cam.t = np.zeros(3)
    cam.cx, cam.cy = 64.5, 40.5
    d = 4.0
    s = 4.0 * d / 80.0
    p = oracle.project(cam, [[0, 0, d]], [[1, 0, 0, 0]], [[s, s, s]], eps2d=0.0)
    assert p["valid"][0] == 1
    np.testing.assert_array_equal(p["rects"][0], [3, 1, 5, 4])
    # nearest tile boundary to any box edge: 76.5 -> 80 and 28.5 -> 32, both 3.5 px
    np.testing.assert_allclose(p["rect_margin"][0], 3.5, atol=1e-9)


def test_tile_rectangle_clamps_to_image_and_culls_offscreen():
    cam = wl.camera_at_distance(0.0, 40, 20, 80.0)  # 3 x 2 tiles, ragged
    cam.t = np.zeros(3)
    d, s = 4.0, 0.5  # sigma' = 10 px -> a box far larger than the image
    p = oracle.project(cam, [[0, 0, d], [100.0, 0, d]], [[1, 0, 0, 0]] * 2, [[s, s, s]] * 2, eps2d=0.0)
    np.testing.assert_array_equal(p["rects"][0], [0, 0, 3, 2])
    assert p["valid"].tolist() == [1, 0]


def test_near_far_and_behind_camera_are_culled():
    cam = wl.camera_at_distance(0.0, 64, 64, 64.0, near=0.5, far=10.0)
    cam.t = np.zeros(3)
    means = [[0, 0, 0.4], [0, 0, 11.0], [0, 0, -3.0], [0, 0, 5.0]]
    p = oracle.project(cam, means, [[1, 0, 0, 0]] * 4, [[0.05] * 3] * 4)
    assert p["valid"].tolist() == [0, 0, 0, 1]
