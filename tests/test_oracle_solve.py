"""Pins of the oracle's linearisation (Eq. 2, 3), regularised solve (Eq. 4, 5) and update."""
import math

import numpy as np
import pytest

from oracle import kf_oracle as O


def _random_rows(rng, m=200):
    p = rng.normal(size=(m, 3)) + np.array([0, 0, 2.0])
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    q = p + 0.01 * rng.normal(size=(m, 3))
    return p, q, n


def test_rows_reproduce_the_small_angle_transform_of_eq2():
    rng = np.random.default_rng(1)
    p, q, n = _random_rows(rng)
    a, b = O.ls_rows(p, q, n)
    al, be, ga, tx, ty, tz = x = 1e-3 * rng.normal(size=6)
    M = np.array([[1.0, -ga, be, tx],
                  [ga, 1.0, -al, ty],
                  [-be, al, 1.0, tz]])          # Eq. 2, entry by entry
    Mp = p @ M[:, :3].T + M[:, 3]
    r = np.einsum("ik,ik->i", Mp - q, n)        # point-to-plane residual of Eq. 1
    assert np.allclose(a @ x - b, r, atol=1e-14)


def test_eq5_is_the_normal_equations_of_the_stacked_least_squares():
    rng = np.random.default_rng(2)
    p, q, n = _random_rows(rng)
    a, b = O.ls_rows(p, q, n)
    AtA, Atb, _ = O.normal_equations(a, b)
    for lam in (0.0, 0.3, 5.0, 1e3):
        m = len(b)
        Hs, g = O.regularised_system(AtA, Atb, lam, m)
        x = O.cholesky_solve(Hs, g)
        P = np.hstack([np.eye(3), np.zeros((3, 3))])
        As = np.vstack([a, math.sqrt(2 * lam * m) * P])
        bs = np.concatenate([b, np.zeros(3)])
        xl = np.linalg.lstsq(As, bs, rcond=None)[0]
        assert np.allclose(x, xl, rtol=1e-9, atol=1e-13)


def test_eq5_minimises_the_regularised_objective_of_eq4():
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    p, q, n = _random_rows(rng, 80)
    a, b = O.ls_rows(p, q, n)
    m, lam = len(b), 0.7
    P = np.hstack([np.eye(3), np.zeros((3, 3))])
    f = lambda x: (0.5 / m) * np.sum((a @ x - b) ** 2) + lam * np.sum((P @ x) ** 2)
    res = opt.minimize(f, np.zeros(6), method="BFGS", options={"gtol": 1e-14, "maxiter": 10000})
    AtA, Atb, _ = O.normal_equations(a, b)
    x = O.cholesky_solve(*O.regularised_system(AtA, Atb, lam, m))
    assert np.allclose(x, res.x, atol=1e-7)
    grad = (1.0 / m) * a.T @ (a @ x - b) + 2 * lam * P.T @ P @ x
    assert np.abs(grad).max() < 1e-12


def test_cholesky_solve_matches_numpy_and_flags_rank_deficiency():
    rng = np.random.default_rng(4)
    B = rng.normal(size=(6, 6))
    Hm = B @ B.T + 0.1 * np.eye(6)
    g = rng.normal(size=6)
    assert np.allclose(O.cholesky_solve(Hm, g), np.linalg.solve(Hm, g), rtol=1e-10)
    # single plane: rows [p x n, n] with one n span only 3 dimensions
    p = np.c_[rng.normal(size=(100, 2)), np.full(100, 2.0)]
    n = np.tile([0.0, 0.0, -1.0], (100, 1))
    a, b = O.ls_rows(p, p, n)
    AtA, Atb, _ = O.normal_equations(a, b)
    assert O.cholesky_solve(*O.regularised_system(AtA, Atb, 0.0, 100)) is None
    assert O.cholesky_solve(*O.regularised_system(AtA, Atb, 5.0, 100)) is None


def test_rodrigues_matches_scipy_rotation():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(5)
    for s in (1e-14, 1e-6, 1e-2, 0.5, 3.0):
        w = s * rng.normal(size=3)
        assert np.allclose(O.rodrigues(w), Rot.from_rotvec(w).as_matrix(), atol=1e-15)


def test_apply_increment_composes_on_the_left():
    rng = np.random.default_rng(6)
    T = np.eye(4)
    T[:3, :3] = O.rodrigues(rng.normal(size=3))
    T[:3, 3] = rng.normal(size=3)
    x = np.r_[0.01, -0.02, 0.03, 0.1, 0.2, -0.3]
    T2 = O.apply_increment(x, T)
    v = rng.normal(size=3)
    p = T[:3, :3] @ v + T[:3, 3]
    assert np.allclose(T2[:3, :3] @ v + T2[:3, 3], O.rodrigues(x[:3]) @ p + x[3:], atol=1e-14)


def test_lambda_schedules():
    assert O.lambda_of_n(O.LAMBDA_CONST, 5.0, 100) == 5.0
    assert O.lambda_of_n(O.LAMBDA_C_SQRT_N, 5.0, 100) == pytest.approx(0.5)
    assert O.lambda_of_n(O.LAMBDA_C_N, 5.0, 100) == pytest.approx(0.05)
    assert O.lambda_of_n(O.LAMBDA_C_N2, 5.0, 100) == pytest.approx(5e-4)
    assert O.lambda_of_n(O.LAMBDA_C_LOG_N, 5.0, 100) == pytest.approx(5.0 * math.log(100))


def test_relative_pose_is_the_inverse_composition():
    rng = np.random.default_rng(8)
    Ts = []
    for _ in range(2):
        T = np.eye(4)
        T[:3, :3] = O.rodrigues(rng.normal(size=3))
        T[:3, 3] = rng.normal(size=3)
        Ts.append(T)
    R, t = O.relative_pose(Ts[0], Ts[1])
    Tr = np.linalg.inv(Ts[1]) @ Ts[0]
    assert np.allclose(R, Tr[:3, :3], atol=1e-14) and np.allclose(t, Tr[:3, 3], atol=1e-14)


def test_rotation_log_inverts_rodrigues_and_matches_scipy():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(11)
    for ang in [0.0, 1e-9, 1e-5, 2e-4, 0.05, 0.7, 2.0, 3.0]:
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        w = ang * axis
        R = O.rodrigues(w)
        got = O.rotation_log(R)
        assert np.allclose(got, w, atol=1e-12), ang
        assert np.allclose(got, Rot.from_matrix(R).as_rotvec(), atol=1e-12), ang


def test_anchored_system_minimises_its_objective():
    """Prior-anchored variant: x minimises (1/2m)|A x - b|^2 + lambda |P x + r|^2
    with r = log(R_cur R_prior^T); gradient zero, and BFGS agrees."""
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(5)
    p, q, n = _random_rows(rng, 60)
    a, b = O.ls_rows(p, q, n)
    m, lam = len(b), 0.4
    Rc = O.rodrigues([0.02, -0.03, 0.01])
    Rp = O.rodrigues([-0.01, 0.02, 0.015])
    r = O.rotation_log(Rc @ Rp.T)
    P = np.hstack([np.eye(3), np.zeros((3, 3))])
    AtA, Atb, _ = O.normal_equations(a, b)
    Hs, _ = O.regularised_system(AtA, Atb, lam, m)
    x = O.cholesky_solve(Hs, O.anchored_rhs(Atb, lam, m, Rc, Rp))
    grad = (1.0 / m) * a.T @ (a @ x - b) + 2 * lam * P.T @ (P @ x + r)
    assert np.abs(grad).max() < 1e-12
    f = lambda y: (0.5 / m) * np.sum((a @ y - b) ** 2) + lam * np.sum((P @ y + r) ** 2)
    res = opt.minimize(f, np.zeros(6), method="BFGS", options={"gtol": 1e-14, "maxiter": 10000})
    assert np.allclose(x, res.x, atol=1e-7)
