"""Pins of the oracle's integral-image normals and normal-shooting association
(the normal estimation and association the paper names in Sec. 3.3).

Each test checks the oracle against something other than itself: a library
routine (scipy's chessboard distance transform and correlation), analytic
plane and sphere geometry, brute force over the candidate window with a
different distance formula, or the geometry of a plane seen through a shifted
camera.
"""
import math

import numpy as np
import pytest

from oracle import kf_normals as NI
from oracle import kf_oracle as O
from synth import scenes as S

F32 = np.float32


def angle_deg(A, b):
    """Angles between the rows of A and b (atan2 form: exact near 0)."""
    A = np.asarray(A, np.float64)
    b = np.broadcast_to(np.asarray(b, np.float64), A.shape)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(A, b), axis=-1), np.einsum("ij,ij->i", A, b)))


def plane_depth(W, H, fx, fy, cx, cy, n, d):
    """Depth of the plane n . X = d seen from the origin (camera frame)."""
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    den = n[0] * (u - cx) / fx + n[1] * (v - cy) / fy + n[2]
    return (d / den).astype(F32)


@pytest.mark.parametrize("density,shape", [(0.002, (37, 53)), (0.02, (40, 31)), (0.2, (17, 64))])
def test_chessboard_distance_matches_scipy(density, shape):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(7)
    E = rng.random(shape) < density
    E[rng.integers(shape[0]), rng.integers(shape[1])] = True
    cap = 9
    ref = ndimage.distance_transform_cdt(~E, metric="chessboard")
    assert np.array_equal(NI.chessboard_distance(E, cap), np.minimum(ref, cap))


@pytest.mark.parametrize("r", [1, 2, 5])
def test_window_gradients_match_correlation(r):
    # g_h and g_v are correlations of Q with a (2r+1)^2 kernel of -1 left /
    # up of the centre line, +1 right / below it, 0 on it (zero outside)
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(r)
    Q = rng.integers(-10**6, 10**6, size=(23, 29, 3)).astype(np.int64)
    kh = np.zeros((2 * r + 1, 2 * r + 1))
    kh[:, r + 1:] = 1
    kh[:, :r] = -1
    kv = kh.T.copy()
    gh, gv = NI.gradients(Q, r)
    for c in range(3):
        Qc = Q[..., c].astype(np.float64)  # sums stay below 2^53: exact
        assert np.array_equal(gh[..., c], ndimage.correlate(Qc, kh, mode="constant").astype(np.int64))
        assert np.array_equal(gv[..., c], ndimage.correlate(Qc, kv, mode="constant").astype(np.int64))


@pytest.mark.parametrize("n,d", [((0.0, 0.0, -1.0), -2.0), ((0.3, -0.2, -0.93), -2.2),
                                 ((-0.5, 0.1, -0.86), -1.8)])
def test_plane_normals_match_plane(n, d):
    n = np.array(n) / np.linalg.norm(n)
    W, H, f = 96, 72, 80.0
    D = plane_depth(W, H, f, f, 47.5, 35.5, n, d)
    V, N = NI.integral_normals(D, f, f, 47.5, 35.5, 0)
    ok = np.isfinite(N).all(-1)
    r = NI.window_radius(D, 0, 2.0, 1.0, 0.02, 8)
    assert ok.sum() > 0.8 * W * H
    assert np.array_equal(ok, r >= 1)
    # the plane's normal faces the camera: sign such that n . X = d < 0
    want = n if d < 0 else -n
    assert angle_deg(N[ok], want).max() < 2e-3
    assert np.all(np.einsum("ij,ij->i", N[ok].astype(np.float64), V[ok].astype(np.float64)) < 0)


def test_radius_follows_depth_and_level():
    W, H = 64, 48
    for z, level, want in ((2.0, 0, 4), (2.0, 1, 2), (2.0, 2, 1), (3.5, 0, 5), (9.0, 0, 8)):
        D = np.full((H, W), z, F32)
        r = NI.window_radius(D, level, 2.0, 1.0, 0.02, 8)
        assert r[H // 2, W // 2] == want
        # the border limits the window: r = distance to the border near it
        assert r[1, W // 2] == min(1, want) and r[H // 2, 0] == 0


def test_depth_step_shrinks_windows_and_drops_edge_pixels():
    W, H = 60, 40
    D = np.full((H, W), 2.0, F32)
    D[:, 30:] = 2.5                      # a 50 cm step, far above delta z
    V, N = NI.integral_normals(D, 50.0, 50.0, 29.5, 19.5, 0)
    r = NI.window_radius(D, 0, 2.0, 1.0, 0.02, 8)
    row = H // 2
    # columns 29 and 30 are edges; 28 and 31 have a window of 0 (no normal);
    # further away the window grows by one per column up to the depth cap
    assert [int(r[row, x]) for x in range(24, 36)] == [4, 3, 2, 1, 0, -1, -1, 0, 1, 2, 3, 4]
    okrow = np.isfinite(N[row]).all(-1)
    assert not okrow[28:32].any() and okrow[20:28].all() and okrow[32:40].all()
    assert np.allclose(N[row, 20:28], [0, 0, -1], atol=1e-6)
    assert np.allclose(N[row, 32:40], [0, 0, -1], atol=1e-6)


def test_windows_hold_no_hole_or_edge():
    rng = np.random.default_rng(3)
    W, H = 48, 36
    D = plane_depth(W, H, 40.0, 40.0, 23.5, 17.5, np.array([0.2, 0.1, -0.97]) / 1.0, -2.0)
    D[rng.random((H, W)) < 0.02] = 0.0
    D[10:20, 5:9] = 1.2                   # an object in front
    E = NI.edge_map(D, 0.02)
    r = NI.window_radius(D, 0, 2.0, 1.0, 0.02, 8)
    for y in range(H):
        for x in range(W):
            if r[y, x] >= 1:
                rr = r[y, x]
                win = E[y - rr:y + rr + 1, x - rr:x + rr + 1]
                assert win.shape == (2 * rr + 1, 2 * rr + 1) and not win.any()
                # maximal: one more row/column would hit an edge, the border or a cap
                bigger = E[max(0, y - rr - 1):y + rr + 2, max(0, x - rr - 1):x + rr + 2]
                capped = rr == 8 or rr == math.floor(2.0 + 1.0 * float(D[y, x]))
                border = min(x, y, W - 1 - x, H - 1 - y) == rr
                assert bigger.any() or capped or border


def test_sphere_normals_are_radial():
    sc = S.Scene(planes=[((0.0, 0.0, -1.0), -3.0)], spheres=[((0.0, 0.0, 2.0), 0.5)])
    K = S.Intrinsics(128, 96, 110.0, 110.0, 63.5, 47.5)
    D = S.render_depth(sc, np.eye(4), K, None, noise=False)
    V, N = NI.integral_normals(D, K.fx, K.fy, K.cx, K.cy, 0)
    ok = np.isfinite(N).all(-1)
    on_sphere = ok & (np.linalg.norm(V.astype(np.float64) - [0, 0, 2.0], axis=-1) < 0.5 + 1e-3)
    assert on_sphere.sum() > 500
    radial = (V[on_sphere].astype(np.float64) - [0, 0, 2.0]) / 0.5
    # the window averages the gradient over up to 2r+1 = 9 pixels (~4 cm) of a
    # 0.5 m sphere: the normal stays within a few degrees of the radius
    assert angle_deg(N[on_sphere], radial).max() < 6.0


def test_integral_mode_in_the_pyramid():
    p = O.Params(normal_mode=O.NORMALS_INTEGRAL)
    K = O.Cam(64, 48, 50.0, 50.0, 31.5, 23.5)
    D = plane_depth(64, 48, 50.0, 50.0, 31.5, 23.5, np.array([0.0, 0.0, -1.0]), -2.0).astype(np.float64)
    levels = O.build_frame_pyramid(D, K, p)
    for l, fl in enumerate(levels):
        ok = np.isfinite(fl.N).all(-1)
        assert np.array_equal(ok, np.isfinite(fl.V).all(-1))
        assert ok.any()
        assert np.allclose(fl.N[ok], [0, 0, -1], atol=1e-6)


# ---------------------------------------------------------------------------
# normal shooting
# ---------------------------------------------------------------------------
def _levels(D, K, p):
    fl = O.build_frame_pyramid(np.asarray(D, np.float64), K, p)[0]
    return fl


def test_shooting_at_identity_equals_projective():
    # model = the frame's own maps, pose = identity: p = q exactly at the
    # projected pixel (line distance 0), so shooting keeps the projection
    # unless an earlier candidate lies on the normal's line too (a concave
    # crease: the floor normal's line runs up the wall)
    sc = S.planar_scene()
    K = S.Intrinsics(80, 60, 70.0, 70.0, 39.5, 29.5)
    D = S.render_depth(sc, np.eye(4), K, None, noise=False)
    cam = O.Cam(*K.as_tuple())
    T = np.eye(4)
    for mode in (O.NORMALS_CROSS, O.NORMALS_INTEGRAL):
        p0 = O.Params(levels=1, normal_mode=mode, bilateral_radius=0)
        p1 = O.Params(levels=1, normal_mode=mode, bilateral_radius=0, shoot_radius=2)
        fl = _levels(D, cam, p0)
        ml = O.build_model_pyramid(fl.V, fl.N, cam, 1)[0]
        xf = O.f32_transforms(T, T)
        a0 = O.associate(fl, ml, T, xf, p0)
        a1 = O.associate(fl, ml, T, xf, p1)
        assert a0.valid.sum() > 0.5 * fl.V.shape[0] * fl.V.shape[1]
        moved = (a0.ui != a1.ui) | (a0.vi != a1.vi)
        assert moved.sum() <= 0.01 * a0.valid.sum()
        for y, x in zip(*np.nonzero(moved)):
            e = ml.V[a1.vi[y, x], a1.ui[y, x]] - fl.V[y, x]
            assert np.linalg.norm(np.cross(e, fl.N[y, x])) < 1e-6
        assert np.array_equal(a0.k[~moved], a1.k[~moved])


def test_shooting_picks_the_candidate_nearest_the_normal_line():
    # brute force in float64 with |e x n| (not the oracle's |e|^2 - s^2 form)
    sc = S.room_scene()
    K = S.Intrinsics(64, 48, 56.0, 56.0, 31.5, 23.5)
    rng = np.random.default_rng(11)
    pair = S.make_pair(sc, K, rng, 3.0, 0.04, 0.3, noise=False)
    cam = O.Cam(*K.as_tuple())
    w = 2
    p = O.Params(levels=1, shoot_radius=w)
    fl = _levels(pair.depth, cam, p)
    ml = O.build_model_pyramid(pair.model_vertex, pair.model_normal, cam, 1)[0]
    T = pair.gt_pose
    xf = O.f32_transforms(T, pair.model_pose)
    a = O.associate(fl, ml, T, xf, O.Params(levels=1, shoot_radius=w, d_max=1e3))
    proj = O.associate(fl, ml, T, xf, O.Params(levels=1, d_max=1e3))
    H, W = fl.V.shape[:2]
    checked = moved = 0
    for y in range(H):
        for x in range(W):
            if not a.valid[y, x]:
                continue
            P = T[:3, :3] @ fl.V[y, x] + T[:3, 3]
            n = T[:3, :3] @ fl.N[y, x]
            n /= np.linalg.norm(n)
            cu, cv = proj.ui[y, x], proj.vi[y, x]
            if cu < 0:
                continue
            best = []
            for dy in range(-w, w + 1):
                for dx in range(-w, w + 1):
                    u, v = cu + dx, cv + dy
                    if 0 <= u < W and 0 <= v < H and np.isfinite(ml.V[v, u]).all():
                        best.append((np.linalg.norm(np.cross(ml.V[v, u] - P, n)), u, v))
            dmin = min(b[0] for b in best)
            u, v = a.ui[y, x], a.vi[y, x]
            assert abs(u - cu) <= w and abs(v - cv) <= w
            chosen = np.linalg.norm(np.cross(ml.V[v, u] - P, n))
            assert chosen <= dmin + 2e-4          # float32 rounding of the choice
            checked += 1
            moved += (u, v) != (cu, cv)
    assert checked > 0.5 * H * W and moved > 0.05 * checked


def test_shooting_follows_the_normal_between_parallel_planes():
    # model: the plane z = 2.0; frame: the plane z = 2.1 seen from the same
    # camera. Shooting along the frame normal (the optical axis) meets the
    # model at the same (x, y), i.e. model column x f / 2.0 + c, where the
    # projection lands at x f / 2.1 + c.
    W, H, f, c = 64, 48, 60.0, (31.5, 23.5)
    cam = O.Cam(W, H, f, f, c[0], c[1])
    Dm = plane_depth(W, H, f, f, c[0], c[1], np.array([0.0, 0.0, -1.0]), -2.0).astype(np.float64)
    Vm = O.vertex_map(Dm, cam)
    Nm = np.broadcast_to(np.array([0.0, 0.0, -1.0]), Vm.shape).copy()
    Df = plane_depth(W, H, f, f, c[0], c[1], np.array([0.0, 0.0, -1.0]), -2.1).astype(np.float64)
    w = 3
    p = O.Params(levels=1, shoot_radius=w, bilateral_radius=0)
    fl = _levels(Df, cam, p)
    ml = O.build_model_pyramid(Vm, Nm, cam, 1)[0]
    T = np.eye(4)
    a = O.associate(fl, ml, T, O.f32_transforms(T, T), p)
    checked = 0
    for y in range(H):
        for x in range(W):
            if not a.valid[y, x]:
                continue
            X = fl.V[y, x]
            um = X[0] * f / 2.0 + c[0]
            vm = X[1] * f / 2.0 + c[1]
            up = X[0] * f / 2.1 + c[0]
            vp = X[1] * f / 2.1 + c[1]
            if (abs(um - round(up)) > w - 0.6 or abs(vm - round(vp)) > w - 0.6
                    or abs(um - math.floor(um) - 0.5) < 0.05 or abs(vm - math.floor(vm) - 0.5) < 0.05
                    or not (0 <= round(um) < W and 0 <= round(vm) < H)):
                continue
            assert (a.ui[y, x], a.vi[y, x]) == (round(um), round(vm))
            checked += 1
    assert checked > 0.3 * W * H
