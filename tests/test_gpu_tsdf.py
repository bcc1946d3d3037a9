"""Model producer on the GPU (TSDF volume + raycast, through the C ABI) against
the oracle: fields bit-exact (same float32 decision chain), raycast vertices
bit-exact with the same hit mask, normals to 1e-5; and the loop closed: a
tracker aligns a frame to the raycast of the frames fused before it."""
import math

import numpy as np
import pytest

from oracle import kf_oracle as O
from oracle import kf_tsdf as TS
from synth import scenes as S
from tests import kfhelp as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03980_gb300 import build
    build()


def _vol(k, res, side, origin, mu, w_max=64.0):
    p = k.kf_volume_params()
    p.res, p.side, p.mu, p.w_max = res, side, mu, w_max
    for a in range(3):
        p.origin[a] = origin[a]
    return k.kf_volume_create(p, 0), TS.Volume(res=res, side=side, origin=tuple(origin), mu=mu, w_max=w_max)


def _orbit(ang_deg, centre):
    Rv = S.axis_angle_matrix(np.array([0.0, 1.0, 0.0]), math.radians(ang_deg))
    P = np.eye(4)
    P[:3, :3] = Rv
    P[:3, 3] = np.asarray(centre) - Rv @ np.asarray(centre)
    return P


@pytest.mark.parametrize("scene", ["sphere_wall", "room"])
def test_integration_and_raycast_match_oracle(scene):
    k = H.kf()
    rng = np.random.default_rng(7)
    if scene == "sphere_wall":
        sc = S.Scene(planes=[((0.0, 0.0, -1.0), -2.6)], spheres=[((0.0, 0.0, 2.0), 0.4)])
        K = S.Intrinsics(48, 36, 40.0, 40.0, 23.5, 17.5)
        res, side, origin, mu = 48, 1.8, (-0.9, -0.9, 1.2), 0.08
        poses = [np.eye(4), _orbit(6.0, (0.0, 0.0, 2.0)), _orbit(-5.0, (0.0, 0.0, 2.0))]
        noise = False
        rc = (1.0, 3.2, 0.03)
    else:
        sc = S.room_scene()
        K = S.Intrinsics(64, 48, 52.5, 52.5, 31.5, 23.5)
        res, side, origin, mu = 80, 4.0, (-2.0, -1.6, 0.8), 0.1
        poses = [np.eye(4), _orbit(4.0, (0.0, 0.0, 2.5))]
        noise = True
        rc = (0.5, 4.5, 0.05)
    cam = O.Cam(*K.as_tuple())
    v, vo = _vol(k, res, side, origin, mu)
    try:
        for P in poses:
            D = np.ascontiguousarray(S.render_depth(sc, P, K, rng, noise=noise), np.float32)
            k.kf_volume_integrate(v, D.ctypes.data, K.as_tuple(), P, False)
            TS.integrate(vo, D, cam, P)
        F, W = k.kf_volume_read(v, res)
        assert np.array_equal(W, vo.W)
        assert np.array_equal(F, vo.F)
        assert (W > 0).sum() > 1000
        Pr = _orbit(2.0, (0.0, 0.0, 2.0))
        V, N = k.kf_volume_raycast(v, K.as_tuple(), Pr, *rc)
    finally:
        k.kf_volume_destroy(v)
    Vo, No = TS.raycast(vo, cam, K.width, K.height, Pr, *rc)
    hit, hit_o = np.isfinite(V[..., 0]), np.isfinite(Vo[..., 0])
    assert np.array_equal(hit, hit_o)
    assert hit.sum() > 200
    assert np.array_equal(V[hit], Vo[hit])
    assert np.abs(N[hit] - No[hit]).max() < 1e-5


def test_tracking_against_the_raycast_model_closes_the_loop():
    """Frames of a smooth path fused at their true poses into a 256^3 cube; a
    later frame, seeded with a noisy IMU prior and the previous pose, aligns
    to the raycast of that model to within 1 cm / 0.2 deg of its truth."""
    import torch
    k = H.kf()
    rng = S.rng_for(5, 7)
    gt = S.trajectory(12, rng)
    scene, K = S.room_6x6x3(), S.kinect_intrinsics()
    Kt = K.as_tuple()
    p = k.kf_volume_params()
    # the cube encloses the 6 x 6 x 3 m room with a margin (walls on its faces
    # would leave no sampleable cell behind them); mu ~4 voxels
    p.res, p.side, p.mu, p.w_max = 256, 6.6, 0.10, 64.0
    for a in range(3):
        p.origin[a] = -3.3
    v = k.kf_volume_create(p, 0)
    tp, op = H.params()
    t = k.kf_track_create(tp, 640, 480, 0)
    try:
        for i in range(10):
            D = np.ascontiguousarray(S.render_depth(scene, gt[i], K, rng, noise=True), np.float32)
            k.kf_volume_integrate(v, D.ctypes.data, Kt, gt[i], False)
        Vd = torch.empty((480, 640, 3), dtype=torch.float32, device="cuda")
        Nd = torch.empty_like(Vd)
        torch.cuda.synchronize()
        k.kf_volume_raycast(v, Kt, gt[9], 0.3, 6.0, 0.02, Vd.data_ptr(), Nd.data_ptr(), True)
        torch.cuda.synchronize()
        assert torch.isfinite(Vd[..., 0]).float().mean().item() > 0.8
        k.kf_set_model(t, Vd.data_ptr(), Nd.data_ptr(), gt[9], Kt, True)
        D = np.ascontiguousarray(S.render_depth(scene, gt[10], K, rng, noise=True, outliers=0.1), np.float32)
        k.kf_set_frame(t, D.ctypes.data, Kt, False)
        prior = S.imu_priors(gt, rng)[10]
        st, pose, res = k.kf_align(t, prior, gt[9], 5.0)
    finally:
        k.kf_track_destroy(t)
        k.kf_volume_destroy(v)
    rot, tr = H.pose_err(pose, gt[10])
    assert st >= 0 and math.degrees(rot) < 0.2 and tr < 0.01, (st, math.degrees(rot), tr)
