"""Pins of the TSDF / raycast oracle (the model producer) against closed forms."""
import math

import numpy as np
import pytest

from oracle import kf_oracle as O
from oracle import kf_tsdf as T
from synth import scenes as S


def _wall_volume():
    # camera at the origin looking down +z; wall at z = 2.0; voxels 5 cm
    vol = T.Volume(res=32, side=1.6, origin=(-0.8, -0.6, 1.2), mu=0.15, w_max=64.0)
    cam = O.Cam(40, 30, 30.0, 30.0, 19.5, 14.5)
    return vol, cam


def test_integration_of_a_wall_is_the_truncated_distance():
    vol, cam = _wall_volume()
    D = np.full((cam.height, cam.width), 2.0, np.float32)
    T.integrate(vol, D, cam, np.eye(4))
    z = 1.2 + (np.arange(32) + 0.5) * 0.05
    x = -0.8 + (np.arange(32) + 0.5) * 0.05
    y = -0.6 + (np.arange(32) + 0.5) * 0.05
    checked = 0
    for k in range(32):
        for j in range(32):
            for i in range(32):
                # inside the view (with a margin from the image border)?
                u = 30.0 * x[i] / z[k] + 19.5
                v = 30.0 * y[j] / z[k] + 14.5
                if not (0.6 < u < cam.width - 1.6 and 0.6 < v < cam.height - 1.6):
                    continue
                eta = 2.0 - z[k]
                if eta >= -0.15 + 1e-6:
                    assert vol.W[k, j, i] == 1.0
                    assert abs(vol.F[k, j, i] - min(1.0, eta / 0.15)) < 2e-6
                    checked += 1
                elif eta < -0.15 - 1e-6:
                    assert vol.W[k, j, i] == 0.0 and vol.F[k, j, i] == 1.0
    assert checked > 1000


def test_weighted_average_and_weight_cap():
    vol, cam = _wall_volume()
    vol.w_max = 2.0
    depths = [2.0, 2.05, 1.95]
    for d in depths:
        T.integrate(vol, np.full((cam.height, cam.width), d, np.float32), cam, np.eye(4))
    # voxel (16, 15, 14): x ~ 0.025, y ~ 0.175, z = 1.2 + 14.5 * 0.05 = 1.925
    k, j, i = 14, 15, 16
    z = 1.2 + (k + 0.5) * 0.05
    f = [min(1.0, (d - z) / 0.15) for d in depths]
    # W = 0 -> 1 -> 2 -> 2 (capped): F = (f0 + f1) / 2, then (2 F + f2) / 3
    want = ((f[0] + f[1]) / 2 * 2 + f[2]) / 3
    assert vol.W[k, j, i] == 2.0
    assert abs(vol.F[k, j, i] - want) < 3e-6


def test_raycast_of_a_wall_is_exact_and_faces_the_camera():
    vol, cam = _wall_volume()
    T.integrate(vol, np.full((cam.height, cam.width), 2.0, np.float32), cam, np.eye(4))
    V, N = T.raycast(vol, cam, cam.width, cam.height, np.eye(4), 1.3, 2.6, 0.06)
    hit = np.isfinite(V[..., 0])
    assert hit[8:28, 10:30].all()  # the view of the wall inside the cube
    # the field is linear in z inside the band, so trilinear sampling and the
    # linear refinement find the wall exactly (to float32 rounding)
    assert np.abs(V[hit][:, 2] - 2.0).max() < 2e-5
    assert np.abs(N[hit] - np.array([0.0, 0.0, -1.0])).max() < 1e-5
    # the vertex lies on the pixel's ray
    vv, uu = np.nonzero(hit)
    ray = np.stack([(uu - 19.5) / 30.0, (vv - 14.5) / 30.0, np.ones_like(uu, float)], -1)
    assert np.abs(V[hit] - ray * V[hit][:, 2:3]).max() < 1e-5


def test_fused_sphere_is_recovered_within_a_voxel():
    sc = S.Scene(planes=[], spheres=[((0.0, 0.0, 2.0), 0.4)])
    K = S.Intrinsics(48, 36, 40.0, 40.0, 23.5, 17.5)
    cam = O.Cam(48, 36, 40.0, 40.0, 23.5, 17.5)
    vol = T.Volume(res=48, side=1.2, origin=(-0.6, -0.6, 1.4), mu=0.08, w_max=64.0)
    rng = np.random.default_rng(3)
    poses = [np.eye(4)]
    for ang in (6.0, -6.0):
        Rv = S.axis_angle_matrix(np.array([0.0, 1.0, 0.0]), math.radians(ang))
        P = np.eye(4)
        P[:3, :3] = Rv
        P[:3, 3] = np.array([0.0, 0.0, 2.0]) - Rv @ np.array([0.0, 0.0, 2.0])
        poses.append(P)
    for P in poses:
        T.integrate(vol, S.render_depth(sc, P, K, rng, noise=False), cam, P)
    V, N = T.raycast(vol, cam, cam.width, cam.height, np.eye(4), 1.0, 3.0, 0.03)
    hit = np.isfinite(V[..., 0])
    assert hit.sum() > 100  # the sphere covers ~200 pixels; silhouette rays see unobserved cells
    r = np.linalg.norm(V[hit] - np.array([0.0, 0.0, 2.0]), axis=1)
    assert np.abs(r - 0.4).max() < 0.025  # one voxel
    radial = (V[hit] - np.array([0.0, 0.0, 2.0])) / r[:, None]
    cosang = np.sum(N[hit] * radial, axis=1)
    assert np.median(cosang) > 0.99 and cosang.min() > 0.9
