"""Seeded synthetic inputs: analytic rooms, rendered depth frames and model maps.

This module only MAKES INPUTS. It holds none of the tracking method's
arithmetic (no pyramid, no association, no filter, no solve): it ray-casts
analytic primitives (planes, spheres, axis-aligned boxes) to produce

* a depth frame in metres (float32, 0 = no measurement) as a range sensor at
  a given camera pose would see it, with the Kinect-like noise model
  sigma(z) = 0.0012 + 0.0019 (z - 0.4)^2, dropout and uniform-depth outliers;
* noise-free model vertex / normal maps in world coordinates (float32, NaN
  where the ray hits nothing), which stand in for the model raycast that
  KinectFusion renders at the previous pose;
* the ground-truth motion and the IMU orientation prior (ground truth rotated
  by a random-axis angle of stated size).

Both the CUDA path's tests / bench and the oracle's tests draw their inputs
here; nothing here depends on either of them.

Conventions: camera frame x right, y down, z forward; a pixel (u, v) has its
centre at integer coordinates; a pose is a 4x4 float64 camera->world matrix.
Seeds follow ``seed = 180203980 + 100 * config + case`` fed to
``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 180203980


def rng_for(config: int, case: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 100 * config + case))


# ----------------------------------------------------------------------------
# small SO(3) helpers used to *generate* motions (not part of the method)
# ----------------------------------------------------------------------------
def axis_angle_matrix(axis, angle_rad: float) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle_rad) * K + (1.0 - math.cos(angle_rad)) * (K @ K)


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def make_pose(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def look_at(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """Camera->world pose for a camera at ``eye`` looking at ``target`` (y-down world)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    upv = np.asarray(up, np.float64)
    x = np.cross(-upv, z)
    if np.linalg.norm(x) < 1e-9:
        x = np.array([1.0, 0.0, 0.0])
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return make_pose(np.stack([x, y, z], axis=1), eye)


# ----------------------------------------------------------------------------
# scene description and ray casting
# ----------------------------------------------------------------------------
@dataclass
class Intrinsics:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def as_tuple(self):
        return (self.width, self.height, self.fx, self.fy, self.cx, self.cy)


@dataclass
class Scene:
    planes: list = field(default_factory=list)   # (unit normal n, offset d): n.x = d
    spheres: list = field(default_factory=list)  # (centre, radius)
    boxes: list = field(default_factory=list)    # (lo, hi) axis-aligned


def raycast(scene: Scene, pose: np.ndarray, K: Intrinsics):
    """Per pixel: hit parameter s (= camera-frame depth), world point, world normal.

    Rays are o + s * R (u - cx)/fx, (v - cy)/fy, 1); the normal returned faces
    the ray (n . dir < 0). Pixels that hit nothing get s = inf and NaN maps.
    """
    H, W = K.height, K.width
    u = np.arange(W, dtype=np.float64)[None, :].repeat(H, 0)
    v = np.arange(H, dtype=np.float64)[:, None].repeat(W, 1)
    dc = np.stack([(u - K.cx) / K.fx, (v - K.cy) / K.fy, np.ones_like(u)], axis=-1)
    R, o = pose[:3, :3], pose[:3, 3]
    dw = dc @ R.T                                   # (H, W, 3)
    best = np.full((H, W), np.inf)
    nrm = np.full((H, W, 3), np.nan)
    eps = 1e-9
    for n, d in scene.planes:
        n = np.asarray(n, np.float64)
        den = dw @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            s = (d - o @ n) / den
        ok = (s > eps) & (s < best) & np.isfinite(s)
        best = np.where(ok, s, best)
        nrm[ok] = n
    for c, r in scene.spheres:
        c = np.asarray(c, np.float64)
        oc = o - c
        a = np.einsum("hwk,hwk->hw", dw, dw)
        b = 2.0 * (dw @ oc)
        c0 = oc @ oc - r * r
        disc = b * b - 4 * a * c0
        with np.errstate(invalid="ignore"):
            sq = np.sqrt(np.maximum(disc, 0.0))
        s1 = (-b - sq) / (2 * a)
        s2 = (-b + sq) / (2 * a)
        s = np.where(s1 > eps, s1, s2)
        ok = (disc >= 0) & (s > eps) & (s < best)
        best = np.where(ok, s, best)
        hit = o + s[..., None] * dw
        nn = (hit - c) / r
        nrm[ok] = nn[ok]
    for lo, hi in scene.boxes:
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo - o) / dw
            t2 = (hi - o) / dw
        tmin3 = np.minimum(t1, t2)
        tmax3 = np.maximum(t1, t2)
        tmin = np.nanmax(tmin3, axis=-1)
        tmax = np.nanmin(tmax3, axis=-1)
        ax = np.nanargmax(tmin3, axis=-1)
        ok = (tmax >= np.maximum(tmin, eps)) & (tmin > eps) & (tmin < best)
        best = np.where(ok, tmin, best)
        nn = np.zeros((H, W, 3))
        sgn = -np.sign(np.take_along_axis(dw, ax[..., None], -1)[..., 0])
        np.put_along_axis(nn, ax[..., None], sgn[..., None], -1)
        nrm[ok] = nn[ok]
    hitp = o + best[..., None] * dw
    valid = np.isfinite(best)
    hitp[~valid] = np.nan
    nrm[~valid] = np.nan
    # face the ray
    flip = np.einsum("hwk,hwk->hw", nrm, dw) > 0
    nrm[flip] *= -1.0
    return best, hitp, nrm


def render_depth(scene, pose, K, rng=None, noise=True, dropout=0.0, outliers=0.0,
                 holes=0.0, z_range=(0.5, 4.0), outlier_range=(0.5, 4.0)):
    """float32 depth (metres, 0 = none) with the Kinect-like noise model."""
    s, _, _ = raycast(scene, pose, K)
    z = s.copy()
    z[~np.isfinite(z)] = 0.0
    if rng is not None and noise:
        sig = 0.0012 + 0.0019 * (z - 0.4) ** 2
        z = z + rng.normal(size=z.shape) * sig
    z[(z < z_range[0] * 0.5) | (z > z_range[1] * 2.0)] = 0.0
    if rng is not None and outliers > 0:
        m = rng.random(z.shape) < outliers
        z[m] = rng.uniform(outlier_range[0], outlier_range[1], size=int(m.sum()))
    if rng is not None and dropout > 0:
        z[rng.random(z.shape) < dropout] = 0.0
    if rng is not None and holes > 0:
        z[rng.random(z.shape) < holes] = 0.0
    return z.astype(np.float32)


def render_model(scene, pose, K):
    """Noise-free float32 world vertex / normal maps (H, W, 3); NaN = no surface."""
    _, p, n = raycast(scene, pose, K)
    return p.astype(np.float32), n.astype(np.float32)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------
def room_scene() -> Scene:
    """Five planes (floor, ceiling, back and side walls), two spheres and a box.

    Seen from a camera near the origin looking down +z, depths are 1.1-3.9 m.
    """
    sc = Scene()
    sc.planes = [
        ((0.0, -1.0, 0.0), -1.2),   # floor y = 1.2   (y down)
        ((0.0, 1.0, 0.0), -1.5),    # ceiling y = -1.5
        ((0.0, 0.0, -1.0), -3.8),   # back wall z = 3.8
        ((1.0, 0.0, 0.0), -2.0),    # left wall x = -2.0
        ((-1.0, 0.0, 0.0), -2.2),   # right wall x = 2.2
    ]
    sc.spheres = [((-0.6, 0.3, 2.2), 0.35), ((0.8, -0.2, 1.6), 0.25)]
    sc.boxes = [((0.1, 0.5, 2.5), (0.7, 1.2, 3.0))]
    return sc


def planar_scene() -> Scene:
    """Piecewise-planar room (planes + box, no spheres): exact-recovery scenes."""
    sc = room_scene()
    sc.spheres = []
    return sc


def random_scene(rng: np.random.Generator) -> Scene:
    """Seeded random room layout: 5 walls at jittered offsets, 1-3 spheres, 1-2 boxes."""
    sc = Scene()
    sc.planes = [
        ((0.0, -1.0, 0.0), -rng.uniform(1.0, 1.4)),
        ((0.0, 1.0, 0.0), -rng.uniform(1.3, 1.7)),
        ((0.0, 0.0, -1.0), -rng.uniform(3.2, 3.8)),
        ((1.0, 0.0, 0.0), -rng.uniform(1.8, 2.4)),
        ((-1.0, 0.0, 0.0), -rng.uniform(1.8, 2.4)),
    ]
    for _ in range(int(rng.integers(1, 4))):
        sc.spheres.append(((rng.uniform(-1.0, 1.0), rng.uniform(-0.5, 0.6),
                            rng.uniform(1.4, 2.8)), rng.uniform(0.15, 0.45)))
    for _ in range(int(rng.integers(1, 3))):
        lo = np.array([rng.uniform(-1.2, 0.8), rng.uniform(0.2, 0.8), rng.uniform(2.0, 2.9)])
        hi = lo + rng.uniform(0.2, 0.6, size=3)
        sc.boxes.append((tuple(lo), tuple(hi)))
    return sc


def kinect_intrinsics(width=640, height=480) -> Intrinsics:
    f = 525.0 * width / 640.0
    return Intrinsics(width, height, f, f, (width - 1) / 2.0, (height - 1) / 2.0)


# ----------------------------------------------------------------------------
# frame pairs
# ----------------------------------------------------------------------------
@dataclass
class FramePair:
    K: Intrinsics              # frame and model intrinsics (same camera)
    depth: np.ndarray          # (H, W) float32 frame depth
    model_vertex: np.ndarray   # (H, W, 3) float32 world
    model_normal: np.ndarray   # (H, W, 3) float32 world
    model_pose: np.ndarray     # 4x4 camera->world of the model render
    gt_pose: np.ndarray        # 4x4 camera->world of the frame
    prior_R: np.ndarray        # 3x3 IMU orientation prior (world)
    init_pose: np.ndarray      # 4x4 initial estimate (= model pose)
    lam: float = 1e3


def make_pair(scene, K, rng, rot_deg, trans_m, prior_noise_deg, noise=True,
              dropout=0.0, outliers=0.0, holes=0.0, lam=1e3, base_pose=None,
              rot_exact=True) -> FramePair:
    """A frame/model pair related by a random rigid motion.

    rot_exact: the motion angle is exactly ``rot_deg`` (else uniform in [0, rot_deg]);
    likewise the translation length ``trans_m``.
    """
    if base_pose is None:
        base_pose = look_at(rng.uniform(-0.1, 0.1, size=3),
                            (rng.uniform(-0.2, 0.2), rng.uniform(-0.1, 0.1), 3.0))
    ang = rot_deg if rot_exact else rng.uniform(0.0, rot_deg)
    tl = trans_m if rot_exact else rng.uniform(0.0, trans_m)
    dR = axis_angle_matrix(random_unit(rng), math.radians(ang))
    dT = make_pose(dR, tl * random_unit(rng))
    gt = base_pose @ dT
    noiseR = axis_angle_matrix(random_unit(rng), math.radians(prior_noise_deg))
    prior = noiseR @ gt[:3, :3]
    depth = render_depth(scene, gt, K, rng, noise=noise, dropout=dropout,
                         outliers=outliers, holes=holes)
    mv, mn = render_model(scene, base_pose, K)
    return FramePair(K, depth, mv, mn, base_pose.copy(), gt, prior, base_pose.copy(), lam)


def config1_tiny(case: int = 0) -> FramePair:
    """160x120, fx=fy=140, 2 deg + 3 cm motion, 0.5 deg prior noise, 2 % dropout."""
    rng = rng_for(1, case)
    K = Intrinsics(160, 120, 140.0, 140.0, 80.0, 60.0)
    return make_pair(room_scene(), K, rng, 2.0, 0.03, 0.5, dropout=0.02, lam=1e3)


def config2_kinect(case: int = 0, width=640, height=480, outliers=0.10) -> FramePair:
    """640x480 Kinect intrinsics, motion <= 5 deg / 5 cm, prior noise 0.3 deg, 10 % outliers."""
    rng = rng_for(2, case)
    K = kinect_intrinsics(width, height)
    return make_pair(room_scene(), K, rng, 5.0, 0.05, 0.3, outliers=outliers,
                     lam=1e3, rot_exact=False)


ANGULAR_SWEEP_DEG = (5.0, 10.0, 20.0, 30.0, 45.0, 60.0)


def angular_case(angle_index: int, case: int, width=640, height=480) -> FramePair:
    """Angular-failure sweep member: Kinect recipe with a rotation of exactly
    ANGULAR_SWEEP_DEG[angle_index] about a random axis, 5 cm translation, prior
    noise 0.3 deg, 10 % outliers (cases 0..15 per angle)."""
    rng = rng_for(6, 16 * angle_index + case)
    K = kinect_intrinsics(width, height)
    return make_pair(room_scene(), K, rng, ANGULAR_SWEEP_DEG[angle_index], 0.05, 0.3,
                     outliers=0.10, lam=1e3, rot_exact=True)


def config4_batch(case: int) -> FramePair:
    """Mixed-resolution batch member: 4 resolutions x 16, 4 seeded scenes."""
    res = [(320, 240), (640, 480), (960, 720), (1280, 960)][case // 16]
    rng = rng_for(4, case)
    scene = random_scene(rng_for(4, 1000 + case % 4))
    K = kinect_intrinsics(*res)
    lam = float(10 ** rng.uniform(0.0, 3.0))
    return make_pair(scene, K, rng, 8.0, 0.08, 0.5, outliers=float(rng.uniform(0, 0.3)),
                     lam=lam, rot_exact=False)


def config3_precision(case: int, lam: float, prior_noise_deg: float) -> FramePair:
    """640x480 pair of the Kinect recipe with a given lambda and IMU prior noise."""
    rng = rng_for(3, case)
    K = kinect_intrinsics()
    return make_pair(room_scene(), K, rng, 5.0, 0.05, prior_noise_deg, outliers=0.10,
                     lam=lam, rot_exact=False)


# ----------------------------------------------------------------------------
# long trajectory (config 5): smooth camera path in a 6 x 6 x 3 m room
# ----------------------------------------------------------------------------
def room_6x6x3() -> Scene:
    """6 x 6 x 3 m room (y down: floor y = 1.5, ceiling y = -1.5), with clutter."""
    sc = Scene()
    sc.planes = [
        ((0.0, -1.0, 0.0), -1.5), ((0.0, 1.0, 0.0), -1.5),
        ((0.0, 0.0, -1.0), -3.0), ((0.0, 0.0, 1.0), -3.0),
        ((1.0, 0.0, 0.0), -3.0), ((-1.0, 0.0, 0.0), -3.0),
    ]
    sc.spheres = [((-1.2, 0.8, 1.5), 0.45), ((1.4, 0.9, -1.0), 0.35), ((0.3, 1.1, -2.0), 0.4)]
    sc.boxes = [((0.8, 0.6, 1.2), (1.6, 1.5, 2.2)), ((-2.2, 0.4, -1.5), (-1.4, 1.5, -0.5)),
                ((-0.5, -1.5, 2.3), (0.5, -0.9, 3.0))]
    return sc


def trajectory(n_frames: int, rng: np.random.Generator, hz: float = 30.0,
               max_ang_deg_s: float = 60.0, max_speed: float = 1.0):
    """Smooth camera->world poses: a slow orbit around the room centre with
    sinusoidal yaw/pitch wobble, speeds capped at max_speed (m/s) and
    max_ang_deg_s (deg/s)."""
    ph = rng.uniform(0, 2 * math.pi, size=6)
    radius = 0.6
    w_orbit = min(max_speed / radius, math.radians(max_ang_deg_s) * 0.5) * 0.6
    poses = []
    for i in range(n_frames):
        t = i / hz
        eye = np.array([radius * math.cos(w_orbit * t + ph[0]), 0.2 * math.sin(0.7 * t + ph[1]),
                        radius * math.sin(w_orbit * t + ph[0])])
        yaw = w_orbit * t + ph[2] + 0.25 * math.sin(1.3 * t + ph[3])
        pitch = 0.15 * math.sin(0.9 * t + ph[4])
        target = eye + np.array([math.cos(yaw) * math.cos(pitch), math.sin(pitch),
                                 math.sin(yaw) * math.cos(pitch)])
        poses.append(look_at(eye, target))
    return poses


def imu_priors(gt_poses, rng: np.random.Generator, hz: float = 30.0, white_deg: float = 0.2,
               drift_deg_s: float = 0.01):
    """IMU orientation = ground truth rotated by a slowly drifting bias (random
    axis, drift_deg_s per second) and white noise of white_deg."""
    axis = random_unit(rng)
    out = []
    for i, T in enumerate(gt_poses):
        bias = axis_angle_matrix(axis, math.radians(drift_deg_s * i / hz))
        noise = axis_angle_matrix(random_unit(rng), math.radians(white_deg) * abs(rng.normal()))
        out.append(noise @ bias @ T[:3, :3])
    return out
