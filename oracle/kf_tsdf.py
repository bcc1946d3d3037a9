"""CPU oracle of the model producer of KinectFusion tracking: TSDF integration
of depth frames into a cube of voxels and raycasting of the model's vertex and
normal maps (the "model reconstructed so far" that each frame is aligned to;
the paper keeps a 512^3 cube of at most 6 m side, Sec. 4.4).

TEST INFRASTRUCTURE ONLY: plain, slow numpy. Only the test suite and the
bench's CPU legs may use it; the CUDA library never does and shares no code
with it.

The paper does not restate integration or raycasting; they are written here
from their usual definitions (Newcombe et al., KinectFusion). As in the ICP
oracle, every floating-point result that DECIDES something discrete (which
pixel a voxel projects to, the truncation test, a zero crossing of the field,
the voxel cell of a sample) is evaluated in IEEE float32 one rounded operation
at a time in the order written here, so that a kernel doing the same
operations reproduces the decisions bit for bit; the stored field is float32.

Definitions (s = side / res, voxel i at o + (i + 1/2) s on each axis):

* integrate: voxel centre x (world) -> camera point p = R^T (x - t) evaluated
  as rows of [R^T | -R^T t] (float32); skip unless p.z > 0; pixel
  (rint(fx p.x / p.z + cx), rint(fy p.y / p.z + cy)) (round half to even);
  skip outside the image or where the raw depth D is not finite and positive;
  eta = D - p.z; skip unless eta >= -mu; f = min(1, eta / mu);
  F <- (W F + f) / (W + 1), W <- min(W + 1, w_max).
* sample(q): grid coordinate g = (q - o) / s - 1/2 per axis; the cell's lower
  corner i0 = floor(g) must satisfy 0 <= i0 <= res - 2 and all 8 corner
  weights W > 0; trilinear interpolation along x, then y, then z, each as
  a + t (b - a).
* raycast at pixel (u, v): camera-frame direction d_c = ((u - cx) / fx,
  (v - cy) / fy, 1), world direction d = R d_c, origin c = t; samples at
  depth z_k = z_near + k dz (k = 0, 1, ... while z_k <= z_far), q_k = c + z_k d.
  Among valid consecutive samples, the first pair with F_prev > 0 >= F_cur is
  the surface: z* = z_prev + dz F_prev / (F_prev - F_cur), vertex c + z* d.
  A pair going from F_prev < 0 to F_cur > 0 (a back face) ends the ray with no
  surface; an invalid sample breaks the pair. Normal: central differences of
  the field at the vertex with step s on each axis (all six samples valid),
  normalised (the field grows toward free space, so it faces the camera).
  Misses are NaN in both maps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

F32 = np.float32


@dataclass
class Volume:
    res: int
    side: float
    origin: tuple          # world position of the cube's lower corner
    mu: float              # truncation distance (m)
    w_max: float
    F: np.ndarray = None   # float32 [z][y][x]
    W: np.ndarray = None   # float32 [z][y][x]

    def __post_init__(self):
        if self.F is None:
            self.F = np.ones((self.res,) * 3, F32)
            self.W = np.zeros((self.res,) * 3, F32)


def _f32(x):
    return F32(x)


def _row(R, t, x, y, z):
    """((R0 x + R1 y) + R2 z) + t, each operation rounded to float32."""
    a = F32(F32(R[0] * x) + F32(R[1] * y))
    a = F32(a + F32(R[2] * z))
    return F32(a + t)


def world_to_camera32(T):
    """Float32 rows of [R^T | -R^T t] for the camera->world pose T (float64)."""
    T = np.asarray(T, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    Rt = R.T
    # -(((r0 t0) + r1 t1) + r2 t2) in float64, in this order, then float32
    tt = np.array([-((Rt[a, 0] * t[0] + Rt[a, 1] * t[1]) + Rt[a, 2] * t[2]) for a in range(3)])
    return Rt.astype(F32), tt.astype(F32)


def voxel_centres(vol: Volume):
    """Float32 world coordinates of the voxel centres per axis (x, y, z)."""
    s = F32(F32(vol.side) / F32(vol.res))
    idx = np.arange(vol.res, dtype=F32) + F32(0.5)
    return [F32(vol.origin[a]) + (idx * s).astype(F32) for a in range(3)], s


def integrate(vol: Volume, depth, cam, T):
    """Fuse one raw depth frame (H x W float32 metres) seen from camera->world
    pose T with intrinsics cam (fx, fy, cx, cy as float32) into vol (in place)."""
    D = np.asarray(depth, F32)
    H, Wd = D.shape
    (cx_, cy_, cz_), s = voxel_centres(vol)
    X = cx_[None, None, :]
    Y = cy_[None, :, None]
    Z = cz_[:, None, None]
    Rt, tt = world_to_camera32(T)
    px = _row(Rt[0], tt[0], X, Y, Z)
    py = _row(Rt[1], tt[1], X, Y, Z)
    pz = _row(Rt[2], tt[2], X, Y, Z)
    px, py, pz = np.broadcast_arrays(px, py, pz)
    fx, fy, ccx, ccy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        front = pz > F32(0)
        # float32 arrays with float32 scalars: every operation rounds to float32
        uf = ((fx * px) / pz + ccx).astype(F32)
        vf = ((fy * py) / pz + ccy).astype(F32)
        ur = np.rint(uf)
        vr = np.rint(vf)
        inside = front & (ur >= 0) & (ur <= Wd - 1) & (vr >= 0) & (vr <= H - 1)
        ui = np.where(inside, ur, 0).astype(np.int64)
        vi = np.where(inside, vr, 0).astype(np.int64)
        d = D[vi, ui]
        ok = inside & np.isfinite(d) & (d > F32(0))
        eta = (d - pz).astype(F32)
        mu = F32(vol.mu)
        ok &= eta >= -mu
        f = np.minimum(F32(1), (eta / mu).astype(F32)).astype(F32)
        Wc, Fc = vol.W, vol.F
        Fn = ((Wc * Fc).astype(F32) + f).astype(F32)
        Fn = (Fn / (Wc + F32(1))).astype(F32)
        Wn = np.minimum(Wc + F32(1), F32(vol.w_max)).astype(F32)
    vol.F = np.where(ok, Fn, Fc).astype(F32)
    vol.W = np.where(ok, Wn, Wc).astype(F32)


def sample(vol: Volume, q):
    """Trilinear field value at world point q (3 float32), or None when the
    cell is outside the cube or has an unobserved corner."""
    s = F32(F32(vol.side) / F32(vol.res))
    g = [F32(F32(F32(q[a] - F32(vol.origin[a])) / s) - F32(0.5)) for a in range(3)]
    i0 = [int(math.floor(float(g[a]))) for a in range(3)]
    if any(i0[a] < 0 or i0[a] > vol.res - 2 for a in range(3)):
        return None
    t = [F32(g[a] - F32(i0[a])) for a in range(3)]
    x0, y0, z0 = i0
    Wc = vol.W[z0:z0 + 2, y0:y0 + 2, x0:x0 + 2]
    if not (Wc > 0).all():
        return None
    Fc = vol.F[z0:z0 + 2, y0:y0 + 2, x0:x0 + 2]

    def lerp(a, b, u):
        return F32(a + F32(u * F32(b - a)))

    c00 = lerp(Fc[0, 0, 0], Fc[0, 0, 1], t[0])
    c10 = lerp(Fc[0, 1, 0], Fc[0, 1, 1], t[0])
    c01 = lerp(Fc[1, 0, 0], Fc[1, 0, 1], t[0])
    c11 = lerp(Fc[1, 1, 0], Fc[1, 1, 1], t[0])
    c0 = lerp(c00, c10, t[1])
    c1 = lerp(c01, c11, t[1])
    return lerp(c0, c1, t[2])


def raycast(vol: Volume, cam, width: int, height: int, T, z_near: float, z_far: float, dz: float):
    """World vertex and normal maps (H x W x 3 float32, NaN = miss) of the
    field seen from camera->world pose T."""
    T = np.asarray(T, np.float64)
    R = T[:3, :3].astype(F32)
    c = T[:3, 3].astype(F32)
    fx, fy, ccx, ccy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    zn, zf, dzf = F32(z_near), F32(z_far), F32(dz)
    s = F32(F32(vol.side) / F32(vol.res))
    V = np.full((height, width, 3), np.nan, F32)
    N = np.full((height, width, 3), np.nan, F32)
    for v in range(height):
        for u in range(width):
            dc = (F32(F32(F32(u) - ccx) / fx), F32(F32(F32(v) - ccy) / fy), F32(1))
            d = [_row(R[a], F32(0), dc[0], dc[1], dc[2]) for a in range(3)]
            prev = None  # (z, F) of the last valid sample; an invalid one resets it
            k = 0
            while True:
                z = F32(zn + F32(F32(k) * dzf))
                if z > zf:
                    break
                k += 1
                q = [F32(c[a] + F32(z * d[a])) for a in range(3)]
                f = sample(vol, q)
                if f is None:
                    prev = None
                    continue
                if prev is not None and prev[1] > 0 and f <= 0:
                    zs = F32(prev[0] + F32(dzf * F32(prev[1] / F32(prev[1] - f))))
                    vx = [F32(c[a] + F32(zs * d[a])) for a in range(3)]
                    g = []
                    for a in range(3):
                        qp, qm = list(vx), list(vx)
                        qp[a] = F32(vx[a] + s)
                        qm[a] = F32(vx[a] - s)
                        fp, fm = sample(vol, qp), sample(vol, qm)
                        if fp is None or fm is None:
                            g = None
                            break
                        g.append(float(fp) - float(fm))
                    if g is not None:
                        nrm = math.sqrt(sum(x * x for x in g))
                        if nrm > 0:
                            V[v, u] = vx
                            N[v, u] = [x / nrm for x in g]
                    break
                if prev is not None and prev[1] < 0 and f > 0:
                    break  # back face: no surface along this ray
                prev = (z, f)
    return V, N
