"""FP64 CPU oracle of the IMU-seeded, median-filtered, orientation-regularised
coarse-to-fine point-to-plane ICP (Giancola et al., arXiv 1802.03980).

TEST INFRASTRUCTURE ONLY. Plain, slow, obviously correct numpy. Only the test
suite, ``__graft_entry__.smoke()`` and the bench's CPU-baseline / reference
legs may import it; the CUDA library never does, and this module shares no
code, table or constant generator with it.

Arithmetic is float64 throughout, with one exception that the paper leaves
open: every floating-point result that DECIDES an integer or a discrete choice
(which model pixel a frame point projects to, which histogram bin a distance
falls in, the distance gate, the pyramid's depth-similarity test, the optional
normal-angle gate) is evaluated in IEEE float32, one rounded operation at a
time in the order written below, exactly as the kernel evaluates it; where
the order says fma(a, b, c), that one operation is the exactly rounded a b + c
(``fma32``). The values that feed the least-squares system (points,
residuals, sums) stay in float64.

Sections followed (paper: "Integration of Absolute Orientation Measurements in
the KinectFusion Reconstruction pipeline"):

* Eq. 1  point-to-plane objective over matched pairs (p_i, q_i, n_i).
* Sec. 3 first paragraph: the IMU orientation pre-rotates the frame points
  (the seed T0 = [R_prior | t_init]).
* Eq. 2  small-angle form of the increment; Eq. 3 its linear least squares
  with rows a_i = [(p_i x n_i)^T, n_i^T], b_i = n_i . (q_i - p_i)  (the rows of
  Low 2004, which the paper defers to).
* Eq. 4 / Eq. 5  regularised problem and normal equations
  (A^T A + 2 lambda n P^T P) x = A^T b, P = [I3 | 0].
* Sec. 3.2  histogram (PDF) of point-to-point distances of matched pairs, its
  CDF; n estimated as the count of good matches.
* Sec. 3.3  median from the CDF up to the histogram's resolution; pairs that do
  not gather around the median are rejected.
* Sec. 3.4  a level stops once the median is unchanged (at histogram
  resolution) over 3 successive iterations.
* Sec. 4.4 (timing): coarse-to-fine cadence (4, 5, 10) iterations,
  coarsest level first.
* Variant (flag PRIOR_ANCHORED, not in the paper): the regulariser of Eq. 4
  anchored to the IMU prior instead of the increment (``anchored_rhs``).
* Sec. 3.3 also names the paper's own choices for normals and association:
  integral-image normals (``normal_mode = NORMALS_INTEGRAL``, written in
  ``kf_normals``) and normal shooting (``shoot_radius``,
  ``_normal_shooting``). Projective association with cross-product normals
  (KinectFusion's) stays the default.

The preprocessing (bilateral filter, pyramid, vertex and normal maps) is the
KinectFusion front end that the paper builds on but does not restate; it is
written here from the definitions given in each function's docstring.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32

# status codes (same numeric values as the C ABI's kf_status)
OK = 0
NOT_CONVERGED = 1
TOO_FEW_INLIERS = -6
DEGENERATE = -7

USE_PRIOR = 1
USE_FILTER = 2
USE_CONVERGENCE = 4
PRIOR_ANCHORED = 32  # regulariser variant (our extension): see anchored_rhs

LAMBDA_CONST, LAMBDA_C_SQRT_N, LAMBDA_C_N, LAMBDA_C_N2, LAMBDA_C_LOG_N = range(5)
NORMALS_CROSS, NORMALS_INTEGRAL = 0, 1


@dataclass
class Params:
    levels: int = 3
    max_iters: tuple = (10, 5, 4)        # finest level first; run coarsest first
    hist_bins: int = 512
    d_max: float = 0.16                  # metres; B / d_max = 3200 bins per metre
    band_kappa: float = 1.0
    cos_angle_min: float = -2.0          # <= -1: angle gate off
    conv_window: int = 3
    lambda_mode: int = LAMBDA_CONST
    lambda_c: float = 5.0
    n_min: int = 6
    flags: int = USE_PRIOR | USE_FILTER | USE_CONVERGENCE
    bilateral_sigma_s: float = 4.0
    bilateral_sigma_r: float = 0.03
    bilateral_radius: int = 2
    normal_mode: int = 0                 # NORMALS_CROSS | NORMALS_INTEGRAL
    ii_radius_a: float = 2.0             # integral-image window half-size a + b z (level 0)
    ii_radius_b: float = 1.0
    ii_depth_change: float = 0.02
    ii_radius_max: int = 8
    shoot_radius: int = 0                # 0: projective association; w: normal shooting


@dataclass
class Cam:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


# ----------------------------------------------------------------------------
# pyramid intrinsics
# ----------------------------------------------------------------------------
def frame_level_cams(K: Cam, levels: int) -> list[Cam]:
    """Frame level l+1 averages 2x2 blocks of level l: f' = f/2, c' = (c - 0.5)/2.

    A level-(l+1) pixel x' covers level-l pixels 2x' and 2x'+1 whose centre is
    2x' + 1/2, so u_l = 2 x' + 1/2 maps to x' = (u_l - 1/2)/2.
    """
    cams = [K]
    for _ in range(1, levels):
        k = cams[-1]
        cams.append(Cam(k.width // 2, k.height // 2, k.fx / 2, k.fy / 2,
                        (k.cx - 0.5) / 2, (k.cy - 0.5) / 2))
    return cams


def model_level_cams(K: Cam, levels: int) -> list[Cam]:
    """Model level l+1 takes level-l pixel (2x', 2y'): f' = f/2, c' = c/2."""
    cams = [K]
    for _ in range(1, levels):
        k = cams[-1]
        cams.append(Cam(k.width // 2, k.height // 2, k.fx / 2, k.fy / 2, k.cx / 2, k.cy / 2))
    return cams


# ----------------------------------------------------------------------------
# front end: bilateral filter, pyramid, vertex and normal maps
# ----------------------------------------------------------------------------
def _valid_depth(D):
    return np.isfinite(D) & (D > 0)


def bilateral_filter(D, sigma_s: float, sigma_r: float, radius: int):
    """Edge-preserving smoothing of the level-0 depth (KinectFusion front end).

    D'(u) = sum_w D(u+d) w / sum_w w over the (2r+1)^2 window, neighbours with
    valid depth and inside the image only, where
    w = exp(-|d|^2 / (2 sigma_s^2) - (D(u+d) - D(u))^2 / (2 sigma_r^2)).
    D'(u) = 0 where D(u) is not a valid depth. radius 0 returns D unchanged
    (invalid samples set to 0).
    """
    D = np.asarray(D, np.float64)
    valid = _valid_depth(D)
    Dz = np.where(valid, D, 0.0)
    if radius <= 0:
        return Dz
    H, W = D.shape
    num = np.zeros_like(Dz)
    den = np.zeros_like(Dz)
    P = np.pad(Dz, radius, mode="constant", constant_values=0.0)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            Nb = P[radius + dy: radius + dy + H, radius + dx: radius + dx + W]
            nv = Nb > 0
            w = np.exp(-(dx * dx + dy * dy) / (2.0 * sigma_s ** 2)
                       - (Nb - Dz) ** 2 / (2.0 * sigma_r ** 2))
            w = np.where(nv & valid, w, 0.0)
            num += w * Nb
            den += w
    out = np.zeros_like(Dz)
    out[valid] = num[valid] / den[valid]
    return out


def downsample(D, sigma_r: float):
    """Level l+1 depth from level l (coarse-to-fine pyramid).

    Each output pixel looks at its 2x2 block in scan order (0,0), (1,0), (0,1),
    (1,1). The anchor is the first valid depth; the output is the mean of the
    valid depths z with |z - anchor| <= 3 sigma_r, or 0 if the block has no
    valid depth. The similarity test is a discrete choice and is evaluated in
    float32: |f32(z) - f32(anchor)| <= f32(3 sigma_r).
    """
    D = np.asarray(D, np.float64)
    H, W = D.shape[0] // 2, D.shape[1] // 2
    thr = F32(3.0 * sigma_r)
    blk = [D[0:2 * H:2, 0:2 * W:2], D[0:2 * H:2, 1:2 * W:2],
           D[1:2 * H:2, 0:2 * W:2], D[1:2 * H:2, 1:2 * W:2]]
    anchor = np.zeros((H, W))
    have = np.zeros((H, W), bool)
    for b in blk:
        take = (~have) & (b > 0)
        anchor = np.where(take, b, anchor)
        have |= take
    s = np.zeros((H, W))
    c = np.zeros((H, W))
    a32 = anchor.astype(F32)
    for b in blk:
        close = np.abs(b.astype(F32) - a32) <= thr
        use = (b > 0) & have & close
        s += np.where(use, b, 0.0)
        c += use
    out = np.zeros((H, W))
    out[c > 0] = s[c > 0] / c[c > 0]
    return out


def vertex_map(D, K: Cam):
    """v(u, v) = z K^-1 (u, v, 1): x = (u - cx) z / fx, y = (v - cy) z / fy.

    NaN where the depth is not valid.
    """
    D = np.asarray(D, np.float64)
    H, W = D.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    V = np.stack([(u - K.cx) * D / K.fx, (v - K.cy) * D / K.fy, D], axis=-1)
    V[~(D > 0)] = np.nan
    return V


def vertex_map32(D, K: Cam):
    """The float32 vertex map that the discrete decisions of the normal map
    see: with z the depth rounded to float32, u_c = float32(u) - float32(c_x)
    and i_x = 1 / float32(f_x) (one rounded float32 division),
    x = (u_c z) i_x, y = (v_c z) i_y, each product one float32 rounding.
    NaN where the depth is not valid (z > 0 fails)."""
    z = np.asarray(D, np.float64).astype(F32)
    H, W = z.shape
    uc = np.arange(W, dtype=F32)[None, :] - F32(K.cx)
    vc = np.arange(H, dtype=F32)[:, None] - F32(K.cy)
    ix = F32(1.0) / F32(K.fx)
    iy = F32(1.0) / F32(K.fy)
    with np.errstate(invalid="ignore", over="ignore"):
        V = np.stack([(uc * z) * ix, (vc * z) * iy, z], axis=-1)
        V[~(z > F32(0))] = np.nan
    return V


def normal_map(V, V32=None):
    """n = normalise((v(x+1,y) - v(x,y)) x (v(x,y+1) - v(x,y))), facing the camera.

    The value is computed in float64 from V. Whether a normal exists and which
    way it points are discrete decisions, taken in float32 (module docstring)
    from the float32 vertices V32 (default: V rounded to float32), each
    operation one rounding, in this order:
      a = v(x+1,y) - v(x,y),  b = v(x,y+1) - v(x,y)  (per component);
      c = (a_y b_z - a_z b_y, a_z b_x - a_x b_z, a_x b_y - a_y b_x), each
          product rounded, then the difference;
      l2 = (c_x c_x + c_y c_y) + c_z c_z: a normal exists iff l2 is finite
          and > 0 (and the float64 cross product does not vanish);
      s = (c_x v_x + c_y v_y) + c_z v_z: the camera sits at the origin of V's
          frame, so the normal is flipped iff s > 0 (decided before any
          normalisation).
    NaN at the last row and column and next to any invalid vertex.
    """
    H, W, _ = V.shape
    N = np.full_like(V, np.nan)
    c = V[:-1, :-1]
    dx = V[:-1, 1:] - c
    dy = V[1:, :-1] - c
    cr = np.cross(dx, dy)
    ln = np.linalg.norm(cr, axis=-1)
    V32 = np.asarray(V, np.float64).astype(F32) if V32 is None else np.asarray(V32, F32)
    c32 = V32[:-1, :-1]
    a32 = V32[:-1, 1:] - c32
    b32 = V32[1:, :-1] - c32
    with np.errstate(invalid="ignore", over="ignore"):
        cx = a32[..., 1] * b32[..., 2] - a32[..., 2] * b32[..., 1]
        cy = a32[..., 2] * b32[..., 0] - a32[..., 0] * b32[..., 2]
        cz = a32[..., 0] * b32[..., 1] - a32[..., 1] * b32[..., 0]
        l2 = cx * cx + cy * cy
        l2 = l2 + cz * cz
        sd = cx * c32[..., 0] + cy * c32[..., 1]
        sd = sd + cz * c32[..., 2]
    ok = np.isfinite(l2) & (l2 > F32(0)) & np.isfinite(ln) & (ln > 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        n = cr / ln[..., None]
    flip = sd > F32(0)
    n[flip] *= -1.0
    n[~ok] = np.nan
    N[:-1, :-1] = n
    return N


@dataclass
class FrameLevel:
    depth: np.ndarray
    V: np.ndarray        # (H, W, 3) camera frame, NaN invalid
    N: np.ndarray        # (H, W, 3) camera frame, NaN invalid
    cam: Cam


@dataclass
class ModelLevel:
    V: np.ndarray        # (H, W, 3) world, NaN invalid
    N: np.ndarray        # (H, W, 3) world
    cam: Cam


def build_frame_pyramid(depth, K: Cam, p: Params) -> list[FrameLevel]:
    """Bilateral filter at level 0, 2x2 downsampling, vertex and normal maps per level."""
    cams = frame_level_cams(K, p.levels)
    D = bilateral_filter(depth, p.bilateral_sigma_s, p.bilateral_sigma_r, p.bilateral_radius)
    out = []
    for l in range(p.levels):
        if l > 0:
            D = downsample(D, p.bilateral_sigma_r)
        V = vertex_map(D, cams[l])
        if p.normal_mode == NORMALS_INTEGRAL:
            N = level_integral_normals(D, cams[l], l, p)
            V = np.where(np.isfinite(N).all(-1)[..., None], V, np.nan)
        else:
            N = normal_map(V, vertex_map32(D, cams[l]))
        out.append(FrameLevel(D, V, N, cams[l]))
    return out


def level_integral_normals(D, cam: Cam, level: int, p: Params):
    """Integral-image normals (Sec. 3.3, Holzer et al.) of one level's depth,
    as float64 holding the float32 results; NaN where none (kf_normals)."""
    from .kf_normals import integral_normals
    _, N = integral_normals(np.asarray(D, F32), cam.fx, cam.fy, cam.cx, cam.cy, level,
                            p.ii_radius_a, p.ii_radius_b, p.ii_depth_change, p.ii_radius_max)
    return N.astype(np.float64)


def frame_level_from_maps(depth, V, N, cam: Cam) -> FrameLevel:
    return FrameLevel(np.asarray(depth, np.float64), np.asarray(V, np.float64),
                      np.asarray(N, np.float64), cam)


def build_model_pyramid(V0, N0, K: Cam, levels: int) -> list[ModelLevel]:
    """Model level l+1 = model level l at even pixels (2x', 2y')."""
    cams = model_level_cams(K, levels)
    V = np.asarray(V0, np.float64)
    N = np.asarray(N0, np.float64)
    out = [ModelLevel(V, N, cams[0])]
    for l in range(1, levels):
        H, W = cams[l].height, cams[l].width
        V = V[0:2 * H:2, 0:2 * W:2]
        N = N[0:2 * H:2, 0:2 * W:2]
        out.append(ModelLevel(V, N, cams[l]))
    return out


# ----------------------------------------------------------------------------
# the float32 transforms that drive association decisions
# ----------------------------------------------------------------------------
def relative_pose(T_cur, T_m):
    """T_rel = T_m^-1 T_cur in float64, summed in the fixed order k = 0, 1, 2.

    R_rel[i][j] = sum_k Rm[k][i] Rc[k][j];  t_rel[i] = sum_k Rm[k][i] (tc[k] - tm[k]).
    Plain Python floats: every product and sum is one IEEE double rounding.
    """
    Rc = [[float(T_cur[i][j]) for j in range(3)] for i in range(3)]
    tc = [float(T_cur[i][3]) for i in range(3)]
    Rm = [[float(T_m[i][j]) for j in range(3)] for i in range(3)]
    tm = [float(T_m[i][3]) for i in range(3)]
    R = [[0.0] * 3 for _ in range(3)]
    t = [0.0] * 3
    dt = [tc[k] - tm[k] for k in range(3)]
    for i in range(3):
        for j in range(3):
            s = Rm[0][i] * Rc[0][j]
            s = s + Rm[1][i] * Rc[1][j]
            s = s + Rm[2][i] * Rc[2][j]
            R[i][j] = s
        s = Rm[0][i] * dt[0]
        s = s + Rm[1][i] * dt[1]
        s = s + Rm[2][i] * dt[2]
        t[i] = s
    return np.array(R), np.array(t)


@dataclass
class Xf32:
    """float32 3x4 transforms used by the association decisions."""
    Rw: np.ndarray   # (3, 3) frame camera -> world
    tw: np.ndarray   # (3,)
    Rr: np.ndarray   # (3, 3) frame camera -> model camera
    tr: np.ndarray


def f32_transforms(T_cur, T_m) -> Xf32:
    Rr, tr = relative_pose(T_cur, T_m)
    T_cur = np.asarray(T_cur, np.float64)
    return Xf32(T_cur[:3, :3].astype(F32), T_cur[:3, 3].astype(F32),
                Rr.astype(F32), tr.astype(F32))


def fma32(a, b, c):
    """float32 fused multiply-add: a b + c rounded once to float32 (nearest,
    ties to even), elementwise.

    The product of two float32 values is exact in float64 (48 significant
    bits). The sum s = fl64(a b + c) may round, and rounding that again to
    float32 can differ from rounding the exact sum once (double rounding).
    Rounding the float64 sum to odd instead removes that: if the addition
    was inexact and s's last bit is even, s moves one float64 ulp towards the
    exact sum. A round-to-odd result with at least two more bits than the
    target rounds to the target correctly (Boldo and Melquiond, "Emulation of
    FMA and correctly rounded sums: proved algorithms using rounding to odd",
    IEEE Trans. Computers 57(4), 2008). The addition's error is exact by
    TwoSum (Knuth).
    """
    a = np.asarray(a, F32).astype(np.float64)
    b = np.asarray(b, F32).astype(np.float64)
    c = np.asarray(c, F32).astype(np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        p = a * b
        s = p + c
        bb = s - p
        e = (p - (s - bb)) + (c - bb)  # exact: p + c = s + e
        bits = s.view(np.int64) if s.ndim else np.array(s).view(np.int64)
        fix = np.isfinite(s) & (e != 0) & ((bits & 1) == 0)
        s = np.where(fix, np.nextafter(s, np.where(e > 0, np.inf, -np.inf)), s)
        return s.astype(F32)


def _xform32(R, t, x, y, z):
    """fma(R2, z, fma(R1, y, fma(R0, x, t))) per row: three fused
    multiply-adds in float32."""
    out = []
    for i in range(3):
        a = fma32(R[i, 0], x, t[i])
        a = fma32(R[i, 1], y, a)
        a = fma32(R[i, 2], z, a)
        out.append(a)
    return out


# ----------------------------------------------------------------------------
# projective association + distance histogram (Sec. 3.2)
# ----------------------------------------------------------------------------
@dataclass
class Assoc:
    valid: np.ndarray    # (H, W) bool: pixel is a matched pair within d_max
    ui: np.ndarray       # (H, W) int model column (-1 where no projection)
    vi: np.ndarray       # (H, W) int model row
    k: np.ndarray        # (H, W) int histogram bin (-1 where not valid)
    d32: np.ndarray      # (H, W) float32 point-to-point distance
    p: np.ndarray        # (H, W, 3) float64 world point T_cur v
    q: np.ndarray        # (H, W, 3) float64 model point
    n: np.ndarray        # (H, W, 3) float64 model normal


def associate(fl: FrameLevel, ml: ModelLevel, T_cur, xf: Xf32, p: Params) -> Assoc:
    """Projective data association and point-to-point distance per frame pixel.

    For each frame pixel with a valid vertex v and a valid normal:
      p   = R_cur v + t_cur (world);  p_m = T_rel v (model camera);
      reject unless p_m.z > 0;
      (u, v)^ = rint(fma(f p_m.xy, 1 / p_m.z, c)) with round-half-to-even
      (the reciprocal and each product rounded to float32);
      reject outside the model image or where the model vertex/normal is invalid;
      d = |p - q| (point-to-point, Sec. 3.2); reject unless d < d_max;
      optional: reject unless (R_cur n_frame) . n_model >= cos_angle_min;
      bin k = min(floor(d * B / d_max), B - 1).
    Variant shoot_radius = w > 0 (normal shooting, Sec. 3.3): the model pixel
    is the one of the (2w+1)^2 window around the projection chosen by
    ``_normal_shooting``; the gates and the bin then follow as above.
    All of the above decisions are float32 (module docstring). p, q, n are
    also returned in float64 for the least-squares rows.
    """
    V = fl.V
    H, W, _ = V.shape
    mc = ml.cam
    fvalid = np.isfinite(V).all(-1) & np.isfinite(fl.N).all(-1)
    V32 = np.where(fvalid[..., None], V, np.nan).astype(F32)
    vx, vy, vz = V32[..., 0], V32[..., 1], V32[..., 2]
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        mx, my, mz = _xform32(xf.Rr, xf.tr, vx, vy, vz)
        px, py, pz = _xform32(xf.Rw, xf.tw, vx, vy, vz)
        ok = fvalid & (mz > F32(0))
        rz = F32(1.0) / mz
        uf = fma32(F32(mc.fx) * mx, rz, F32(mc.cx))
        vf = fma32(F32(mc.fy) * my, rz, F32(mc.cy))
        ur = np.rint(uf)
        vr = np.rint(vf)
        ok &= (ur >= 0) & (ur <= mc.width - 1) & (vr >= 0) & (vr <= mc.height - 1)
    ui = np.where(ok, ur, -1).astype(np.int64)
    vi = np.where(ok, vr, -1).astype(np.int64)
    if p.shoot_radius > 0:
        ui, vi = _normal_shooting(fl, ml, xf, ok, ui, vi, (px, py, pz), p.shoot_radius)
        ok &= ui >= 0
    uc = np.clip(ui, 0, mc.width - 1)
    vc = np.clip(vi, 0, mc.height - 1)
    q = ml.V[vc, uc]
    nq = ml.N[vc, uc]
    mvalid = np.isfinite(q).all(-1) & np.isfinite(nq).all(-1) & (nq != 0).any(-1)
    ok &= mvalid
    q32 = q.astype(F32)
    with np.errstate(invalid="ignore", over="ignore"):
        dx = px - q32[..., 0]
        dy = py - q32[..., 1]
        dz = pz - q32[..., 2]
        d2 = fma32(dz, dz, fma32(dy, dy, dx * dx))
        d32 = np.sqrt(d2)
        ok &= d32 < F32(p.d_max)
        if p.cos_angle_min > -1.0:
            N32 = fl.N.astype(F32)
            nx, ny, nz = _xform32(xf.Rw, np.zeros(3, F32), N32[..., 0], N32[..., 1], N32[..., 2])
            n32 = nq.astype(F32)
            dot = nx * n32[..., 0] + ny * n32[..., 1]
            dot = dot + nz * n32[..., 2]
            ok &= dot >= F32(p.cos_angle_min)
        scale = F32(p.hist_bins / p.d_max)
        kf = np.floor(d32 * scale)
    k = np.where(ok, np.minimum(np.nan_to_num(kf, nan=0.0), p.hist_bins - 1), -1).astype(np.int64)
    T = np.asarray(T_cur, np.float64)
    P64 = V @ T[:3, :3].T + T[:3, 3]
    return Assoc(ok, np.where(ok, ui, -1), np.where(ok, vi, -1), k, d32, P64, q, nq)


def _normal_shooting(fl: FrameLevel, ml: ModelLevel, xf: Xf32, ok, ui, vi, p32, w: int):
    """Normal-shooting association (Sec. 3.3): among the valid model pixels
    of the (2w+1)^2 window around the projected pixel (ui, vi), the one whose
    vertex q lies closest to the line through the frame point p along the
    frame normal n (R_cur n_frame, unit). Squared distance to the line, in
    float32 with each operation rounded in this order:
      e = q - p;  s = (e_x n_x + e_y n_y) + e_z n_z;
      l2 = ((e_x e_x + e_y e_y) + e_z e_z) - s s.
    Candidates are visited row by row (dy = -w..w, then dx = -w..w inside);
    a candidate replaces the best only with a strictly smaller l2, so ties
    keep the first. Returns the chosen (u, v), -1 where no candidate is valid
    or the projection itself failed."""
    mc = ml.cam
    N32 = np.where(ok[..., None], fl.N, 0.0).astype(F32)
    nx, ny, nz = _xform32(xf.Rw, np.zeros(3, F32), N32[..., 0], N32[..., 1], N32[..., 2])
    px, py, pz = p32
    best = np.full(ok.shape, np.inf, F32)
    bu = np.full(ok.shape, -1, np.int64)
    bv = np.full(ok.shape, -1, np.int64)
    mvalid = np.isfinite(ml.V).all(-1) & np.isfinite(ml.N).all(-1) & (ml.N != 0).any(-1)
    V32 = ml.V.astype(F32)
    for dy in range(-w, w + 1):
        for dx in range(-w, w + 1):
            cu, cv = ui + dx, vi + dy
            inside = ok & (cu >= 0) & (cu <= mc.width - 1) & (cv >= 0) & (cv <= mc.height - 1)
            cuc = np.clip(cu, 0, mc.width - 1)
            cvc = np.clip(cv, 0, mc.height - 1)
            valid = inside & mvalid[cvc, cuc]
            q = V32[cvc, cuc]
            with np.errstate(invalid="ignore", over="ignore"):
                ex = q[..., 0] - px
                ey = q[..., 1] - py
                ez = q[..., 2] - pz
                sd = ex * nx + ey * ny
                sd = sd + ez * nz
                ee = ex * ex + ey * ey
                ee = ee + ez * ez
                l2 = ee - sd * sd
                better = valid & (l2 < best)
            best = np.where(better, l2, best)
            bu = np.where(better, cu, bu)
            bv = np.where(better, cv, bv)
    return bu, bv


def histogram(a: Assoc, bins: int) -> np.ndarray:
    """PDF of the matched pairs' distances as bin counts (Sec. 3.2)."""
    return np.bincount(a.k[a.valid], minlength=bins).astype(np.int64)


def median_bin(H) -> int:
    """Median from the CDF, to the histogram's resolution (Sec. 3.3).

    k_med = min { k : 2 * sum_{j<=k} H[j] >= N }, N = sum H.
    """
    C = np.cumsum(H)
    N = C[-1]
    return int(np.argmax(2 * C >= N))


def band(kmed: int, kappa: float, bins: int):
    """Bins that gather around the median (Sec. 3.3): |d - m| <= kappa m in bin units.

    With m = k_med + 1/2 (the median bin's centre, in bins):
    k_hi = min(B - 1, floor((1 + kappa) m)), k_lo = max(0, ceil((1 - kappa) m) - 1).
    """
    m = kmed + 0.5
    khi = min(bins - 1, int(math.floor((1.0 + kappa) * m)))
    klo = max(0, int(math.ceil((1.0 - kappa) * m)) - 1)
    return klo, khi


def converged(history, window: int) -> bool:
    """Sec. 3.4: the median bin equal over `window` successive iterations."""
    return len(history) >= window and len(set(history[-window:])) == 1


# ----------------------------------------------------------------------------
# linear least squares (Eq. 3 - 5)
# ----------------------------------------------------------------------------
def ls_rows(p, q, n):
    """Rows of Eq. 3 for the increment x = (alpha, beta, gamma, tx, ty, tz).

    With the small-angle transform of Eq. 2, M p = p + w x p + t, so the
    residual (M p - q) . n = w . (p x n) + t . n - n . (q - p) is linear in x:
    a = [(p x n)^T, n^T], b = n . (q - p).
    """
    a = np.concatenate([np.cross(p, n), n], axis=-1)
    b = np.einsum("ik,ik->i", n, q - p)
    return a, b


def normal_equations(a, b):
    """A^T A (6x6) and A^T b (6) of Eq. 3 plus sum b^2."""
    return a.T @ a, a.T @ b, float(b @ b)


def lambda_of_n(mode: int, c: float, n: int) -> float:
    """lambda as a constant or a function of n (Sec. 3.1; schedules of the lambda table).

    The table prints the last form as -c ln(n); for n > 1 that is negative and
    makes the system indefinite, so it is read as c ln(n).
    """
    if mode == LAMBDA_CONST:
        return c
    if mode == LAMBDA_C_SQRT_N:
        return c / math.sqrt(n)
    if mode == LAMBDA_C_N:
        return c / n
    if mode == LAMBDA_C_N2:
        return c / (n * n)
    if mode == LAMBDA_C_LOG_N:
        return c * math.log(n)
    raise ValueError(mode)


def regularised_system(AtA, Atb, lam: float, n: int):
    """Eq. 5: (A^T A + 2 lambda n P^T P) x = A^T b with P = [I3 | 0]."""
    P = np.hstack([np.eye(3), np.zeros((3, 3))])
    return AtA + 2.0 * lam * n * (P.T @ P), Atb


def rotation_log(R):
    """Rotation vector w with Exp(w) = R, angle in [0, pi): with
    v = (R21 - R12, R02 - R20, R10 - R01), sin(t) = |v| / 2 and
    cos(t) = (trace R - 1) / 2, t = atan2(sin t, cos t) and w = t / (2 sin t) v
    (t / (2 sin t) = (1 + t^2 / 6) / 2 to 1e-17 below t = 1e-4)."""
    R = np.asarray(R, np.float64)
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    s = 0.5 * math.sqrt(float(v @ v))
    c = 0.5 * (R[0, 0] + R[1, 1] + R[2, 2] - 1.0)
    t = math.atan2(s, c)
    f = 0.5 * (1.0 + t * t / 6.0) if t < 1e-4 else t / (2.0 * s)
    return f * v


def anchored_rhs(Atb, lam: float, n: int, R_cur, R_prior):
    """Prior-anchored variant of Eq. 4/5 (an extension, not in the paper):
    instead of the increment's rotation, the rotation of the UPDATED pose is
    held toward the IMU prior, lambda |log(Exp(w) R_cur R_prior^T)|^2, linearised as
    lambda |w + r|^2 with r = log(R_cur R_prior^T). The matrix of Eq. 5 is
    unchanged; the right-hand side becomes A^T b - 2 lambda n P^T r."""
    r = rotation_log(np.asarray(R_cur, np.float64) @ np.asarray(R_prior, np.float64).T)
    g = np.array(Atb, np.float64).copy()
    g[:3] -= 2.0 * lam * n * r
    return g


def cholesky_solve(Hm, g):
    """Solve H x = g by a Cholesky factorisation.

    Returns None (degenerate system) when a pivot is not above 1e-12 times its
    own diagonal entry H[j, j]; a per-column test, so a large regulariser on the
    rotation block does not mask a well-posed translation block or vice versa.
    """
    Hm = np.asarray(Hm, np.float64)
    m = Hm.shape[0]
    L = np.zeros_like(Hm)
    for j in range(m):
        s = Hm[j, j] - L[j, :j] @ L[j, :j]
        if not (s > 1e-12 * Hm[j, j]):
            return None
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, m):
            L[i, j] = (Hm[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    y = np.zeros(m)
    for i in range(m):
        y[i] = (g[i] - L[i, :i] @ y[:i]) / L[i, i]
    x = np.zeros(m)
    for i in reversed(range(m)):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def rodrigues(w):
    """Exp of a rotation vector: I + sin(t)/t [w]x + (1 - cos t)/t^2 [w]x^2."""
    w = np.asarray(w, np.float64)
    t = math.sqrt(float(w @ w))
    Kx = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if t < 1e-12:
        return np.eye(3) + Kx + 0.5 * (Kx @ Kx)
    return np.eye(3) + (math.sin(t) / t) * Kx + ((1.0 - math.cos(t)) / (t * t)) * (Kx @ Kx)


def apply_increment(x, T):
    """T <- [dR | dt] T with dR = Exp(alpha, beta, gamma), dt = (tx, ty, tz)."""
    D = np.eye(4)
    D[:3, :3] = rodrigues(x[:3])
    D[:3, 3] = x[3:]
    return D @ np.asarray(T, np.float64)


# ----------------------------------------------------------------------------
# the alignment loop
# ----------------------------------------------------------------------------
@dataclass
class IterRecord:
    level: int
    it: int
    N: int
    kmed: int
    klo: int
    khi: int
    n: int
    x: np.ndarray
    AtA: np.ndarray
    Atb: np.ndarray
    sum_b2: float
    lam: float


@dataclass
class Result:
    pose: np.ndarray
    status: int
    iters: list
    total_iters: int
    inliers: int
    valid_pairs: int
    median_bin: list
    rms_residual: float
    trace: list = field(default_factory=list)


def seed_pose(prior_R, init_pose, p: Params):
    """T0 = [R_prior | t_init] when the IMU prior is used (Sec. 3), else init_pose."""
    T = np.array(init_pose, np.float64).reshape(4, 4).copy()
    if prior_R is not None and (p.flags & USE_PRIOR):
        T[:3, :3] = np.asarray(prior_R, np.float64).reshape(3, 3)
    return T


def align(frame: list, model: list, model_pose, prior_R, init_pose, lam: float,
          p: Params, keep_trace=False) -> Result:
    """Coarse-to-fine regularised point-to-plane ICP, coarsest level first.

    Per iteration, in the paper's order: associate + distance histogram
    (Sec. 3.2); median and band, inlier mask (Sec. 3.3); rows of Eq. 3 over the
    inliers; regularised normal equations (Eq. 5) with n = inlier count;
    Cholesky solve; T <- [Exp(w) | t] T; convergence test on the median
    (Sec. 3.4). ``lam`` is the constant c of the lambda schedule (a negative
    value selects p.lambda_c).
    """
    c = p.lambda_c if lam < 0 else lam
    T_m = np.asarray(model_pose, np.float64).reshape(4, 4)
    T = seed_pose(prior_R, init_pose, p)
    iters = [0] * p.levels
    med = [-1] * p.levels
    total = 0
    status = OK
    last_n = last_N = 0
    rms = 0.0
    trace = []
    for l in reversed(range(p.levels)):
        hist = []
        conv = False
        for it in range(p.max_iters[l]):
            xf = f32_transforms(T, T_m)
            a = associate(frame[l], model[l], T, xf, p)
            Hh = histogram(a, p.hist_bins)
            N = int(Hh.sum())
            if N < p.n_min:
                status = TOO_FEW_INLIERS
                break
            kmed = median_bin(Hh)
            if p.flags & USE_FILTER:
                klo, khi = band(kmed, p.band_kappa, p.hist_bins)
            else:
                klo, khi = 0, p.hist_bins - 1
            inl = a.valid & (a.k >= klo) & (a.k <= khi)
            n = int(inl.sum())
            if n < p.n_min:
                status = TOO_FEW_INLIERS
                break
            A, b = ls_rows(a.p[inl], a.q[inl], a.n[inl])
            AtA, Atb, sb2 = normal_equations(A, b)
            lamv = lambda_of_n(p.lambda_mode, c, n)
            Hs, g = regularised_system(AtA, Atb, lamv, n)
            if (p.flags & PRIOR_ANCHORED) and prior_R is not None:
                g = anchored_rhs(Atb, lamv, n, T[:3, :3], np.asarray(prior_R, np.float64).reshape(3, 3))
            x = cholesky_solve(Hs, g)
            if x is None:
                status = DEGENERATE
                break
            T = apply_increment(x, T)
            iters[l] += 1
            total += 1
            med[l] = kmed
            last_n, last_N = n, N
            rms = math.sqrt(sb2 / n)
            if keep_trace:
                trace.append(IterRecord(l, it, N, kmed, klo, khi, n, x, AtA, Atb, sb2, lamv))
            hist.append(kmed)
            if (p.flags & USE_CONVERGENCE) and converged(hist, p.conv_window):
                conv = True
                break
        if status < 0:
            break
        if l == 0 and (p.flags & USE_CONVERGENCE) and not conv:
            status = NOT_CONVERGED
    return Result(T, status, iters, total, last_n, last_N, med, rms, trace)


def align_from_depth(depth, K: Cam, model_V, model_N, Km: Cam, model_pose, prior_R,
                     init_pose, lam, p: Params, keep_trace=False) -> Result:
    fr = build_frame_pyramid(depth, K, p)
    mo = build_model_pyramid(model_V, model_N, Km, p.levels)
    return align(fr, mo, model_pose, prior_R, init_pose, lam, p, keep_trace)


def rotation_angle(Ra, Rb) -> float:
    """Angle of Ra Rb^T in radians, from |Ra - Rb|_F = 2 sqrt(2) sin(angle / 2).

    (The chord form keeps full precision for tiny angles, where acos of the
    trace loses half the digits.)
    """
    f = float(np.linalg.norm(np.asarray(Ra, np.float64) - np.asarray(Rb, np.float64)))
    return 2.0 * math.asin(min(1.0, f / (2.0 * math.sqrt(2.0))))
