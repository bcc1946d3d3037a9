"""CPU oracle of the frame normals the paper names for its own pipeline
(Sec. 3.3): surface normals from integral images (Holzer et al. 2012, the
average-3D-gradient form with a window adapted to depth and to depth
discontinuities).

TEST INFRASTRUCTURE ONLY: plain, slow numpy. Only the test suite and the
bench's CPU legs may use it; the CUDA library never does and shares no code
with it.

The paper names the method and gives no parameters. The reading taken here,
for one pyramid level l with depth z (float32, 0 = none) and intrinsics
(f_x, f_y, c_x, c_y):

* vertex (float32, each operation rounded, the front end's own vertex):
  v = (((x - c_x) z) (1 / f_x), ((y - c_y) z) (1 / f_y), z);
* fixed point: Q = round-half-even(v * 2^20), integers in units of 2^-20 m,
  so that every window sum below is exact whatever order adds it (the kernel
  sums through integral images, this oracle sums the rectangles directly);
* edges: a pixel is an edge when its depth is not valid, or when one of its
  4-neighbours inside the image is not valid or differs from it by more than
  delta z (float32: |z_w - z| > delta z);
* dist(u): chessboard distance to the nearest edge pixel, capped at
  r_max + 1 (the window of half-size dist - 1 holds no edge);
* half-size r(u) = min(floor((a + b z) 2^-l), dist(u) - 1, distance to the
  image border, r_max), (a + b z) rounded to float32 as a + (b z);
  no normal unless r >= 1;
* gradients, exact integers over rows y-r..y+r (columns x-r..x+r):
  g_h = sum of Q over columns x+1..x+r  -  sum over columns x-r..x-1,
  g_v = sum of Q over rows    y+1..y+r  -  sum over rows    y-r..y-1;
* normal: g_h and g_v rounded to float32 and scaled by 2^-20 (exact), then
  c = g_h x g_v, |c|^2 = (c_x^2 + c_y^2) + c_z^2, s = sqrt(|c|^2),
  n = c / s, every operation a rounded float32 one; no normal where
  |c|^2 = 0; n flipped when (n_x v_x + n_y v_y) + n_z v_z > 0 (the camera is
  at the origin, normals face it).
A pixel without a normal has no vertex either (NaN), as in the front end.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
FIX_SCALE = F32(2.0 ** 20)
FIX_INV = F32(2.0 ** -20)


def vertex32(D, fx: float, fy: float, cx: float, cy: float):
    """(H, W, 3) float32 vertex map of depth D (float32), NaN where not valid."""
    z = np.asarray(D, F32)
    H, W = z.shape
    ux = (np.arange(W, dtype=F32) - F32(cx))[None, :]
    uy = (np.arange(H, dtype=F32) - F32(cy))[:, None]
    ifx = F32(1) / F32(fx)
    ify = F32(1) / F32(fy)
    V = np.stack([((ux * z).astype(F32) * ifx).astype(F32),
                  ((uy * z).astype(F32) * ify).astype(F32),
                  z], axis=-1).astype(F32)
    V[~valid_depth(z)] = np.nan
    return V


def valid_depth(z):
    z = np.asarray(z, F32)
    with np.errstate(invalid="ignore"):
        return np.isfinite(z) & (z > 0)


def fixed_point(V32):
    """Vertices in units of 2^-20 m (int64), 0 where not valid."""
    ok = np.isfinite(V32).all(-1)
    Q = np.rint(np.where(ok[..., None], V32, F32(0)) * FIX_SCALE).astype(np.int64)
    return Q


def edge_map(D, delta: float):
    """True where the pixel is not valid or a 4-neighbour inside the image is
    not valid or differs in depth by more than delta z (float32)."""
    z = np.asarray(D, F32)
    ok = valid_depth(z)
    H, W = z.shape
    E = ~ok
    thr = (F32(delta) * z).astype(F32)
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        y0, y1 = max(0, -dy), H - max(0, dy)
        x0, x1 = max(0, -dx), W - max(0, dx)
        zc = z[y0:y1, x0:x1]
        zn = z[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        okn = ok[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        with np.errstate(invalid="ignore", over="ignore"):
            jump = np.abs((zn - zc).astype(F32)) > thr[y0:y1, x0:x1]
        E[y0:y1, x0:x1] |= ~okn | jump
    return E


def chessboard_distance(E, cap: int):
    """Per pixel the smallest d such that the (2d+1)^2 square around it holds
    an edge pixel of E, or cap when none has d < cap."""
    H, W = E.shape
    dist = np.full((H, W), cap, np.int64)
    for d in range(cap - 1, -1, -1):
        hit = np.zeros((H, W), bool)
        for dy in range(-d, d + 1):
            for dx in range(-d, d + 1):
                y0, y1 = max(0, -dy), H - max(0, dy)
                x0, x1 = max(0, -dx), W - max(0, dx)
                if y0 < y1 and x0 < x1:
                    hit[y0:y1, x0:x1] |= E[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        dist[hit] = d
    return dist


def window_radius(D, level: int, a: float, b: float, delta: float, rmax: int):
    """Half-size r(u) of each pixel's window (values < 1: no normal)."""
    z = np.asarray(D, F32)
    H, W = z.shape
    E = edge_map(z, delta)
    dist = chessboard_distance(E, rmax + 1)
    with np.errstate(invalid="ignore", over="ignore"):
        t = (F32(a) + (F32(b) * z).astype(F32)).astype(F32) * F32(2.0 ** -level)
        t = np.where(np.isfinite(t), np.minimum(t, F32(rmax)), F32(0))
    rdd = np.floor(t).astype(np.int64)
    xs = np.arange(W)[None, :]
    ys = np.arange(H)[:, None]
    rimg = np.minimum(np.minimum(xs, W - 1 - xs), np.minimum(ys, H - 1 - ys))
    return np.minimum(np.minimum(rdd, dist - 1), np.minimum(rimg, rmax))


def box_sum(Q, dx0: int, dx1: int, dy0: int, dy1: int):
    """S[y, x] = sum of Q[y + dy, x + dx] over dy0 <= dy <= dy1 and
    dx0 <= dx <= dx1 (zero outside the image), exact for integers."""
    H, W = Q.shape[:2]

    def shifted(A, dy, dx):
        out = np.zeros_like(A)
        y0, y1 = max(0, -dy), H - max(0, dy)
        x0, x1 = max(0, -dx), W - max(0, dx)
        if y0 < y1 and x0 < x1:
            out[y0:y1, x0:x1] = A[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        return out

    rows = np.zeros_like(Q)
    for dx in range(dx0, dx1 + 1):
        rows += shifted(Q, 0, dx)
    S = np.zeros_like(Q)
    for dy in range(dy0, dy1 + 1):
        S += shifted(rows, dy, 0)
    return S


def gradients(Q, r: int):
    """Exact integer (g_h, g_v) of every pixel for half-size r."""
    gh = box_sum(Q, 1, r, -r, r) - box_sum(Q, -r, -1, -r, r)
    gv = box_sum(Q, -r, r, 1, r) - box_sum(Q, -r, r, -r, -1)
    return gh, gv


def normals_from_gradients(gh, gv, V32):
    """float32 unit normals from integer gradients (module docstring), NaN
    where the cross product vanishes; flipped to face the camera."""
    h = gh.astype(np.float64).astype(F32) * FIX_INV
    v = gv.astype(np.float64).astype(F32) * FIX_INV
    cx = (h[..., 1] * v[..., 2]).astype(F32) - (h[..., 2] * v[..., 1]).astype(F32)
    cy = (h[..., 2] * v[..., 0]).astype(F32) - (h[..., 0] * v[..., 2]).astype(F32)
    cz = (h[..., 0] * v[..., 1]).astype(F32) - (h[..., 1] * v[..., 0]).astype(F32)
    n2 = ((cx * cx).astype(F32) + (cy * cy).astype(F32)).astype(F32) + (cz * cz).astype(F32)
    n2 = n2.astype(F32)
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.sqrt(n2).astype(F32)
        n = np.stack([cx / s, cy / s, cz / s], axis=-1).astype(F32)
        dot = ((n[..., 0] * V32[..., 0]).astype(F32) + (n[..., 1] * V32[..., 1]).astype(F32)).astype(F32)
        dot = (dot + (n[..., 2] * V32[..., 2]).astype(F32)).astype(F32)
    n = np.where((dot > 0)[..., None], -n, n).astype(F32)
    n[~(n2 > 0)] = np.nan
    return n


def integral_normals(D, fx: float, fy: float, cx: float, cy: float, level: int,
                     a: float = 2.0, b: float = 1.0, delta: float = 0.02, rmax: int = 8):
    """(V32, N32) of one level: float32 vertex and integral-image normal maps,
    both NaN where the pixel has no normal."""
    z = np.asarray(D, F32)
    V32 = vertex32(z, fx, fy, cx, cy)
    Q = fixed_point(V32)
    r = window_radius(z, level, a, b, delta, rmax)
    N = np.full(V32.shape, np.nan, F32)
    for rr in range(1, rmax + 1):
        m = r == rr
        if not m.any():
            continue
        gh, gv = gradients(Q, rr)
        N[m] = normals_from_gradients(gh, gv, V32)[m]
    ok = np.isfinite(N).all(-1)
    V = np.where(ok[..., None], V32, F32(np.nan)).astype(F32)
    return V, np.where(ok[..., None], N, F32(np.nan)).astype(F32)
