"""Pins of the oracle's front end (bilateral filter, pyramid, vertex/normal maps).

Each test checks the oracle against something other than itself: a library
routine it reduces to, a closed form, or the analytic scene geometry.
"""
import math

import numpy as np
import pytest

from oracle import kf_oracle as O
from synth import scenes as S


def test_bilateral_constant_depth_is_fixed_point():
    D = np.full((20, 24), 2.5)
    out = O.bilateral_filter(D, 4.0, 0.03, 2)
    assert np.allclose(out, 2.5, rtol=0, atol=1e-15)


def test_bilateral_reduces_to_normalised_gaussian_when_range_kernel_is_flat():
    # sigma_r -> infinity: w = exp(-|d|^2 / 2 sigma_s^2); on interior pixels of an
    # all-valid image the filter equals scipy's correlation with the normalised kernel.
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    D = 1.0 + rng.random((30, 40))
    r, ss = 2, 1.7
    out = O.bilateral_filter(D, ss, 1e12, r)
    g = np.array([[math.exp(-(x * x + y * y) / (2 * ss * ss)) for x in range(-r, r + 1)]
                  for y in range(-r, r + 1)])
    ref = ndimage.correlate(D, g / g.sum(), mode="constant")
    assert np.allclose(out[r:-r, r:-r], ref[r:-r, r:-r], rtol=0, atol=1e-12)


def test_bilateral_preserves_depth_step_and_holes():
    D = np.full((16, 16), 1.0)
    D[:, 8:] = 3.0           # 2 m step >> sigma_r
    D[5, 5] = 0.0            # a hole stays a hole
    out = O.bilateral_filter(D, 4.0, 0.03, 2)
    assert out[5, 5] == 0.0
    assert np.allclose(out[:, :8][D[:, :8] > 0], 1.0, atol=1e-12)
    assert np.allclose(out[:, 8:], 3.0, atol=1e-12)


def test_downsample_constant_and_similarity_rule():
    D = np.full((8, 8), 2.0)
    assert np.allclose(O.downsample(D, 0.03), 2.0)
    # block: anchor 1.00 (top-left), 1.05 within 3 sigma_r = 0.09, 1.50 outside, hole
    B = np.array([[1.00, 1.05], [1.50, 0.0]])
    assert O.downsample(B, 0.03)[0, 0] == pytest.approx((1.00 + 1.05) / 2, abs=1e-15)
    # anchor is the first VALID depth in scan order (0,0),(1,0),(0,1),(1,1)
    B = np.array([[0.0, 2.0], [2.05, 2.5]])
    assert O.downsample(B, 0.03)[0, 0] == pytest.approx((2.0 + 2.05) / 2, abs=1e-15)
    assert O.downsample(np.zeros((2, 2)), 0.03)[0, 0] == 0.0


def test_level_intrinsics_make_downsampled_vertices_the_block_mean():
    # Fronto-parallel wall at Z: a level-1 vertex, back-projected with the level-1
    # intrinsics, is the mean of its four level-0 vertices (pins c' = (c - 0.5)/2).
    K = O.Cam(32, 24, 30.0, 31.0, 15.5, 11.5)
    cams = O.frame_level_cams(K, 3)
    Z = 1.7
    D0 = np.full((24, 32), Z)
    V0 = O.vertex_map(D0, cams[0])
    V1 = O.vertex_map(O.downsample(D0, 0.03), cams[1])
    mean4 = 0.25 * (V0[0::2, 0::2] + V0[0::2, 1::2] + V0[1::2, 0::2] + V0[1::2, 1::2])
    assert np.allclose(V1, mean4, atol=1e-14)
    assert (cams[2].width, cams[2].height) == (8, 6)
    assert cams[2].fx == pytest.approx(7.5)


def test_model_level_intrinsics_match_subsampled_render():
    # Subsampling a render at even pixels equals rendering with f/2, c/2.
    sc = S.room_scene()
    pose = S.look_at((0.05, -0.02, 0.0), (0.1, 0.0, 3.0))
    K = S.Intrinsics(64, 48, 56.0, 56.0, 32.0, 24.0)
    V0, N0 = S.render_model(sc, pose, K)
    mo = O.build_model_pyramid(V0, N0, O.Cam(*K.as_tuple()), 3)
    c2 = mo[2].cam
    V2, _ = S.render_model(sc, pose, S.Intrinsics(c2.width, c2.height, c2.fx, c2.fy, c2.cx, c2.cy))
    assert np.allclose(mo[2].V, V2, atol=1e-5, equal_nan=True)


def test_vertex_map_back_projects_the_rendered_surface():
    sc = S.room_scene()
    pose = S.look_at((0.0, 0.0, 0.0), (0.0, 0.0, 3.0))
    K = S.Intrinsics(40, 30, 35.0, 35.0, 19.5, 14.5)
    s, P, _ = S.raycast(sc, pose, K)
    V = O.vertex_map(s, O.Cam(*K.as_tuple()))
    Pw = V @ pose[:3, :3].T + pose[:3, 3]
    ok = np.isfinite(s)
    assert np.allclose(Pw[ok], P[ok], atol=1e-12)


def test_normals_of_planes_match_scene_geometry_and_face_camera():
    sc = S.planar_scene()
    pose = S.look_at((0.1, 0.0, 0.2), (0.3, 0.1, 3.0))
    K = S.Intrinsics(80, 60, 70.0, 70.0, 39.5, 29.5)
    s, Pw, Nw = S.raycast(sc, pose, K)
    V = O.vertex_map(s, O.Cam(*K.as_tuple()))
    N = O.normal_map(V)
    Nc = Nw @ pose[:3, :3]            # world -> camera
    # pixels whose right and lower neighbours lie on the same plane
    def on_plane(dy, dx):
        nb_p = Pw[dy:Pw.shape[0] - 1 + dy, dx:Pw.shape[1] - 1 + dx]
        nb_n = Nw[dy:Nw.shape[0] - 1 + dy, dx:Nw.shape[1] - 1 + dx]
        c_p, c_n = Pw[:-1, :-1], Nw[:-1, :-1]
        return ((np.abs(np.einsum("hwk,hwk->hw", nb_p - c_p, c_n)) < 1e-9)
                & (np.abs(nb_n - c_n).max(-1) < 1e-12))
    same = np.zeros(s.shape, bool)
    same[:-1, :-1] = on_plane(0, 1) & on_plane(1, 0)
    ok = same & np.isfinite(N).all(-1)
    assert ok.sum() > 0.8 * s.size
    assert np.allclose(N[ok], Nc[ok], atol=1e-9)
    assert (np.einsum("hwk,hwk->hw", N[ok][None], V[ok][None]) < 0).all()
    assert np.isnan(N[-1]).all() and np.isnan(N[:, -1]).all()


def test_float32_vertex_map_is_the_rounded_back_projection():
    """vertex_map32 is the float32 chain ((u - c) z) (1 / f): within three
    float32 roundings of the float64 back-projection, exact on the optical
    axis, and worked by hand at one pixel."""
    K = O.Cam(64, 48, 60.0, 61.0, 31.5, 23.5)
    rng = np.random.default_rng(3)
    D = rng.uniform(0.5, 4.0, (48, 64)).astype(np.float32)
    D[5, 6] = 0.0
    V = O.vertex_map(D, K)
    V32 = O.vertex_map32(D, K)
    ok = D > 0
    assert (np.isfinite(V32).all(-1) == ok).all()
    rel = np.abs(V32[ok] - V[ok]) / np.maximum(np.abs(V[ok]), 1e-30)
    assert rel.max() <= 3 * 2.0 ** -24
    assert (V32[..., 2][ok] == D[ok]).all()
    # pixel (u, v) = (40, 10): x = float32(float32(8.5 z) * float32(1 / 60))
    z = np.float32(D[10, 40])
    x = np.float32(np.float32(np.float32(40) - np.float32(31.5)) * z) * (np.float32(1) / np.float32(60.0))
    y = np.float32(np.float32(np.float32(10) - np.float32(23.5)) * z) * (np.float32(1) / np.float32(61.0))
    assert V32[10, 40, 0] == x and V32[10, 40, 1] == y


def test_normal_orientation_is_a_float32_decision_before_normalising():
    """The facing test uses the float32 cross product of the float32
    vertices: a normal flips exactly where s = c . v > 0, and an edge-on
    configuration (c . v = 0) keeps the cross product's own sign."""
    V = np.full((3, 3, 3), np.nan)
    # a wall at z = 2 seen head-on: a = (+x), b = (+y), a x b = +z, c . v > 0: flipped
    V[0, 0] = (0.0, 0.0, 2.0)
    V[0, 1] = (0.01, 0.0, 2.0)
    V[1, 0] = (0.0, 0.01, 2.0)
    N = O.normal_map(V)
    assert np.allclose(N[0, 0], (0.0, 0.0, -1.0))
    # a plane containing the viewing ray (edge-on): s = 0 exactly, no flip
    V[0, 0] = (0.0, 0.0, 2.0)
    V[0, 1] = (0.0, 0.0, 3.0)
    V[1, 0] = (0.0, 0.01, 2.0)
    N = O.normal_map(V)
    c = np.cross(V[0, 1] - V[0, 0], V[1, 0] - V[0, 0])
    assert np.dot(c, V[0, 0]) == 0.0
    assert np.allclose(N[0, 0], c / np.linalg.norm(c))
    # float32 decisions follow the float32 vertices given, not the float64 ones
    V64 = np.zeros((3, 3, 3))
    V64[0, 0] = (0.0, 0.0, 2.0)
    V64[0, 1] = (0.01, 0.0, 2.0)
    V64[1, 0] = (0.0, 0.01, 2.0)
    V32 = V64.astype(np.float32)
    V32[0, 1, 2] = np.float32(np.nan)
    assert np.isnan(O.normal_map(V64, V32)[0, 0]).all()


def test_frame_pyramid_sizes_and_holes():
    K = O.Cam(64, 48, 60.0, 60.0, 31.5, 23.5)
    D = np.full((48, 64), 2.0)
    D[10, 10] = 0.0
    D[20, 30] = np.nan
    fr = O.build_frame_pyramid(D, K, O.Params())
    assert [f.V.shape[:2] for f in fr] == [(48, 64), (24, 32), (12, 16)]
    assert np.isnan(fr[0].V[10, 10]).all() and np.isnan(fr[0].V[20, 30]).all()
    assert np.isfinite(fr[1].V[5, 5]).all()      # a single hole does not empty a block
