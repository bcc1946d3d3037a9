"""Pins of the oracle's projective association, histogram, median and band."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import kf_oracle as O
from synth import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _levels(depth, K, V, N, Km, p):
    fr = O.build_frame_pyramid(depth, O.Cam(*K.as_tuple()), p)
    mo = O.build_model_pyramid(V, N, O.Cam(*Km.as_tuple()), p.levels)
    return fr, mo


def test_identity_pose_associates_every_pixel_with_itself():
    sc = S.room_scene()
    pose = S.look_at((0.0, 0.0, 0.0), (0.1, 0.0, 3.0))
    K = S.Intrinsics(48, 36, 42.0, 42.0, 23.5, 17.5)
    s, _, _ = S.raycast(sc, pose, K)
    V, N = S.render_model(sc, pose, K)
    p = O.Params(levels=1, max_iters=(3,), bilateral_radius=0)
    fr, mo = _levels(s, K, V, N, K, p)
    a = O.associate(fr[0], mo[0], pose, O.f32_transforms(pose, pose), p)
    vv, uu = np.nonzero(a.valid)
    assert a.valid.sum() > 0.9 * (47 * 35)
    assert (a.ui[a.valid] == uu).all() and (a.vi[a.valid] == vv).all()
    assert (a.k[a.valid] == 0).all()


def test_one_pixel_translation_shifts_association_by_one_column():
    # Wall at z = Z seen head-on; the frame camera sits delta = Z / fx to the +x
    # side of the model camera, so frame pixel u sees the point that the model
    # camera images at u + 1.
    Z, f = 2.0, 50.0
    sc = S.Scene(planes=[((0.0, 0.0, -1.0), -Z)])
    K = S.Intrinsics(40, 30, f, f, 19.5, 14.5)
    Tm = np.eye(4)
    Tf = np.eye(4)
    Tf[0, 3] = Z / f
    s, _, _ = S.raycast(sc, Tf, K)
    V, N = S.render_model(sc, Tm, K)
    p = O.Params(levels=1, max_iters=(3,), bilateral_radius=0)
    fr, mo = _levels(s, K, V, N, K, p)
    a = O.associate(fr[0], mo[0], Tf, O.f32_transforms(Tf, Tm), p)
    vv, uu = np.nonzero(a.valid)
    assert len(uu) == 39 * 29                      # every pixel with a valid frame normal
    assert (a.ui[a.valid] == uu + 1).all() and (a.vi[a.valid] == vv).all()
    # the matched points coincide: d = 0 up to float32 rounding
    assert (a.k[a.valid] == 0).all()


def _exact_projection(v32, T, Tm, cam):
    """Rational projection of float32 vertex v under float64 poses (no rounding)."""
    Fr = lambda x: Fraction(float(x))
    p = [sum(Fr(T[i][j]) * Fr(v32[j]) for j in range(3)) + Fr(T[i][3]) for i in range(3)]
    d = [p[k] - Fr(Tm[k][3]) for k in range(3)]
    m = [sum(Fr(Tm[k][i]) * d[k] for k in range(3)) for i in range(3)]
    if m[2] <= 0:
        return None
    return (Fr(cam.fx) * m[0] / m[2] + Fr(cam.cx), Fr(cam.fy) * m[1] / m[2] + Fr(cam.cy))


def test_association_matches_exact_rational_projection_on_a_tiny_frame():
    pr = S.config1_tiny()
    K = O.Cam(16, 12, 14.0, 14.0, 8.0, 6.0)
    D = pr.depth[::10, ::10].astype(np.float64)
    Ks = S.Intrinsics(16, 12, 14.0, 14.0, 8.0, 6.0)
    V, N = S.render_model(S.room_scene(), pr.model_pose, Ks)
    p = O.Params(levels=1, max_iters=(1,), bilateral_radius=0, d_max=10.0)
    fr, mo = _levels(D, Ks, V, N, Ks, p)
    T = O.seed_pose(pr.prior_R, pr.init_pose, p)
    a = O.associate(fr[0], mo[0], T, O.f32_transforms(T, pr.model_pose), p)
    v32 = np.where(np.isfinite(fr[0].V), fr[0].V, 0).astype(np.float32)
    checked = 0
    for y in range(12):
        for x in range(16):
            if not (np.isfinite(fr[0].V[y, x]).all() and np.isfinite(fr[0].N[y, x]).all()):
                assert not a.valid[y, x]
                continue
            e = _exact_projection(v32[y, x], T, pr.model_pose, K)
            if e is None:
                continue
            # skip projections within 1e-3 px of a rounding boundary (float32 ties)
            if any(abs((c - math.floor(c)) - Fraction(1, 2)) < Fraction(1, 1000) for c in e):
                continue
            ue, ve = round(e[0]), round(e[1])
            inside = 0 <= ue < 16 and 0 <= ve < 12
            if not inside:
                assert not a.valid[y, x]
                continue
            q, n = mo[0].V[ve, ue], mo[0].N[ve, ue]
            if not np.isfinite(q).all():
                assert not a.valid[y, x]
                continue
            assert a.valid[y, x]
            assert (a.ui[y, x], a.vi[y, x]) == (ue, ve)
            checked += 1
    assert checked > 100


def test_distance_and_bin_agree_with_float64_brute_force():
    pr = S.config1_tiny()
    p = O.Params(levels=1, max_iters=(1,))
    fr, mo = _levels(pr.depth, pr.K, pr.model_vertex, pr.model_normal, pr.K, p)
    T = O.seed_pose(pr.prior_R, pr.init_pose, p)
    a = O.associate(fr[0], mo[0], T, O.f32_transforms(T, pr.model_pose), p)
    d64 = np.linalg.norm(a.p - a.q, axis=-1)[a.valid]
    # float32 points carry ~1 ulp of their 1-4 m coordinates (<= 5e-7 m) per operation
    assert np.allclose(a.d32[a.valid], d64, rtol=0, atol=2e-6)
    x = d64 * 3200.0
    safe = np.abs(x - np.rint(x)) > 1e-2
    assert (a.k[a.valid][safe] == np.floor(x[safe])).all()
    assert a.valid.sum() > 10000


def test_histogram_counts_and_median_against_sorted_list():
    rng = np.random.default_rng(7)
    for trial in range(50):
        Nn = int(rng.integers(1, 400))
        k = rng.integers(0, 64, size=Nn) if trial % 2 else (rng.gamma(2.0, 6.0, Nn)).astype(int).clip(0, 511)
        H = np.bincount(k, minlength=512)
        assert H.sum() == Nn
        kmed = O.median_bin(H)
        assert kmed == np.sort(k)[(Nn + 1) // 2 - 1]        # ceil(N/2)-th smallest


def test_band_and_median_on_hand_worked_histograms():
    with open(os.path.join(GOLDEN, "band_median_cases.txt")) as f:
        lines = [l for l in f if l.strip() and not l.startswith("#")]
    assert len(lines) == 7
    for line in lines:
        head, hist, want = [s.strip() for s in line.split("|")]
        bins, kappa = head.split()
        bins, kappa = int(bins), float(kappa)
        H = np.zeros(bins, int)
        for kv in hist.split(","):
            k, c = kv.split(":")
            H[int(k)] = int(c)
        kmed, klo, khi = map(int, want.split())
        assert O.median_bin(H) == kmed, line
        assert O.band(kmed, kappa, bins) == (klo, khi), line


def test_convergence_rule_needs_three_equal_medians():
    assert not O.converged([5, 5], 3)
    assert O.converged([5, 5, 5], 3)
    assert not O.converged([4, 5, 5], 3)
    assert O.converged([9, 4, 5, 5, 5], 3)
    assert not O.converged([5, 5, 5, 6], 3)


def test_angle_gate_rejects_pairs_on_different_surfaces():
    pr = S.config1_tiny()
    p_off = O.Params(levels=1, max_iters=(1,))
    p_on = O.Params(levels=1, max_iters=(1,), cos_angle_min=math.cos(math.radians(20)))
    fr, mo = _levels(pr.depth, pr.K, pr.model_vertex, pr.model_normal, pr.K, p_off)
    T = O.seed_pose(pr.prior_R, pr.init_pose, p_off)
    xf = O.f32_transforms(T, pr.model_pose)
    a0 = O.associate(fr[0], mo[0], T, xf, p_off)
    a1 = O.associate(fr[0], mo[0], T, xf, p_on)
    assert (a1.valid <= a0.valid).all()
    nf = fr[0].N @ T[:3, :3].T
    cosang = np.einsum("hwk,hwk->hw", nf, a0.n)
    clear = np.abs(cosang - math.cos(math.radians(20))) > 1e-4
    assert (a1.valid[a0.valid & clear] == (cosang >= math.cos(math.radians(20)))[a0.valid & clear]).all()
    assert a1.valid.sum() < a0.valid.sum()
