"""CUDA path vs the FP64 oracle, through the C ABI (needs a GPU).

Bars (see the oracle's module docstring for the precision rules):
  * association indices, histogram bins and counts: bit-exact (both sides take
    every decision in float32 with the same operation order);
  * front-end maps: validity masks exact, values within float32 rounding;
  * 29 normal-equation sums: per-sum tolerance of kfhelp.sum_tolerances;
  * final poses: 1e-5 rad and 1e-5 m; iteration counts and median bins equal.
"""
import math

import numpy as np
import pytest

from oracle import kf_oracle as O
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


# ---------------------------------------------------------------------------
# front end
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("size", [(640, 480), (100, 75)])
def test_frontend_maps_match_oracle_stages(size):
    pr = S.config2_kinect(0, *size)
    p, op = H.params()
    with H.Tracker(p, *size) as t:
        t.set_pair(pr)
        lv = t.frame_levels(3)
    cams = O.frame_level_cams(O.Cam(*pr.K.as_tuple()), 3)
    # bilateral filter (level 0) against the raw depth
    Db = O.bilateral_filter(pr.depth, op.bilateral_sigma_s, op.bilateral_sigma_r, op.bilateral_radius)
    D0 = lv[0][0]
    assert ((D0 > 0) == (Db > 0)).all()
    assert np.abs(D0 - Db).max() < 5e-6
    for l in range(3):
        D, V, N = lv[l]
        if l > 0:  # downsampling of the GPU's own level above: decisions exact
            Dd = O.downsample(lv[l - 1][0], op.bilateral_sigma_r)
            assert ((D > 0) == (Dd > 0)).all()
            assert np.abs(D - Dd).max() <= 4e-7 * max(1.0, float(Dd.max()))
        # vertices: the float32 back-projection, bit for bit
        V32 = O.vertex_map32(D, cams[l])
        No = O.normal_map(O.vertex_map(D, cams[l]), V32)
        ok_o = np.isfinite(V32).all(-1) & np.isfinite(No).all(-1)
        ok_g = np.isfinite(V).all(-1)
        assert (ok_o == ok_g).all(), l
        assert (V[ok_g] == V32[ok_g]).all(), l
        # normals: the same float32 decisions (exists, faces the camera) on
        # both sides, so every orientation agrees; the value differs from the
        # float64 normal of the same float32 vertices only by the kernel's
        # float32 cross product and its rsqrtf (2 ulp) normalisation
        Nv = O.normal_map(V32.astype(np.float64), V32)
        assert (np.isfinite(Nv).all(-1) == ok_g).all(), l
        assert (np.einsum("ik,ik->i", N[ok_g], Nv[ok_g]) > 0).all(), l
        assert (np.abs(N - Nv).max(-1)[ok_g] <= normal_bound(V32)[ok_g]).all(), l


def normal_bound(V32):
    """Per-pixel bound on |n_gpu - n|: float32 rounding of the differences,
    products and differences of the cross product (3u of each product plus u
    of the result), then rsqrtf (2 ulp), the rounding of l2 and the final
    products (8u in all), doubled."""
    u = 2.0 ** -24
    V = V32.astype(np.float64)
    B = np.full(V.shape[:2], np.inf)
    c = V[:-1, :-1]
    a = V[:-1, 1:] - c
    b = V[1:, :-1] - c
    terms = np.stack([np.abs(a[..., 1] * b[..., 2]) + np.abs(a[..., 2] * b[..., 1]),
                      np.abs(a[..., 2] * b[..., 0]) + np.abs(a[..., 0] * b[..., 2]),
                      np.abs(a[..., 0] * b[..., 1]) + np.abs(a[..., 1] * b[..., 0])], -1)
    cr = np.cross(a, b)
    with np.errstate(invalid="ignore", divide="ignore"):
        E = (3 * u * terms + u * np.abs(cr)).max(-1) / np.linalg.norm(cr, axis=-1)
    B[:-1, :-1] = 2.0 * (2.0 * E + 8 * u)
    return B


def test_model_maps_are_subsampled_and_holes_masked():
    pr = S.config2_kinect(1, 160, 120)
    pr.model_vertex[5, 7] = np.nan
    pr.model_normal[9, 9] = 0.0
    p, op = H.params()
    with H.Tracker(p, 160, 120) as t:
        t.set_pair(pr)
        ml = t.model_levels(3)
    mo = O.build_model_pyramid(pr.model_vertex, pr.model_normal, O.Cam(*pr.K.as_tuple()), 3)
    for l in range(3):
        V, N = ml[l]
        hole = ~(np.isfinite(mo[l].V).all(-1) & np.isfinite(mo[l].N).all(-1) & (mo[l].N != 0).any(-1))
        assert (np.isnan(V).all(-1) == hole).all()
        assert np.array_equal(V[~hole], mo[l].V[~hole].astype(np.float32))
        assert np.array_equal(N[~hole], mo[l].N[~hole].astype(np.float32))


# ---------------------------------------------------------------------------
# association + histogram: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case,size,gate", [(0, (640, 480), False), (1, (160, 120), False),
                                            (2, (333, 251), True)])
def test_association_and_histogram_are_bit_exact(case, size, gate):
    pr = S.config2_kinect(case, *size)
    kw = {"cos_angle_min": math.cos(math.radians(20))} if gate else {}
    p, op = H.params(**kw)
    with H.Tracker(p, *size) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
        T0 = O.seed_pose(pr.prior_R, pr.init_pose, op)
        rng = np.random.default_rng(case)
        for l in range(3):
            for trial in range(2):
                T = T0.copy()
                if trial:
                    T = O.apply_increment(np.r_[0.01 * rng.normal(size=3), 0.02 * rng.normal(size=3)], T)
                idx, b, hist = H.kf().kf_debug_associate(t.h, l, T, fr[l].V.shape[:2], p.hist_bins)
                a = O.associate(fr[l], mo[l], T, O.f32_transforms(T, pr.model_pose), op)
                mw = mo[l].cam.width
                want_idx = np.where(a.valid, a.vi * mw + a.ui, -1)
                assert np.array_equal(idx, want_idx), (l, trial, int((idx != want_idx).sum()))
                assert np.array_equal(b, np.where(a.valid, a.k, -1))
                assert np.array_equal(hist.astype(np.int64), O.histogram(a, p.hist_bins))


# ---------------------------------------------------------------------------
# filter + reduction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_filtered_normal_equation_sums(precision):
    pr = S.config2_kinect(3, 640, 480)
    p, op = H.params(precision=precision)
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
        T = O.seed_pose(pr.prior_R, pr.init_pose, op)
        for l in range(3):
            a = O.associate(fr[l], mo[l], T, O.f32_transforms(T, pr.model_pose), op)
            kmed = O.median_bin(O.histogram(a, p.hist_bins))
            for klo, khi in [O.band(kmed, 1.0, p.hist_bins), (0, p.hist_bins - 1), (3, kmed)]:
                inl = a.valid & (a.k >= klo) & (a.k <= khi)
                want, A, bb = H.oracle_sums(a, inl)
                got = H.kf().kf_debug_reduce(t.h, l, T, klo, khi)
                assert got[27] == want[27]
                tol = H.sum_tolerances(A, bb)
                bad = np.abs(got - want) > tol
                assert not bad.any(), (l, klo, khi, np.nonzero(bad), got[bad], want[bad])


# ---------------------------------------------------------------------------
# end to end
# ---------------------------------------------------------------------------
def _check_against_oracle(pose, res, ref, tol=1e-5):
    rot, tr = H.pose_err(pose, ref.pose)
    assert res.status == ref.status
    assert rot < tol and tr < tol, (rot, tr)
    L = len(ref.iters)
    assert list(res.iters)[:L] == ref.iters
    assert list(res.median_bin)[:L] == ref.median_bin
    # counts: equal up to pixels whose float32 decision sits at a rounding
    # boundary after the GPU's and the oracle's poses drift apart by ~1e-9
    assert abs(res.inliers - ref.inliers) <= 2 + 1e-4 * ref.inliers
    assert abs(res.valid_pairs - ref.valid_pairs) <= 2 + 1e-4 * ref.valid_pairs


@pytest.mark.parametrize("lam,prior", [(1e3, True), (0.0, True), (5.0, False)])
def test_alignment_on_gpu_maps_matches_oracle(lam, prior):
    pr = S.config2_kinect(4, 640, 480)
    p, op = H.params()
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
        st, pose, res = t.align(pr, lam, prior)
        trace = H.kf().kf_debug_trace(t.h)
    ref = O.align(fr, mo, pr.model_pose, pr.prior_R if prior else None, pr.init_pose, lam, op,
                  keep_trace=True)
    _check_against_oracle(pose, res, ref)
    assert [r.kmed for r in trace] == [r.kmed for r in ref.trace]
    assert all(abs(a.n - b.n) <= 2 + 1e-4 * b.n for a, b in zip(trace, ref.trace))


def test_config1_tiny_from_depth():
    pr = S.config1_tiny()
    p, op = H.params(levels=1, caps=(10,))
    with H.Tracker(p, 160, 120) as t:
        t.set_pair(pr, device=True)
        st, pose, res = t.align(pr)
    ref = O.align_from_depth(pr.depth, O.Cam(*pr.K.as_tuple()), pr.model_vertex, pr.model_normal,
                             O.Cam(*pr.K.as_tuple()), pr.model_pose, pr.prior_R, pr.init_pose,
                             pr.lam, op)
    _check_against_oracle(pose, res, ref)


@pytest.mark.parametrize("case", [0, 5])
def test_config2_kinect_from_depth(case):
    pr = S.config2_kinect(case)
    p, op = H.params()
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        st, pose, res = t.align(pr)
    ref = O.align_from_depth(pr.depth, O.Cam(*pr.K.as_tuple()), pr.model_vertex, pr.model_normal,
                             O.Cam(*pr.K.as_tuple()), pr.model_pose, pr.prior_R, pr.init_pose,
                             pr.lam, op)
    rot, tr = H.pose_err(pose, ref.pose)
    assert st == ref.status and rot < 1e-5 and tr < 1e-5, (st, ref.status, rot, tr)
    assert list(res.iters)[:3] == ref.iters


COS20 = float(np.cos(np.radians(20.0)))


def test_angle_gate_from_depth_fp32_matches_oracle():
    """The normal-angle gate at cos 20 deg (the original KinectFusion gate)
    from raw depth: the frame normals feed a discrete decision, so their
    orientation has to agree with the oracle's pixel for pixel."""
    pr = S.config2_kinect(7)
    p, op = H.params(cos_angle_min=COS20)
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        st, pose, res = t.align(pr)
    ref = O.align_from_depth(pr.depth, O.Cam(*pr.K.as_tuple()), pr.model_vertex, pr.model_normal,
                             O.Cam(*pr.K.as_tuple()), pr.model_pose, pr.prior_R, pr.init_pose,
                             pr.lam, op)
    rot, tr = H.pose_err(pose, ref.pose)
    assert st == ref.status and rot < 1e-5 and tr < 1e-5, (st, ref.status, rot, tr)
    assert list(res.iters)[:3] == ref.iters and list(res.median_bin)[:3] == ref.median_bin


def test_angle_gate_from_depth_fp16_matches_oracle_on_dequantised_maps():
    pr = S.config2_kinect(8)
    p, op = H.params(precision=1, cos_angle_min=COS20)
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
        st, pose, res = t.align(pr)
    ref = O.align(fr, mo, pr.model_pose, pr.prior_R, pr.init_pose, pr.lam, op)
    _check_against_oracle(pose, res, ref)


def test_fp16_form_matches_oracle_on_dequantised_maps():
    pr = S.config2_kinect(6)
    p, op = H.params(precision=1)
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
        st, pose, res = t.align(pr, 0.0)
    ref = O.align(fr, mo, pr.model_pose, pr.prior_R, pr.init_pose, 0.0, op)
    _check_against_oracle(pose, res, ref)


# ---------------------------------------------------------------------------
# batching, determinism, edge cases
# ---------------------------------------------------------------------------
def test_batch_equals_single_alignments_bit_for_bit():
    sizes = [(320, 240), (640, 480), (160, 120), (333, 251), (640, 480)]
    pairs = [S.config2_kinect(10 + i, *sz) for i, sz in enumerate(sizes)]
    p, op = H.params()
    ts = [H.Tracker(p, 640, 480) for _ in pairs]
    try:
        for t, pr in zip(ts, pairs):
            t.set_pair(pr)
        k = H.kf()
        st, poses, res = k.kf_align_batch([t.h for t in ts], np.stack([pr.prior_R for pr in pairs]),
                                          np.stack([pr.init_pose for pr in pairs]),
                                          np.array([pr.lam for pr in pairs]))
        for i, (t, pr) in enumerate(zip(ts, pairs)):
            st1, pose1, res1 = t.align(pr)
            assert np.array_equal(poses[i], pose1)
            assert list(res[i].iters) == list(res1.iters)
        # and the second batch call (cached plan and graph) repeats the first
        st2, poses2, _ = k.kf_align_batch([t.h for t in ts], np.stack([pr.prior_R for pr in pairs]),
                                          np.stack([pr.init_pose for pr in pairs]),
                                          np.array([pr.lam for pr in pairs]))
        assert np.array_equal(poses, poses2)
    finally:
        for t in ts:
            t.close()


def test_empty_frame_reports_too_few_inliers_and_returns_the_seed():
    pr = S.config1_tiny()
    p, op = H.params(levels=1, caps=(10,))
    with H.Tracker(p, 160, 120) as t:
        t.set_pair(pr, depth=np.zeros_like(pr.depth))
        st, pose, res = t.align(pr)
    assert st == O.TOO_FEW_INLIERS and res.status == st
    assert np.array_equal(pose, O.seed_pose(pr.prior_R, pr.init_pose, op))


def test_nan_depth_is_no_measurement():
    pr = S.config1_tiny()
    d = pr.depth.copy()
    d[::3, ::2] = np.nan
    d[1::7] = -1.0
    p, op = H.params(levels=1, caps=(10,))
    with H.Tracker(p, 160, 120) as t:
        t.set_pair(pr, depth=d)
        st, pose, res = t.align(pr)
    ref = O.align_from_depth(d, O.Cam(*pr.K.as_tuple()), pr.model_vertex, pr.model_normal,
                             O.Cam(*pr.K.as_tuple()), pr.model_pose, pr.prior_R, pr.init_pose,
                             pr.lam, op)
    rot, tr = H.pose_err(pose, ref.pose)
    assert st == ref.status and rot < 1e-5 and tr < 1e-5


def test_single_plane_is_degenerate_on_gpu():
    sc = S.Scene(planes=[((0.0, 0.0, -1.0), -2.0)])
    K = S.Intrinsics(40, 30, 35.0, 35.0, 19.5, 14.5)
    pr = S.make_pair(sc, K, S.rng_for(9, 20), 1.0, 0.01, 0.1, noise=False)
    p, op = H.params(levels=1, caps=(5,), bilateral_radius=0)
    with H.Tracker(p, 40, 30) as t:
        t.set_pair(pr)
        st, pose, res = t.align(pr, 0.0)
    assert st == O.DEGENERATE


def test_caps_and_flags():
    pr = S.config1_tiny()
    for caps, flags, want in [((2,), 7, O.NOT_CONVERGED), ((4,), 3, O.OK)]:
        p, op = H.params(levels=1, caps=caps, flags=flags)
        with H.Tracker(p, 160, 120) as t:
            t.set_pair(pr)
            st, pose, res = t.align(pr, 5.0)
        ref = O.align_from_depth(pr.depth, O.Cam(*pr.K.as_tuple()), pr.model_vertex,
                                 pr.model_normal, O.Cam(*pr.K.as_tuple()), pr.model_pose,
                                 pr.prior_R, pr.init_pose, 5.0, op)
        assert st == want == ref.status
        assert list(res.iters)[:1] == ref.iters == [caps[0]]


def test_lambda_schedules_match_oracle():
    pr = S.config2_kinect(7, 320, 240)
    for mode in range(5):
        p, op = H.params(lambda_mode=mode)
        with H.Tracker(p, 320, 240) as t:
            t.set_pair(pr)
            fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
            st, pose, res = t.align(pr, 2.0)
        ref = O.align(fr, mo, pr.model_pose, pr.prior_R, pr.init_pose, 2.0, op)
        _check_against_oracle(pose, res, ref)


def test_repeated_alignment_is_deterministic():
    pr = S.config2_kinect(8)
    p, op = H.params()
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        a = t.align(pr)[1]
        b = t.align(pr)[1]
    assert np.array_equal(a, b)


def test_invalid_calls_return_errors():
    k = H.kf()
    p, op = H.params()
    with H.Tracker(p, 160, 120) as t:
        with pytest.raises(k.KFError) as e:
            k.kf_align(t.h, None, np.eye(4), 1.0)
        assert e.value.status == k.KF_ERR_NO_FRAME
        with pytest.raises(k.KFError) as e:
            k.kf_set_frame(t.h, np.zeros((240, 320), np.float32).ctypes.data, (320, 240, 1, 1, 1, 1), False)
        assert e.value.status == k.KF_ERR_INVALID_ARG


def test_band_edge_window_hits_on_most_iterations_and_matches_oracle():
    """The association pass sums the rows of the pixels below the window in
    which it expects the band edge and records those inside it; when the new
    edge lands in the window (passes == 1) the reduction pass only adds the
    recorded rows. Either way the alignment follows the oracle. A band that
    does not start at bin 0 (kappa < 1) never takes the window."""
    sizes = [(320, 240), (640, 480), (160, 120), (333, 251)]
    pairs = [S.config2_kinect(20 + i, *sz) for i, sz in enumerate(sizes)]
    k = H.kf()
    for kappa in (1.0, 0.6):
        p, op = H.params(band_kappa=kappa)
        ts = [H.Tracker(p, 640, 480) for _ in pairs]
        try:
            for t, pr in zip(ts, pairs):
                t.set_pair(pr)
            fr_mo = [H.oracle_levels_from_gpu(t, pr, 3) for t, pr in zip(ts, pairs)]
            st, poses, res = k.kf_align_batch([t.h for t in ts], np.stack([pr.prior_R for pr in pairs]),
                                              np.stack([pr.init_pose for pr in pairs]),
                                              np.array([pr.lam for pr in pairs]))
            traces = [k.kf_debug_trace(t.h) for t in ts]
        finally:
            for t in ts:
                t.close()
        for i, pr in enumerate(pairs):
            fr, mo = fr_mo[i]
            ref = O.align(fr, mo, pr.model_pose, pr.prior_R, pr.init_pose, pr.lam, op, keep_trace=True)
            _check_against_oracle(poses[i], res[i], ref)
            assert [(r.klo, r.khi) for r in traces[i]] == [(r.klo, r.khi) for r in ref.trace]
        # each iteration's window comes from the band edge before it (the
        # alignment's first iteration has none); the band decides the way: the
        # recorded pixels only (passes 1) exactly when the band starts at bin 0
        # and its edge lies in [w0 - 1, w1 - 1]
        hit_px = all_px = 0
        for i, tr in enumerate(traces):
            lv_px = [(sizes[i][0] >> l) * (sizes[i][1] >> l) for l in range(3)]
            for j, r in enumerate(tr):
                if j == 0:
                    assert r.w0 == -1 and r.passes == 2
                elif kappa < 1.0:
                    assert r.w0 == -1 and r.passes == 2
                else:
                    g = tr[j - 1].khi   # the previous edge lies in the window made from it
                    assert r.w0 >= 0 and r.w0 - 1 <= g <= r.w1 - 1, (i, j, r.w0, r.w1, g)
                    want = 1 if (r.klo == 0 and r.w0 - 1 <= r.khi <= r.w1 - 1) else 2
                    assert r.passes == want, (i, j, r.w0, r.w1, r.khi)
                hit_px += lv_px[r.level] * (r.passes == 1)
                all_px += lv_px[r.level]
        if kappa == 1.0:
            assert hit_px > 0.75 * all_px, (hit_px, all_px)


def _align_mixed_batch(flags, pairs, depths):
    k = H.kf()
    p, op = H.params(flags=flags)
    ts = [H.Tracker(p, 640, 480) for _ in pairs]
    try:
        for t, pr, dep in zip(ts, pairs, depths):
            t.set_pair(pr, depth=dep)
        st, poses, res = k.kf_align_batch([t.h for t in ts], np.stack([pr.prior_R for pr in pairs]),
                                          np.stack([pr.init_pose for pr in pairs]),
                                          np.array([pr.lam for pr in pairs]))
        traces = [k.kf_debug_trace(t.h) for t in ts]
        fr_mo = [H.oracle_levels_from_gpu(t, pr, 3) for t, pr in zip(ts, pairs)]
    finally:
        for t in ts:
            t.close()
    return st, poses, res, traces, fr_mo, op


def _trace_key(r):
    return (r.level, r.iter, r.N, r.kmed, r.klo, r.khi, r.n, r.passes, r.lambda_, tuple(r.x))


def test_scheduled_launch_equals_per_iteration_launches_bit_for_bit():
    """The default persistent launch (pairs advance independently) and one
    launch per stage and iteration give the same bits: same items, same
    fixed-order sums, same solve. The batch mixes sizes (ragged 333x251), an
    empty frame (stops at its first median) and more pairs than one ring of
    the queue holds over a whole alignment (the ring wraps)."""
    sizes = [(320, 240), (640, 480), (160, 120), (333, 251), (640, 480)] * 4
    pairs = [S.config2_kinect(40 + i, *sz) for i, sz in enumerate(sizes)]
    depths = [pr.depth for pr in pairs]
    depths[6] = np.zeros_like(depths[6])
    k = H.kf()
    a = _align_mixed_batch(7, pairs, depths)
    b = _align_mixed_batch(7 | k.KF_LAUNCH_PER_ITERATION, pairs, depths)
    assert a[0] == b[0] == O.TOO_FEW_INLIERS
    assert np.array_equal(a[1], b[1])
    for ra, rb, ta, tb in zip(a[2], b[2], a[3], b[3]):
        assert ra.status == rb.status and list(ra.iters) == list(rb.iters)
        assert list(ra.median_bin) == list(rb.median_bin)
        assert (ra.inliers, ra.valid_pairs, ra.rms_residual) == (rb.inliers, rb.valid_pairs, rb.rms_residual)
        assert [_trace_key(r) for r in ta] == [_trace_key(r) for r in tb]
    seed = pairs[6].init_pose.copy()
    seed[:3, :3] = pairs[6].prior_R
    assert a[2][6].status == O.TOO_FEW_INLIERS and np.array_equal(a[1][6], seed)
    # and both match the oracle on the sampled pairs
    for i in (0, 3, 6, 9):
        fr, mo = a[4][i]
        ref = O.align(fr, mo, pairs[i].model_pose, pairs[i].prior_R, pairs[i].init_pose, pairs[i].lam, a[5])
        _check_against_oracle(a[1][i], a[2][i], ref)


def test_scheduled_launch_profile_counts_one_launch_per_alignment():
    pr = S.config2_kinect(3, 320, 240)
    p, op = H.params()
    k = H.kf()
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        k.kf_profile_enable(t.h, 1)
        for _ in range(3):
            t.align(pr)
        prof = k.kf_profile_read(t.h)
        k.kf_profile_enable(t.h, 0)
    assert prof.sched_launches == 3 and prof.graph_launches == 3
    assert prof.assoc_launches == prof.reduce_launches == 0
    assert 0 < prof.sched_ms <= prof.align_ms


def test_bounded_device_waits_run_out_and_report_timeout():
    """Failure detection without a fault: an empty scheduled launch never
    queues a task, so every block's bounded wait for its next task runs out;
    the launch ends by itself with its error word set, the call returns
    KF_ERR_TIMEOUT, and the context and tracker stay usable."""
    import time
    k = H.kf()
    pr = S.config1_tiny()
    p, op = H.params(levels=1, caps=(10,))
    with H.Tracker(p, 160, 120) as t:
        t0 = time.perf_counter()
        assert k.kf_debug_wait_timeout(t.h, 20.0) == k.KF_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 1)
        st, pose, res = t.align(pr)
    ref = O.align(fr, mo, pr.model_pose, pr.prior_R, pr.init_pose, pr.lam, op)
    _check_against_oracle(pose, res, ref)


def test_original_kinectfusion_mode_matches_oracle():
    """The ablation baseline of the paper's timing comparison: no IMU seed, no
    median filter, no convergence rule, lambda = 0, fixed 4/5/10 iterations
    coarse to fine; and the paper's mode with the shorter (2,2,3) cadence."""
    pr = S.config2_kinect(11, 320, 240)
    for caps, flags, lam in [((10, 5, 4), 0, 0.0), ((3, 2, 2), 7, pr.lam)]:
        p, op = H.params(caps=caps, flags=flags)
        with H.Tracker(p, 320, 240) as t:
            t.set_pair(pr)
            fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
            st, pose, res = t.align(pr, lam, prior=bool(flags & 1))
        ref = O.align(fr, mo, pr.model_pose, pr.prior_R if flags & 1 else None, pr.init_pose, lam, op)
        _check_against_oracle(pose, res, ref)
        if flags == 0:
            assert list(res.iters)[:3] == [10, 5, 4] and res.status == O.OK


def test_large_rotation_needs_the_imu_seed():
    """Sec. 4.2's claim on one 30 deg pair (synthetic): seeded with the IMU
    orientation the alignment converges, from the previous pose it fails;
    both runs match the oracle."""
    pr = S.angular_case(3, 0, 320, 240)
    for flags, prior, lam in [(7, True, pr.lam), (6, False, 0.0)]:
        p, op = H.params(flags=flags)
        with H.Tracker(p, 320, 240) as t:
            t.set_pair(pr)
            fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
            st, pose, res = t.align(pr, lam, prior=prior)
        ref = O.align(fr, mo, pr.model_pose, pr.prior_R if prior else None, pr.init_pose, lam, op)
        _check_against_oracle(pose, res, ref)
        rot, tr = H.pose_err(pose, pr.gt_pose)
        if prior:
            assert math.degrees(rot) < 1.0 and tr < 0.02, (rot, tr)
        else:
            assert math.degrees(rot) > 5.0 or tr > 0.1, (rot, tr)


def test_prior_anchored_variant_matches_oracle():
    """Regulariser anchored to the IMU prior (KF_PRIOR_ANCHORED): seeded from
    the prior and from the previous pose (the anchor then pulls the rotation
    to the prior), several lambdas; scheduled and per-iteration launches."""
    k = H.kf()
    pr = S.config2_kinect(13, 320, 240)
    for base, lam in [(7, 5.0), (7, 1e3), (6, 50.0)]:
        for extra in (0, k.KF_LAUNCH_PER_ITERATION):
            flags = base | k.KF_PRIOR_ANCHORED | extra
            p, op = H.params(flags=flags)
            with H.Tracker(p, 320, 240) as t:
                t.set_pair(pr)
                fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
                st, pose, res = t.align(pr, lam)
            op.flags = base | O.PRIOR_ANCHORED
            ref = O.align(fr, mo, pr.model_pose, pr.prior_R, pr.init_pose, lam, op)
            _check_against_oracle(pose, res, ref)


def test_page_locked_host_frames_are_read_in_place_with_the_same_result():
    """Host frames in page-locked memory are read by the front-end kernel over
    the host link instead of being copied first; pageable host frames are
    copied; device frames are read in place; with KF_FRAME_HOST_COPY_ENGINE
    page-locked and pageable frames are copied into a staging buffer, one
    copy per run of frames that follow one another in host memory (frames
    apart, all back to back, two of three back to back; and a first call with
    one frame, so that the second call grows the buffer). All give the same
    maps and the same alignments, bit for bit."""
    import torch
    k = H.kf()
    pairs = [S.config2_kinect(80 + i, *sz) for i, sz in enumerate([(640, 480), (333, 251), (320, 240)])]
    p, op = H.params()
    out = {}
    mode = {"pageable": k.KF_FRAME_HOST, "pinned": k.KF_FRAME_HOST, "device": k.KF_FRAME_DEVICE,
            "pinned_copy_engine": k.KF_FRAME_HOST_COPY_ENGINE,
            "pageable_copy_engine": k.KF_FRAME_HOST_COPY_ENGINE,
            "pinned_flat_copy_engine": k.KF_FRAME_HOST_COPY_ENGINE,
            "pageable_flat_copy_engine": k.KF_FRAME_HOST_COPY_ENGINE,
            "pinned_two_runs_copy_engine": k.KF_FRAME_HOST_COPY_ENGINE,
            "pinned_flat_grow_copy_engine": k.KF_FRAME_HOST_COPY_ENGINE}
    flat32 = [np.ascontiguousarray(pr.depth, np.float32).reshape(-1) for pr in pairs]
    for kind in mode:
        ts = [H.Tracker(p, 640, 480) for _ in pairs]
        keep = []
        try:
            for t, pr in zip(ts, pairs):
                t.set_pair(pr)  # model (and a first frame)
            if "flat" in kind or "two_runs" in kind:
                # frames back to back in one buffer (two_runs: a gap before the third)
                gap = 64 if "two_runs" in kind else 0
                whole = np.zeros(sum(f.size for f in flat32) + gap, np.float32)
                offs, o = [], 0
                for i, f in enumerate(flat32):
                    o += gap if i == 2 else 0
                    whole[o:o + f.size] = f
                    offs.append(o)
                    o += f.size
                if kind.startswith("pinned"):
                    buf = torch.from_numpy(whole).pin_memory()
                    base = buf.data_ptr()
                else:
                    buf = whole
                    base = whole.ctypes.data
                bufs = [buf]
                ptrs = [base + 4 * o for o in offs]
                if "grow" in kind:  # a smaller batch first: the next call grows the staging buffer
                    k.kf_set_frame_batch([ts[0].h], ptrs[:1], [pairs[0].K.as_tuple()], mode[kind])
            elif kind.startswith("pageable"):
                bufs = [np.ascontiguousarray(pr.depth, np.float32) for pr in pairs]
                ptrs = [b.ctypes.data for b in bufs]
            elif kind.startswith("pinned"):
                bufs = [torch.from_numpy(np.ascontiguousarray(pr.depth, np.float32)).pin_memory() for pr in pairs]
                ptrs = [b.data_ptr() for b in bufs]
            else:
                bufs = [torch.from_numpy(np.ascontiguousarray(pr.depth, np.float32)).cuda() for pr in pairs]
                torch.cuda.synchronize()
                ptrs = [b.data_ptr() for b in bufs]
            keep.append(bufs)
            k.kf_set_frame_batch([t.h for t in ts], ptrs, [pr.K.as_tuple() for pr in pairs], mode[kind])
            torch.cuda.synchronize()
            st, poses, res = k.kf_align_batch([t.h for t in ts], np.stack([pr.prior_R for pr in pairs]),
                                              np.stack([pr.init_pose for pr in pairs]),
                                              np.array([pr.lam for pr in pairs]))
            maps = [k.kf_debug_frame_level(t.h, 0) for t in ts]
        finally:
            for t in ts:
                t.close()
        out[kind] = (poses, [list(r.iters) for r in res], maps)
    for kind in mode:
        assert np.array_equal(out[kind][0], out["pageable"][0]), kind
        assert out[kind][1] == out["pageable"][1], kind
        for (Da, Va, Na), (Db, Vb, Nb) in zip(out[kind][2], out["pageable"][2]):
            assert np.array_equal(Da, Db)
            assert np.array_equal(Va, Vb, equal_nan=True) and np.array_equal(Na, Nb, equal_nan=True)
