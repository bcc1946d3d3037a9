"""Test helpers: drive the C ABI with synthetic pairs and run the oracle on the
same inputs (or on the maps the GPU built, for per-stage parity)."""
from __future__ import annotations

import math

import numpy as np

from oracle import kf_oracle as O


def kf():
    import paper_1802_03980_gb300 as m
    return m


def params(levels=3, caps=(10, 5, 4), **kw):
    """C-ABI params and the matching oracle params."""
    k = kf()
    p = k.kf_default_params()
    p.levels = levels
    for i, c in enumerate(caps):
        p.max_iters[i] = c
    for name, v in kw.items():
        setattr(p, name, v)
    op = O.Params(levels=levels, max_iters=tuple(caps), hist_bins=p.hist_bins, d_max=p.d_max,
                  band_kappa=p.band_kappa, cos_angle_min=p.cos_angle_min,
                  conv_window=p.conv_window, lambda_mode=p.lambda_mode, lambda_c=p.lambda_c,
                  n_min=p.n_min, flags=p.flags, bilateral_sigma_s=p.bilateral_sigma_s,
                  bilateral_sigma_r=p.bilateral_sigma_r, bilateral_radius=p.bilateral_radius,
                  normal_mode=p.normal_mode, ii_radius_a=p.ii_radius_a, ii_radius_b=p.ii_radius_b,
                  ii_depth_change=p.ii_depth_change, ii_radius_max=p.ii_radius_max,
                  shoot_radius=p.shoot_radius)
    return p, op


class Tracker:
    """Owns one C-ABI tracker; uploads a FramePair's frame and model."""

    def __init__(self, p, max_w, max_h, stream=0):
        self.k = kf()
        self.h = self.k.kf_track_create(p, max_w, max_h, stream)
        self.p = p

    def close(self):
        if self.h is not None:
            self.k.kf_track_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_pair(self, pr, depth=None, device=False):
        import torch
        K = pr.K.as_tuple()
        d = np.ascontiguousarray(pr.depth if depth is None else depth, np.float32)
        if device:
            td = torch.from_numpy(d).cuda()
            torch.cuda.synchronize()   # the tracker's stream does not order after torch's
            self.k.kf_set_frame(self.h, td.data_ptr(), K, True)
            torch.cuda.synchronize()
        else:
            self.k.kf_set_frame(self.h, d.ctypes.data, K, False)
        mv = np.ascontiguousarray(pr.model_vertex, np.float32)
        mn = np.ascontiguousarray(pr.model_normal, np.float32)
        self.k.kf_set_model(self.h, mv.ctypes.data, mn.ctypes.data, pr.model_pose, K, False)

    def align(self, pr, lam=None, prior=True):
        return self.k.kf_align(self.h, pr.prior_R if prior else None, pr.init_pose,
                               pr.lam if lam is None else lam)

    def frame_levels(self, levels):
        out = []
        for l in range(levels):
            D, V, N = self.k.kf_debug_frame_level(self.h, l)
            out.append((D, V, N))
        return out

    def model_levels(self, levels):
        return [self.k.kf_debug_model_level(self.h, l) for l in range(levels)]


def oracle_levels_from_gpu(trk: Tracker, pr, levels):
    """Oracle level objects holding exactly the maps the GPU built."""
    fc = O.frame_level_cams(O.Cam(*pr.K.as_tuple()), levels)
    mc = O.model_level_cams(O.Cam(*pr.K.as_tuple()), levels)
    fr = [O.frame_level_from_maps(D, V, N, fc[l]) for l, (D, V, N) in enumerate(trk.frame_levels(levels))]
    mo = [O.ModelLevel(np.asarray(V, np.float64), np.asarray(N, np.float64), mc[l])
          for l, (V, N) in enumerate(trk.model_levels(levels))]
    return fr, mo


def pose_err(A, B):
    return O.rotation_angle(A[:3, :3], B[:3, :3]), float(np.linalg.norm(A[:3, 3] - B[:3, 3]))


def sum_tolerances(a_rows, b, pos_eps=3e-6, rel=1e-5):
    """Per-sum tolerance of the 29 float32 sums against the float64 oracle.

    rel * sum |term| covers float32 accumulation; pos_eps (metres) covers the
    float32 rounding of the transformed points that b and p x n are built from.
    """
    terms = []
    for r in range(6):
        for c in range(r, 6):
            terms.append((np.abs(a_rows[:, r] * a_rows[:, c]).sum(),
                          pos_eps * (np.abs(a_rows[:, r]).sum() + np.abs(a_rows[:, c]).sum())))
    for r in range(6):
        terms.append((np.abs(a_rows[:, r] * b).sum(),
                      pos_eps * (np.abs(a_rows[:, r]).sum() + np.abs(b).sum())))
    terms.append((0.0, 0.0))
    terms.append(((b * b).sum(), 2 * pos_eps * np.abs(b).sum()))
    return np.array([rel * s + e for s, e in terms])


def oracle_sums(a: O.Assoc, inl):
    A, b = O.ls_rows(a.p[inl], a.q[inl], a.n[inl])
    AtA, Atb, sb2 = O.normal_equations(A, b)
    up = [AtA[r, c] for r in range(6) for c in range(r, 6)]
    return np.array(up + list(Atb) + [float(inl.sum()), sb2]), A, b


def deg(x):
    return math.degrees(x)
