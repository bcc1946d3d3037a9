"""Accuracy of the 29 normal-equation sums: plain float32 per-thread sums
against compensated (Kahan) ones, both combined across warps and items in
FP64.

The library's per-thread sums are plain fused multiply-adds. A build with
-DKF_KAHAN=1 compensates them (a second register per sum carries the lost
low-order part). This test builds that library to a temporary path and
computes, for the same 640x480 pairs, levels, poses and bands, the sums of
kf_debug_reduce with both libraries (the compensated one in a child process
that loads it), and two errors per sum, each relative to the sum of the
absolute values of its terms:

* accumulation error: against the FP64 sum of the very float32 rows the
  kernel forms (p = R v + t and the rows of Eq. 3 evaluated in float32 in the
  kernel's operation order, each fused multiply-add emulated with an exact
  float64 product), so only the summation's rounding remains;
* error against the definition: against the oracle's FP64 sums (rows from
  FP64 points), which adds the float32 rounding of the points and rows.

It also times one scheduled launch of a 32-pair 640x480 batch with each
library. The figures are printed as one line starting with KAHAN.
"""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from oracle import kf_oracle as O
from synth import scenes as S
from tests import kfhelp as H

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F32 = np.float32

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
from tests.test_gpu_kahan import sum_errors
print("RESULT " + json.dumps(sum_errors()))
"""


def _fmaf(x, y, z):
    """float32 fused multiply-add: the float64 product of two float32 values
    is exact; the addition and the final rounding may round twice (an error
    of one float32 ulp in rare rows, far below what is measured here)."""
    return (x.astype(np.float64) * y.astype(np.float64) + z.astype(np.float64)).astype(F32)


def kernel_rows32(p, q, n):
    """The rows of Eq. 3 as the kernel evaluates them in float32:
    a = [p x n, n] with each component fma(p_i, n_j, -(p_k n_l)),
    b = fma(n0, q0 - p0, fma(n1, q1 - p1, n2 (q2 - p2)))."""
    p, q, n = p.astype(F32), q.astype(F32), n.astype(F32)
    a = np.empty((p.shape[0], 6), F32)
    a[:, 0] = _fmaf(p[:, 1], n[:, 2], -(p[:, 2] * n[:, 1]))
    a[:, 1] = _fmaf(p[:, 2], n[:, 0], -(p[:, 0] * n[:, 2]))
    a[:, 2] = _fmaf(p[:, 0], n[:, 1], -(p[:, 1] * n[:, 0]))
    a[:, 3:] = n
    d = q - p
    b = _fmaf(n[:, 0], d[:, 0], _fmaf(n[:, 1], d[:, 1], n[:, 2] * d[:, 2]))
    return a, b


def _sums_and_scale(A, b):
    """The 29 sums in FP64 and, per sum, the sum of its terms' magnitudes."""
    A = A.astype(np.float64)
    b = b.astype(np.float64)
    s, m = [], []
    for r in range(6):
        for c in range(r, 6):
            t = A[:, r] * A[:, c]
            s.append(t.sum())
            m.append(np.abs(t).sum())
    for r in range(6):
        t = A[:, r] * b
        s.append(t.sum())
        m.append(np.abs(t).sum())
    s.append(float(A.shape[0]))
    m.append(float(A.shape[0]))
    s.append((b * b).sum())
    m.append((b * b).sum())
    return np.array(s), np.array(m)


def sum_errors(cases=(3, 5), levels=3):
    """Per-sum relative errors of kf_debug_reduce (the library loaded in this
    process) against both references, over cases x levels x two poses x three
    bands (the median band, the whole histogram, a band not starting at bin
    0: the last one sums by re-association, the others split rows between the
    association pass and the recorded band edge)."""
    k = H.kf()
    acc, dfn, within = [], [], True
    for case in cases:
        pr = S.config2_kinect(case, 640, 480)
        p, op = H.params()
        with H.Tracker(p, 640, 480) as t:
            t.set_pair(pr)
            fr, mo = H.oracle_levels_from_gpu(t, pr, levels)
            T0 = O.seed_pose(pr.prior_R, pr.init_pose, op)
            T1 = O.apply_increment(np.array([0.004, -0.003, 0.002, 0.01, -0.008, 0.005]), T0)
            for l in range(levels):
                for T in (T0, T1):
                    xf = O.f32_transforms(T, pr.model_pose)
                    a = O.associate(fr[l], mo[l], T, xf, op)
                    kmed = O.median_bin(O.histogram(a, p.hist_bins))
                    for klo, khi in [O.band(kmed, 1.0, p.hist_bins), (0, p.hist_bins - 1),
                                     (3, max(3, kmed))]:
                        inl = a.valid & (a.k >= klo) & (a.k <= khi)
                        got = k.kf_debug_reduce(t.h, l, T, klo, khi)
                        want, A64, b64 = H.oracle_sums(a, inl)
                        within &= bool((np.abs(got - want) <= H.sum_tolerances(A64, b64)).all())
                        V32 = fr[l].V[inl].astype(F32)
                        p32 = np.stack(O._xform32(xf.Rw, xf.tw, V32[:, 0], V32[:, 1], V32[:, 2]), -1)
                        A32, b32 = kernel_rows32(p32, a.q[inl], a.n[inl])
                        s32, m32 = _sums_and_scale(A32, b32)
                        _, m64 = _sums_and_scale(A64, b64)
                        keep = np.arange(29) != 27  # the count is exact on both sides
                        acc.extend((np.abs(got - s32) / np.maximum(m32, 1e-300))[keep].tolist())
                        dfn.extend((np.abs(got - want) / np.maximum(m64, 1e-300))[keep].tolist())
                        assert got[27] == want[27]
    acc, dfn = np.array(acc), np.array(dfn)
    return dict(within_tolerance=within, n=int(acc.size),
                acc_max=float(acc.max()), acc_median=float(np.median(acc)),
                acc_rms=float(np.sqrt((acc ** 2).mean())),
                def_max=float(dfn.max()), def_median=float(np.median(dfn)),
                acc=acc.tolist())


def _time_launch(lib: str, data: str) -> dict:
    env = dict(os.environ, KF_TRACK_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "paper_1802_03980_gb300.tune", "--worker", data,
                        "--steps", "5", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads([x for x in r.stdout.splitlines() if x.startswith("TUNE ")][-1][5:])


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03980_gb300 import build
    build()


def test_compensated_sums_against_plain_sums():
    from paper_1802_03980_gb300 import build, tune
    from paper_1802_03980_gb300.build import LIB
    plain = sum_errors()
    with tempfile.TemporaryDirectory() as tmp:
        lib = build(defines=["KF_KAHAN=1"], out=os.path.join(tmp, "libkftrack_kahan.so"))
        env = dict(os.environ, KF_TRACK_LIB=lib)
        r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-2000:]
        kahan = json.loads([x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1][7:])
        data = os.path.join(tmp, "batch.npz")
        tune.make_batch(data, 32, 640, 480)
        tp, tk = _time_launch(LIB, data), _time_launch(lib, data)
    assert plain["within_tolerance"] and kahan["within_tolerance"]
    assert plain["n"] == kahan["n"]
    # both are float32 sums combined in FP64: far inside the tolerance's 1e-5
    assert plain["acc_max"] < 1e-6 and kahan["acc_max"] < 1e-6
    pa, ka = np.array(plain.pop("acc")), np.array(kahan.pop("acc"))
    rot, tr = tune._pose_err(np.array(tk["poses"]), np.array(tp["poses"]))
    summary = dict(plain=plain, kahan=kahan,
                   kahan_smaller=float((ka < pa).mean()), kahan_equal=float((ka == pa).mean()),
                   launch_ms=dict(plain=tp["launch_ms"], kahan=tk["launch_ms"]),
                   poses_kahan_vs_plain=dict(rot_rad=rot, trans_m=tr))
    print("KAHAN " + json.dumps(summary))
    # the compensated build aligns to the same poses within the parity bar
    assert rot < 1e-5 and tr < 1e-5
