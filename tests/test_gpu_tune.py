"""The autotuner end to end on a small sweep.

Two candidates of the association pass's pixels per thread are built,
timed on a batch of six 320x240 pairs and checked against poses the FP64
oracle computes from the same depth frames (1e-5 rad, 1e-5 m); the winner is
written to a tuned file whose defines build() would compile with.
"""
import json
import os
import tempfile

import numpy as np
import pytest

from oracle import kf_oracle as O
from synth import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03980_gb300 import build
    build()


def test_mini_sweep_builds_times_checks_and_writes_the_winner():
    from paper_1802_03980_gb300 import tune
    pairs, w, h = 6, 320, 240
    op = O.Params()
    ref = []
    for i in range(pairs):  # the tuner's workload: config2_kinect(1000 + i) at w x h
        pr = S.config2_kinect(1000 + i, w, h)
        c = O.Cam(*pr.K.as_tuple())
        r = O.align_from_depth(pr.depth, c, pr.model_vertex, pr.model_normal, c, pr.model_pose,
                               pr.prior_R, pr.init_pose, pr.lam, op)
        ref.append(r.pose)
    grid = {"KF_ASSOC_U": [4, 2]}
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "tuned.json")
        res = tune.sweep(grid=grid, pairs=pairs, width=w, height=h, steps=2, warmup=1,
                         reference=np.array(ref), out=out, workdir=tmp, log=lambda *_: None)
        rows = res["candidates"]
        assert [r["defines"] for r in rows] == tune.candidates(grid)
        for r in rows:
            assert r["built"] and r["valid"], r
            assert r["max_rot_rad"] < 1e-5 and r["max_trans_m"] < 1e-5
            assert r["launch_ms"] > 0
        best = min(rows, key=lambda r: r["launch_ms"])
        assert res["defines"] == best["defines"]
        with open(out) as f:
            assert json.load(f)["defines"] == best["defines"]
        assert tune.tuned_defines(out) == [f"{k}={v}" for k, v in sorted(best["defines"].items())]
