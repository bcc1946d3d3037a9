"""The guarded build (-DKF_CHECKED) on the GPU.

In place of a memory checker run, the library has a checked build: every
guarded index (work-item partials, per-pixel buffers,
active lists, record regions and counts) is tested before its access, and a violation
records its code and values in a device word and skips the access; the host
turns it into KF_ERR_INTERNAL. This test builds that library to a temporary
path, aligns the mixed batch of the scheduled-launch test (ragged 333x251,
an empty frame, enough pairs to wrap the queue's ring) in a child process
that loads it, and checks that no guard fired and that the poses equal the
unguarded build's bit for bit. The checked library is built with
KF_FUSE_GRID_DIV=100000, so its scheduled launch runs every hit's reduction
pass inside the pair's median epilogue (fixup_all), while the unguarded
build, with this batch's 20 pairs below its threshold, spreads it over
reduction tasks: the equal poses also show that the two ways give the same
bits.
"""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from synth import scenes as S
from tests import kfhelp as H

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
from synth import scenes as S
from tests import kfhelp as H
from tests.test_gpu_checked import batch_inputs, align_batch
pairs, depths = batch_inputs()
out = {{}}
for flags in (7, 7 | 16):
    st, poses, res = align_batch(flags, pairs, depths)
    out[str(flags)] = dict(status=int(st), poses=poses.tolist(),
                           iters=[list(r.iters) for r in res])
print("RESULT " + json.dumps(out))
"""


def batch_inputs():
    sizes = [(320, 240), (640, 480), (160, 120), (333, 251), (640, 480)] * 4
    pairs = [S.config2_kinect(40 + i, *sz) for i, sz in enumerate(sizes)]
    depths = [pr.depth for pr in pairs]
    depths[6] = np.zeros_like(depths[6])
    return pairs, depths


def align_batch(flags, pairs, depths):
    k = H.kf()
    p, _ = H.params(flags=flags)
    ts = [H.Tracker(p, 640, 480) for _ in pairs]
    try:
        for t, pr, dep in zip(ts, pairs, depths):
            t.set_pair(pr, depth=dep)
        st, poses, res = k.kf_align_batch([t.h for t in ts], np.stack([pr.prior_R for pr in pairs]),
                                          np.stack([pr.init_pose for pr in pairs]),
                                          np.array([pr.lam for pr in pairs]))
    finally:
        for t in ts:
            t.close()
    return st, poses, res


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03980_gb300 import build
    build()


def test_checked_build_records_no_violation_and_matches_the_unguarded_build():
    from paper_1802_03980_gb300 import build
    k = H.kf()
    with tempfile.TemporaryDirectory() as tmp:
        lib = build(defines=["KF_CHECKED", "KF_FUSE_GRID_DIV=100000"],
                    out=os.path.join(tmp, "libkftrack_checked.so"))
        env = dict(os.environ, KF_TRACK_LIB=lib)
        r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    got = json.loads(line[len("RESULT "):])
    pairs, depths = batch_inputs()
    for flags in (7, 7 | k.KF_LAUNCH_PER_ITERATION):
        st, poses, res = align_batch(flags, pairs, depths)
        g = got[str(flags)]
        # a guard that fired would turn the batch's status into KF_ERR_INTERNAL
        assert g["status"] == st == k.KF_ERR_TOO_FEW_INLIERS, (g["status"], st)
        assert np.array_equal(np.array(g["poses"]), poses)
        assert g["iters"] == [list(r.iters) for r in res]
