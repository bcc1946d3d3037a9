"""kf_reduce_noalloc: the reduction for callers that cannot allocate device memory.

Some callers run inside a host application whose CUDA allocator belongs to
another runtime, or may not add cudaMalloc / cudaFree synchronisation while
their other work is in flight; this entry point works on their buffers only and
keeps its scratch in a fixed array inside the library. The test feeds it the
maps a tracker built and checks its sums against the tracker's own reduction
entry point (kf_debug_reduce), on two calls in a row, within the tolerance the
other reduction tests use. The file name makes pytest collect it last.
"""
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


def test_noalloc_reduction_matches_the_tracker_reduction_on_two_calls():
    import torch
    k = H.kf()
    pr = S.config2_kinect(3, 640, 480)
    p, op = H.params()
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
        T = O.seed_pose(pr.prior_R, pr.init_pose, op)
        for l in (0, 1):
            a = O.associate(fr[l], mo[l], T, O.f32_transforms(T, pr.model_pose), op)
            kmed = O.median_bin(O.histogram(a, p.hist_bins))
            klo, khi = O.band(kmed, 1.0, p.hist_bins)
            want = k.kf_debug_reduce(t.h, l, T, klo, khi)
            _, A, bb = H.oracle_sums(a, a.valid & (a.k >= klo) & (a.k <= khi))
            tol = H.sum_tolerances(A, bb)
            fv = torch.from_numpy(np.ascontiguousarray(fr[l].V, np.float32)).cuda()
            mv = torch.from_numpy(np.ascontiguousarray(mo[l].V, np.float32)).cuda()
            mn = torch.from_numpy(np.ascontiguousarray(mo[l].N, np.float32)).cuda()
            out = torch.full((2, 29), float("nan"), dtype=torch.float64, device="cuda")
            mc = mo[l].cam
            h, w = fr[l].V.shape[:2]
            torch.cuda.synchronize()
            for call in range(2):
                st = k.kf_reduce_noalloc(fv.data_ptr(), w, h, mv.data_ptr(), mn.data_ptr(),
                                         (mc.width, mc.height, mc.fx, mc.fy, mc.cx, mc.cy), T,
                                         pr.model_pose, p.d_max, p.hist_bins, klo, khi,
                                         out[call].data_ptr(), 0)
                assert st == k.KF_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for call in range(2):
                assert got[call][27] == want[27]
                assert (np.abs(got[call] - want) <= tol).all(), (l, call)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    k = H.kf()
    st = k.kf_reduce_noalloc(1, 4096, 1025, 1, 1, (64, 48, 50.0, 50.0, 32.0, 24.0), np.eye(4),
                             np.eye(4), 0.16, 512, 0, 10, 1, 0)
    assert st == k.KF_ERR_SCRATCH_LIMIT
